// md_neigh.cu -- Verlet neighbor list by binning (paper, Section "Neighbor
// List Creation": "traditional binning methods used in many MD applications
// (Verlet lists)", stored in a dense padded format).
//
// One warp per cell, home atoms in batches of 32.  For a batch, the warp
// takes the bounding box of its home atoms' FP32 shadows and stages the
// candidates of the cell's 27-cell stencil into its own shared-memory window,
// slot by slot in stencil order, 32 candidates of a slot at a time: FP32
// coordinates relative to the box's centre (the cell-local shadow plus the
// slot's offset, the centre folded into the offset), leaving out those
// farther than rs from the box (about half of them at liquid density).  It then takes the
// window 64 candidates at a time: each lane holds two and tests them against
// every home atom (a broadcast read), one ballot per home atom and candidate
// half, which lands in that atom's lane as a 32-bit accept mask (through
// shared memory); each lane then writes its atom's accepted candidates, in
// window order, into the atom's row of the warp-transposed padded list.  Rows
// thus list the neighbor cells in stencil order, each cell's atoms together,
// the order the force kernel's gathers read best.  A second kernel then writes
// the sentinel entry into the slots past each atom's count up to its
// warp-tile's longest row (the rows of padding slots hold it from the list's
// allocation on).
//
// Decision rule (bit-exact with the FP64 definition): a pair is a neighbor iff
// the nearest-image FP64 distance r^2 = (dx*dx + dy*dy) + dz*dz, every op
// rounded separately, is < (rc+skin)^2 = rs^2.  The FP32 test evaluates
// r^2 = |c|^2 + |h|^2 - 2 c.h for the staged candidate c and home atom h
// (|h|^2 and -2 h kept per home atom, |c|^2 per candidate: one add and three
// FMAs per pair).  It differs from the FP64 r^2 by less than 8e-6 rs^2: with
// u = 2^-24, cell edge h < 1.5 rs, shadows refreshed at the sort (|shadow| <=
// h/2) and staged candidates within rs of the box, a component of c - h
// carries at most u (h/2 + h/2 + h + 1.5 h + h/2 + rs + h/2) <= 7.75 u rs (the
// two shadows, the FP32 cell edge, the shifted offset, the staged candidate,
// the shifted home atom), so the exact |c - h|^2 near rs^2 is off by at most
// 2 sqrt(3) rs 7.75 u rs < 27 u rs^2; and with |c| components <= 1.75 rs and
// |h| components <= 0.75 rs, the roundings of |c|^2, |h|^2, their sum and the
// three FMAs add at most (27.6 + 5.1 + 10.9 + 3 * 18.75) u rs^2 < 100 u rs^2.
// Candidates with FP32 r^2 outside [rs^2 - band, rs^2 + band], band = 3e-5
// rs^2 (> 500 u rs^2), are decided in FP32; the few inside are re-tested with
// the exact FP64 rule on the wrapped FP64 positions.  When an axis has only 2
// cells, the -1 and +1 stencil slots hold the same cell under two images; only
// one image can lie within rs (L > 2 rs), and the FP64 re-test checks that the
// slot's image is the nearest one.
#include <algorithm>

#include "md_common.cuh"

namespace mdb {
namespace {

constexpr int kWarps = 4;       // cells per CTA (one warp each)
// Kept candidates staged per warp per window (a multiple of 64): a typical
// stencil at liquid density (~300 kept of ~550) takes two windows; 256 leaves
// room for 8 resident CTAs per SM.
#ifndef MD_BUILD_CAND
#define MD_BUILD_CAND 256
#endif
constexpr int kCand = MD_BUILD_CAND;
static_assert(kCand % 64 == 0 && kCand >= 64, "windows are tested 64 candidates at a time");

struct BuildArgs {
    const Box *boxes;
    const int32_t *cell_box;
    const int32_t *cstart;
    const float4 *sh;
    const double *xws;
    int64_t ns;
    int32_t ncell;
    double rs2;
    float rs2f, bandf;
    int pad, R;
    int half;  // 1: keep pair (i, j) only if j's cell is forward of i's (code > 13) or
               // it is i's cell and j comes after i
    int32_t *nn;
    uint32_t *nbr;
    Flags *fl;
};

__device__ __forceinline__ bool exact_test(const BuildArgs &a, const Box &B, int64_t i, int64_t j,
                                           float dfx, float dfy, float dfz) {
    const float df[3] = {dfx, dfy, dfz};
    double d[3];
    bool same_image = true;
    for (int ax = 0; ax < 3; ++ax) {
        const double L = B.L[ax];
        const double h = 0.5 * L;
        double t = __dsub_rn(a.xws[ax * a.ns + j], a.xws[ax * a.ns + i]);
        if (t > h) t = __dsub_rn(t, L);
        else if (t < -h) t = __dadd_rn(t, L);
        d[ax] = t;
        same_image &= fabs(t - (double)df[ax]) < 1.0;
    }
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                __dmul_rn(d[2], d[2]));
    return same_image && (r2 < a.rs2);
}

// Order-preserving integer key of a float (for warp min / max reductions).
__device__ __forceinline__ int fkey(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float funkey(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// Resident CTAs per SM the build's register budget is sized for (8: 64
// registers, no spills; the shared memory of 8 CTAs fits with kCand 256).
#ifndef MD_BUILD_MINB
#define MD_BUILD_MINB 8
#endif

template <int T>
__global__ void __launch_bounds__(kWarps * 32, MD_BUILD_MINB) k_build(BuildArgs a) {
    constexpr int A = 32 / T;
    if (a.fl->status & ST_FREEZE) return;
    __shared__ __align__(16) float4 cand[kWarps][kCand];
    __shared__ int32_t s_start[kWarps][27];
    __shared__ int32_t s_cnt[kWarps][27];
    __shared__ __align__(16) float4 s_off[kWarps][27];
    __shared__ __align__(16) float4 hpos[kWarps][32];  // (-2 h, |h|^2) of home atom hh
    __shared__ int32_t s_self[kWarps][32];
    __shared__ __align__(16) uint4 s_mask[kWarps][32];  // home atom hh's accept masks
    __shared__ __align__(16) float4 s_be[kWarps];        // the batch box's half extents
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * kWarps + w;
    if (c >= a.ncell) return;  // whole warp
    const Box &B = a.boxes[a.cell_box[c]];
    const int64_t base = (int64_t)B.slot_off - B.atom_base;
    const int hm = a.cstart[c + 1] - a.cstart[c];
    if (hm == 0) return;  // whole warp
    const int64_t h0 = base + a.cstart[c];
    // stencil slots: first slot and count of each of the 27 cells
    if (lane < 27) {
        const int loc = c - B.cell_off;
        const int cx = loc % B.nc[0], cy = (loc / B.nc[0]) % B.nc[1], cz = loc / (B.nc[0] * B.nc[1]);
        int nx = cx + lane % 3 - 1, ny = cy + (lane / 3) % 3 - 1, nz = cz + lane / 9 - 1;
        nx += nx < 0 ? B.nc[0] : (nx >= B.nc[0] ? -B.nc[0] : 0);  // periodic wrap
        ny += ny < 0 ? B.nc[1] : (ny >= B.nc[1] ? -B.nc[1] : 0);
        nz += nz < 0 ? B.nc[2] : (nz >= B.nc[2] ? -B.nc[2] : 0);
        const int ncl = B.cell_off + (nz * B.nc[1] + ny) * B.nc[0] + nx;
        s_start[w][lane] = (int32_t)(base + a.cstart[ncl]);
        s_cnt[w][lane] = a.cstart[ncl + 1] - a.cstart[ncl];
    }
    __syncwarp();

    const float hi = a.rs2f + a.bandf, lo = a.rs2f - a.bandf;
    // padding candidates of a window: far away, never accepted
    const float4 far = make_float4(1e4f, 1e4f, 1e4f, __uint_as_float(sentinel_entry(a.ns)));
    // A candidate farther than rs from every point of the batch's box cannot
    // be a neighbor of any of its atoms and is not staged (a 1e-4 relative
    // margin covers the FP32 rounding of the coordinates).
    const float cull2 = a.rs2f * 1.0002f;
    const unsigned below = (1u << lane) - 1u;
    for (int hb = 0; hb < hm; hb += 32) {
        const int nh = min(32, hm - hb);
        const bool active = lane < nh;
        const int64_t i = chk_index(h0 + hb + (active ? lane : 0), a.ns, CHK_BUILD_HOME, a.fl,
                                    0);  // this lane's home atom
        {
            // the batch's box: centre bc, half extents (with margins) to s_be;
            // slot offsets and the home atoms taken relative to bc
            const float4 si = a.sh[i];
            const float v[3] = {si.x, si.y, si.z};
            float bc[3], be[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const float l = funkey(__reduce_min_sync(0xffffffffu, active ? fkey(v[ax]) : 0x7fffffff));
                const float u = funkey(__reduce_max_sync(0xffffffffu, active ? fkey(v[ax]) : (int)0x80000000));
                bc[ax] = 0.5f * (l + u);
                be[ax] = 0.5f * (u - l) * 1.0001f + 1e-5f * B.hf[ax];
            }
            // (every lane is past the previous batch's staging: the reductions
            // above are warp-wide)
            if (lane == 0) s_be[w] = make_float4(be[0], be[1], be[2], 0.f);
            if (lane < 27)
                s_off[w][lane] = make_float4((float)(lane % 3 - 1) * B.hf[0] - bc[0],
                                             (float)((lane / 3) % 3 - 1) * B.hf[1] - bc[1],
                                             (float)(lane / 9 - 1) * B.hf[2] - bc[2], 0.f);
            const float hx = si.x - bc[0], hy = si.y - bc[1], hz = si.z - bc[2];
            hpos[w][lane] = make_float4(-2.f * hx, -2.f * hy, -2.f * hz, fmaf(hx, hx, fmaf(hy, hy, hz * hz)));
        }
        // window * kCand + position of home atom hb + lane once it is staged;
        // until then past every window position, so that no home-cell
        // candidate staged before it counts as after it (half lists)
        s_self[w][lane] = 1 << 30;
        __syncwarp();
        // row of atom i: entry k at ((i / A) R + k / T) 32 + (i % A) T + k % T
        uint32_t *const rowp = a.nbr + ((size_t)(i / A) * a.R) * 32 + (i % A) * T;
        int cnt = 0;
        // this lane's accepted candidates among window slots [32 c, 32 c + 32),
        // in window order, into its atom's row (its own atom already cleared)
        auto write_chunk = [&](int c, unsigned m_hi, unsigned m_lo) {
            const int gb = 32 * c;
            unsigned acc = m_lo, band = m_hi & ~m_lo;
            while (band) {  // rare: candidates near rs^2 take the exact FP64 decision
                const int k = __ffs(band) - 1;
                band &= band - 1u;
                const float4 p = cand[w][gb + k];
                const uint32_t meta = __float_as_uint(p.w);
                // the home atom's staged coordinates, back from hpos (exact)
                const float4 hq = hpos[w][lane];
                if (exact_test(a, B, i, meta & MD_IDX_MASK, p.x + 0.5f * hq.x, p.y + 0.5f * hq.y,
                               p.z + 0.5f * hq.z))
                    acc |= 1u << k;
            }
            while (acc) {
                const int k = __ffs(acc) - 1;
                acc &= acc - 1u;
                const uint32_t meta = __float_as_uint(cand[w][gb + k].w);
                const unsigned uc = (unsigned)cnt;
                if (cnt < a.pad) rowp[(uc / T) * 32u + uc % T] = meta;
                ++cnt;
            }
        };
        // The 27 slots are staged into windows of up to kCand kept candidates,
        // 32 candidates of one slot at a time.
        int s = 0, g_off = 0, win = 0;
        while (s < 27) {
            __syncwarp();
            int mc = 0;  // candidates of this window kept in cand[w]
            while (s < 27) {
                const int cnt_s = s_cnt[w][s];
                const int take = min(32, cnt_s - g_off);
                if (mc + take > kCand) break;  // the window is full (uniform)
                // Every lane loads: lanes from take on repeat the chunk's last
                // candidate (an empty slot reads the slot's start, at most the
                // dummy slot ns, which the shadows hold); only lanes below take
                // may keep theirs.
                const int64_t j = chk_index(s_start[w][s] + g_off + min(lane, max(take - 1, 0)),
                                            a.ns + 1, CHK_BUILD_CAND, a.fl, 0);
                const float4 p = a.sh[j];
                const float4 o = s_off[w][s];
                const float4 q = make_float4(p.x + o.x, p.y + o.y, p.z + o.z,
                                             __uint_as_float((uint32_t)j | ((uint32_t)s << MD_IDX_BITS)));
                const float4 be = s_be[w];
                const float ex = fmaxf(fabsf(q.x) - be.x, 0.f);
                const float ey = fmaxf(fabsf(q.y) - be.y, 0.f);
                const float ez = fmaxf(fabsf(q.z) - be.z, 0.f);
                const bool keep = lane < take && fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < cull2;
                const unsigned bk = __ballot_sync(0xffffffffu, keep);
                const int pos = mc + __popc(bk & below);
                if (keep) cand[w][pos] = q;
                if (s == (int)kCodeZero) {
                    // the home cell: record where this batch's home atoms sit
                    const int hk = g_off + lane - hb;
                    if (keep && hk >= 0 && hk < nh) s_self[w][hk] = win * kCand + pos;
                }
                mc += __popc(bk);
                g_off += take;
                if (g_off >= cnt_s) {
                    ++s;
                    g_off = 0;
                }
            }
            // C chunks of 32 window slots (an even number; slots from mc on
            // hold far padding)
            const int C = ((mc + 63) >> 6) << 1;
            for (int g = mc + lane; g < 32 * C; g += 32) cand[w][g] = far;
            __syncwarp();
            // this lane's atom: its window slot P (negative: staged in an
            // earlier window; >= 32 C: in a later one or not staged yet), and
            // the chunk cs and bit bs that hold it
            const int P = s_self[w][lane] - win * kCand;
            const int cs = (P >= 0 && P < 32 * C) ? P >> 5 : -1, bs = P & 31;
            // bits k of chunk cc whose slots come after P (half lists)
            auto after = [&](int cc) -> unsigned {
                const int kt = P - 32 * cc;  // the atom's bit in chunk cc
                if (kt < 0) return 0xffffffffu;
                if (kt >= 31) return 0u;
                return ~((2u << kt) - 1u);
            };
            for (int c = 0; c < C; c += 2) {
                // Test phase: lane = candidates 32 c + lane and 32 c + 32 + lane
                // against every home atom; home atom hh's ballots land in lane hh.
                const float4 c0 = cand[w][32 * c + lane], c1 = cand[w][32 * c + 32 + lane];
                const float cc0 = fmaf(c0.x, c0.x, fmaf(c0.y, c0.y, c0.z * c0.z));
                const float cc1 = fmaf(c1.x, c1.x, fmaf(c1.y, c1.y, c1.z * c1.z));
                for (int hh = 0; hh < nh; ++hh) {
                    const float4 h = hpos[w][hh];
                    const float r20 = fmaf(c0.x, h.x, fmaf(c0.y, h.y, fmaf(c0.z, h.z, cc0 + h.w)));
                    const float r21 = fmaf(c1.x, h.x, fmaf(c1.y, h.y, fmaf(c1.z, h.z, cc1 + h.w)));
                    const unsigned bh0 = __ballot_sync(0xffffffffu, r20 <= hi);
                    const unsigned bl0 = __ballot_sync(0xffffffffu, r20 < lo);
                    const unsigned bh1 = __ballot_sync(0xffffffffu, r21 <= hi);
                    const unsigned bl1 = __ballot_sync(0xffffffffu, r21 < lo);
                    if (lane == 0) s_mask[w][hh] = make_uint4(bh0, bl0, bh1, bl1);
                }
                // half lists: candidates of a forward stencil cell, and of the
                // home cell
                unsigned fw0 = 0u, fw1 = 0u, hc0 = 0u, hc1 = 0u;
                if (a.half) {
                    const unsigned k0 = __float_as_uint(c0.w) >> MD_IDX_BITS;
                    const unsigned k1 = __float_as_uint(c1.w) >> MD_IDX_BITS;
                    fw0 = __ballot_sync(0xffffffffu, k0 > kCodeZero);
                    fw1 = __ballot_sync(0xffffffffu, k1 > kCodeZero);
                    hc0 = __ballot_sync(0xffffffffu, k0 == kCodeZero);
                    hc1 = __ballot_sync(0xffffffffu, k1 == kCodeZero);
                }
                __syncwarp();
                if (!active) continue;
                const uint4 m = s_mask[w][lane];
                unsigned hi0 = m.x, lo0 = m.y, hi1 = m.z, lo1 = m.w;
                // the atom itself (distance 0, in the window once) is no neighbor
                if (c == cs) { hi0 &= ~(1u << bs); lo0 &= ~(1u << bs); }
                if (c + 1 == cs) { hi1 &= ~(1u << bs); lo1 &= ~(1u << bs); }
                if (a.half) {
                    // home-cell candidates staged after the atom itself (the
                    // far padding has code 13 but is never accepted)
                    const unsigned keep0 = fw0 | (hc0 & after(c)), keep1 = fw1 | (hc1 & after(c + 1));
                    hi0 &= keep0; lo0 &= keep0; hi1 &= keep1; lo1 &= keep1;
                }
                write_chunk(c, hi0, lo0);
                write_chunk(c + 1, hi1, lo1);
            }
            ++win;
        }
        if (active) {
            a.nn[i] = cnt;
            if (cnt > a.pad) atomicOr(&a.fl->status, ST_OVERFLOW);
        }
        const int mx = __reduce_max_sync(0xffffffffu, active ? cnt : 0);
        const unsigned sm = __reduce_add_sync(0xffffffffu, active ? (unsigned)cnt : 0u);
        if (lane == 0) {
            atomicMax(&a.fl->maxnn, mx);
            atomicAdd(&a.fl->sumnn, (unsigned long long)sm);
        }
    }
}

// After a build: in each warp-tile (A atoms, T lanes each), the slots of rows
// up to the tile's longest row that lie past their atom's count get the
// sentinel entry, one coalesced row store at a time, so that the force kernel
// can take whole rows up to the longest (rows past it are never read).
template <int T>
__global__ void __launch_bounds__(256) k_fill_tails(const int32_t *__restrict__ nn,
                                                   uint32_t *__restrict__ nbr, int64_t nwt, int R,
                                                   int pad, uint32_t sent, const Flags *fl) {
    constexpr int A = 32 / T;
    if (fl->status & ST_FREEZE) return;
    const int64_t wt = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (wt >= nwt) return;  // whole warp
    const int lane = threadIdx.x & 31, sub = lane % T;
    const int ni = min(__ldg(nn + wt * A + lane / T), pad);
    const int nq = ni > sub ? (ni - sub + T - 1) / T : 0;  // this lane's entries
    const int r0 = __reduce_min_sync(0xffffffffu, nq), r1 = __reduce_max_sync(0xffffffffu, nq);
    uint32_t *row = nbr + (size_t)wt * R * 32 + lane;
    for (int q = r0; q < r1; ++q)
        if (q >= nq) row[(size_t)q * 32] = sent;
}

__global__ void k_fill_u32(uint32_t *__restrict__ p, size_t n, uint32_t v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

template <int T>
cudaError_t launch_build_t(md_ctx *c, const BuildArgs &a) {
    const unsigned grid = (unsigned)((c->ncell_tot + kWarps - 1) / kWarps);
    k_build<T><<<grid, kWarps * 32, 0, c->stream>>>(a);
    const int64_t nwt = c->ns / (32 / T);
    k_fill_tails<T><<<(unsigned)((nwt * 32 + 255) / 256), 256, 0, c->stream>>>(
        c->nn, c->nbr, nwt, c->R, c->pad, sentinel_entry(c), c->dflags);
    return cudaGetLastError();
}

}  // namespace

// At allocation every list slot gets the sentinel entry; the rows of padding
// slots keep it (no build writes them); a build writes each real atom's
// entries, then k_fill_tails the sentinels its warp-tile's readers need.
cudaError_t fill_list_sentinel(md_ctx *c) {
    const size_t words = (size_t)c->ns * c->pad;
    k_fill_u32<<<(unsigned)std::min<size_t>((words + 255) / 256, 65535), 256, 0, c->stream>>>(
        c->nbr, words, sentinel_entry(c));
    c->kernels += 1;
    return cudaGetLastError();
}

size_t build_smem_bytes(int) { return 0; }

cudaError_t launch_build(md_ctx *c) {
    BuildArgs a;
    a.boxes = c->dbox;
    a.cell_box = c->cell_box;
    a.cstart = c->cstart;
    a.sh = c->sh[c->pc];
    a.xws = c->xws;
    a.ns = c->ns;
    a.ncell = c->ncell_tot;
    a.rs2 = c->hpair.rs2;
    a.rs2f = c->hpair.rs2f;
    a.bandf = c->hpair.bandf;
    a.pad = c->pad;
    a.R = c->R;
    a.half = c->params.half_list ? 1 : 0;
    a.nn = c->nn;
    a.nbr = c->nbr;
    a.fl = c->dflags;
    cudaError_t e;
    switch (c->T) {
        case 1: e = launch_build_t<1>(c, a); break;
        case 2: e = launch_build_t<2>(c, a); break;
        case 4: e = launch_build_t<4>(c, a); break;
        case 8: e = launch_build_t<8>(c, a); break;
        default: return cudaErrorInvalidValue;
    }
    c->kernels += 2;
    return e;
}

}  // namespace mdb

// md_neigh.cu -- Verlet neighbor list by binning (paper, Section "Neighbor
// List Creation": "traditional binning methods used in many MD applications
// (Verlet lists)", stored in a dense padded format).
//
// One CTA per cell.  The CTA stages the candidates of the 27-cell stencil in
// shared memory (FP32 cell-local coordinates shifted by the stencil offset, so
// a candidate's coordinate is relative to the home cell's centre), then each
// warp takes one home atom at a time and its 32 lanes test 32 candidates per
// step; accepted candidates are compacted with a ballot into the atom's row
// (staged in shared memory) and finally written out in the warp-transposed
// padded layout with full 128-byte row stores.
//
// Decision rule (bit-exact with the FP64 definition): a pair is a neighbor iff
// the nearest-image FP64 distance r^2 = (dx*dx + dy*dy) + dz*dz, every op
// rounded separately, is < (rc+skin)^2.  The FP32 r^2 of the staged
// coordinates differs from it by < 2e-5 (|coords| <= 1.5 h, h <= 4.2; each
// coordinate carries <= 2^-24 relative rounding), so candidates with FP32 r^2
// outside [rs^2 - band, rs^2 + band], band = 1e-3 rs^2, are decided in FP32
// and the few inside the band are re-tested with the exact FP64 rule on the
// wrapped FP64 positions.  When an axis has only 2 cells, the -1 and +1 stencil
// slots hold the same cell under two images; only one image can lie within
// rs (L > 2 rs), and the FP64 re-test checks that the slot's image is the
// nearest one.
#include <algorithm>

#include "md_common.cuh"

namespace mdb {
namespace {

constexpr int kMaxCand = 1024;  // candidates staged per window
constexpr int kHome = 32;       // home atoms per chunk
constexpr int kThreads = 128;

struct BuildArgs {
    const Box *boxes;
    const int32_t *cell_box;
    const int32_t *cstart;
    const float4 *sh;
    const double *xws;
    int64_t ns;
    double rs2;
    float rs2f, bandf;
    int pad, R, T;
    uint32_t sentinel;
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

__global__ void __launch_bounds__(kThreads) k_build(BuildArgs a) {
    if (a.fl->status & ST_FREEZE) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *cpos = reinterpret_cast<float4 *>(smem);
    uint32_t *cmeta = reinterpret_cast<uint32_t *>(cpos + kMaxCand);
    uint32_t *lst = cmeta + kMaxCand;  // kHome * pad
    __shared__ int64_t s_start[27];
    __shared__ int32_t s_pref[28];
    __shared__ float4 s_off[27];
    __shared__ int32_t s_cnt[kHome];
    __shared__ int32_t s_maxe;

    const int c = blockIdx.x;
    const Box &B = a.boxes[a.cell_box[c]];
    const int64_t base = (int64_t)B.slot_off - B.atom_base;
    const int hm = a.cstart[c + 1] - a.cstart[c];
    if (hm == 0) return;
    const int64_t h0 = base + a.cstart[c];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    constexpr int NW = kThreads / 32;

    if (tid < 27) {
        const int loc = c - B.cell_off;
        const int cx = loc % B.nc[0], cy = (loc / B.nc[0]) % B.nc[1],
                  cz = loc / (B.nc[0] * B.nc[1]);
        const int ox = tid % 3 - 1, oy = (tid / 3) % 3 - 1, oz = tid / 9 - 1;
        const int nx = (cx + ox + B.nc[0]) % B.nc[0];
        const int ny = (cy + oy + B.nc[1]) % B.nc[1];
        const int nz = (cz + oz + B.nc[2]) % B.nc[2];
        const int nc = B.cell_off + (nz * B.nc[1] + ny) * B.nc[0] + nx;
        s_start[tid] = base + a.cstart[nc];
        s_pref[tid + 1] = a.cstart[nc + 1] - a.cstart[nc];
        s_off[tid] = make_float4((float)ox * B.hf[0], (float)oy * B.hf[1], (float)oz * B.hf[2], 0.f);
    }
    __syncthreads();
    if (tid == 0) {
        s_pref[0] = 0;
        for (int s = 0; s < 27; ++s) s_pref[s + 1] += s_pref[s];
    }
    __syncthreads();
    const int M = s_pref[27];
    const int nwin = (M + kMaxCand - 1) / kMaxCand;
    const int T = a.T, A = 32 / T;

    for (int hc = 0; hc < hm; hc += kHome) {
        const int na = min(kHome, hm - hc);
        if (tid < kHome) s_cnt[tid] = 0;
        if (tid == 0) s_maxe = 0;
        for (int w = 0; w < nwin; ++w) {
            const int w0 = w * kMaxCand;
            const int Mw = min(kMaxCand, M - w0);
            if (nwin > 1 || hc == 0) {
                __syncthreads();
                for (int k = tid; k < Mw; k += kThreads) {
                    const int g = w0 + k;
                    int s = 0;
                    while (s_pref[s + 1] <= g) ++s;
                    const int64_t j = s_start[s] + (g - s_pref[s]);
                    const float4 p = a.sh[j];
                    const float4 o = s_off[s];
                    cpos[k] = make_float4(p.x + o.x, p.y + o.y, p.z + o.z, 0.f);
                    cmeta[k] = (uint32_t)j | ((uint32_t)s << MD_IDX_BITS);
                }
            }
            __syncthreads();
            for (int ha = wib; ha < na; ha += NW) {
                const int64_t i = h0 + hc + ha;
                const float4 si = a.sh[i];
                int cnt = s_cnt[ha];
                for (int kb = 0; kb < Mw; kb += 32) {
                    const int k = kb + lane;
                    bool acc = false;
                    uint32_t meta = 0;
                    if (k < Mw) {
                        const float4 p = cpos[k];
                        meta = cmeta[k];
                        const int64_t j = meta & MD_IDX_MASK;
                        const float dx = p.x - si.x, dy = p.y - si.y, dz = p.z - si.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (j != i) {
                            if (r2 < a.rs2f - a.bandf) acc = true;
                            else if (r2 <= a.rs2f + a.bandf) acc = exact_test(a, B, i, j, dx, dy, dz);
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, acc);
                    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                    if (acc && pos < a.pad) lst[ha * a.pad + pos] = meta;
                    cnt += __popc(m);
                }
                if (lane == 0) s_cnt[ha] = cnt;
                __syncwarp();
            }
        }
        __syncthreads();
        if (tid < na) {
            const int cnt = s_cnt[tid];
            const int64_t i = h0 + hc + tid;
            a.nn[i] = cnt;
            atomicMax(&a.fl->maxnn, cnt);
            atomicAdd(&a.fl->sumnn, (unsigned long long)cnt);
            atomicMax(&s_maxe, min(cnt, a.pad));
            if (cnt > a.pad) atomicOr(&a.fl->status, ST_OVERFLOW);
        }
        __syncthreads();
        // Write the rows of this chunk: warp-tiles W0..W1, all R rows; each
        // store is one 32-word row (lanes of atoms outside the chunk masked).
        // Slots past an atom's count get the sentinel entry (a dummy slot far
        // away, zero offset), so readers may run whole batches unpredicated.
        const int64_t first = h0 + hc, last = h0 + hc + na - 1;
        const int64_t W0 = first / A, W1 = last / A;
        const int rows = a.R;
        const int64_t items = (W1 - W0 + 1) * rows;
        for (int64_t it = wib; it < items; it += NW) {
            const int64_t W = W0 + it / rows;
            const int q = (int)(it % rows);
            const int64_t i = W * A + lane / T;
            const int64_t ha = i - first;
            const int k = q * T + lane % T;
            if (ha >= 0 && ha < na)
                a.nbr[((size_t)W * a.R + q) * 32 + lane] =
                    k < min(s_cnt[ha], a.pad) ? lst[ha * a.pad + k] : a.sentinel;
        }
        __syncthreads();
    }
}

__global__ void k_fill_u32(uint32_t *__restrict__ p, size_t n, uint32_t v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

// Every list slot (including the rows of padding slots, which no build
// writes) starts as the sentinel entry.
cudaError_t fill_list_sentinel(md_ctx *c) {
    const size_t words = (size_t)c->ns * c->pad;
    k_fill_u32<<<(unsigned)std::min<size_t>((words + 255) / 256, 65535), 256, 0, c->stream>>>(
        c->nbr, words, sentinel_entry(c));
    c->kernels += 1;
    return cudaGetLastError();
}

size_t build_smem_bytes(int pad) {
    return (size_t)kMaxCand * (sizeof(float4) + sizeof(uint32_t)) +
           (size_t)kHome * pad * sizeof(uint32_t);
}

cudaError_t launch_build(md_ctx *c) {
    BuildArgs a;
    a.boxes = c->dbox;
    a.cell_box = c->cell_box;
    a.cstart = c->cstart;
    a.sh = c->sh[c->pc];
    a.xws = c->xws;
    a.ns = c->ns;
    a.rs2 = c->hpair.rs2;
    a.rs2f = c->hpair.rs2f;
    a.bandf = c->hpair.bandf;
    a.pad = c->pad;
    a.R = c->R;
    a.T = c->T;
    a.sentinel = sentinel_entry(c);
    a.nn = c->nn;
    a.nbr = c->nbr;
    a.fl = c->dflags;
    const size_t smem = build_smem_bytes(c->pad);
    static size_t smem_set = 0;  // raised only when a larger pad needs it
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(k_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    k_build<<<c->ncell_tot, kThreads, smem, c->stream>>>(a);
    c->kernels += 1;
    return cudaGetLastError();
}

}  // namespace mdb

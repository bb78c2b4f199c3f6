// md_force.cu -- Lennard-Jones 12-6 pair forces over the Verlet list, fused
// with the velocity-Verlet update (paper: the LJ short-range benchmark kernel
// of CabanaMD, Section "CabanaMD"; "forces are calculated to propagate the
// particles to new positions", Introduction).
//
// Per pair, with d = x_j - x_i and r^2 = |d|^2 < rc^2:
//   phi = 24 eps / r^2 [2 (sigma^2/r^2)^6 - (sigma^2/r^2)^3],  F_i += -phi d,
//   e_i += 1/2 * 4 eps [(sigma^2/r^2)^6 - (sigma^2/r^2)^3]  (- U(rc) if shifted).
//
// Mixed precision: pair arithmetic in FP32 on the cell-local shadow
// coordinates (x_j - x_i = (s_j + delta h) - s_i, delta from the list entry's
// stencil code); each lane keeps a Kahan-compensated FP32 sum of its share of
// the neighbors, adding one FMA-chained group of MD_FORCE_GROUP terms per
// Kahan step; the T lanes of an atom fold their compensations and add their
// partials in a fixed xor-shuffle order; the result is converted to FP64
// once.  Velocities, positions and energy totals are FP64.
//
// Launch: persistent grids (SM count x resident CTAs); a warp-tile is A = 32/T
// consecutive atoms, T lanes each, and row q of its list block holds entry q
// of each lane (one 128-byte row).
//
// Modes: FORCE_ONLY (store F, energy), FINAL (store F, v += dt/2 F/m, thermo),
// FUSED (v += dt/2 F/m [thermo at v_n] v += dt/2 F/m, x += dt v, write the next
// shadow; the list-side reads use the current buffers, writes go to the
// other buffer, so the kernel never reads what it writes).
#include <algorithm>
#include <atomic>
#include <mutex>

#include "md_common.cuh"

namespace mdb {
namespace {

constexpr int kBlock64 = 256;       // FP64 kernel: CTAs of up to 256 threads
constexpr int kMaxWarps = kBlock64 / 32;
constexpr int kMaxWarpsMixed = 24;  // mixed kernel: CTAs up to 768 threads
constexpr int kBatch = MD_FORCE_BATCH;        // list entries per lane per batch
constexpr uint32_t kNoEntry = 0xFFFFFFFFu;   // code 31: zero offset, far position

struct ForceArgs {
    const Box *boxes;
    const int32_t *tile_box;
    const Pair *pair;
    int64_t ns, nwt;  // slots, warp-tiles
    int pad, R;
    const float4 *sh_in;
    float4 *sh_out;
    const double *r_in;
    double *r_out;
    double *v;
    double *f;
    const double *rbuild;
    const int32_t *type;
    const int32_t *nn;
    const uint32_t *nbr;
    double *tpart;
    Flags *fl;
    int mode;
    int thermo_every;
    unsigned int *done;
    uint32_t tx_extra;  // test hook: list-copy bytes that never arrive (0 normally)
    float4 *facc;       // half lists: force (x, y, z) and energy accumulators per slot
    double *facc64;     // half lists, FP64 context: the same, 4 doubles per slot
    const float *shv;   // shadow_vl > 0: the shadows in blocks of x[VL], y[VL], z[VL], type[VL]
};

// Neighbor j's shadow for the mixed kernels: one 16-byte load from the float4
// array (VL = 0), or from the AoSoA copy, one 4-byte load per component (the
// type only when there are several).
template <int VL, bool ONE>
__device__ __forceinline__ float4 gather_shadow(const ForceArgs &a, uint32_t en) {
    const int64_t j = chk_index(en & MD_IDX_MASK, a.ns + 1, CHK_FORCE_GATHER, a.fl, a.ns);
    if constexpr (VL == 0) {
        return __ldg(a.sh_in + j);
    } else {
        const float *p = a.shv + (j / VL) * (4 * VL) + (j % VL);
        return make_float4(__ldg(p), __ldg(p + VL), __ldg(p + 2 * VL), ONE ? 0.f : __ldg(p + 3 * VL));
    }
}

// Half lists: add (x, y, z, e) to slot j's accumulator (one vector reduction).
__device__ __forceinline__ void red_add4(float4 *p, float x, float y, float z, float e) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z),
                 "f"(e)
                 : "memory");
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float t) {
    const float y = t - c;
    const float u = s + y;
    c = (u - s) - y;
    s = u;
}

// 1/x by the hardware's approximate reciprocal (one instruction, within about
// an ulp; denormal results flush to zero), where __fdividef(1, x) adds a range
// check and a multiply (B300, 4M atoms: 0.697 -> 0.666 ms per force launch).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}


template <int T>
__device__ __forceinline__ double sum_lanes_d(double x) {
#pragma unroll
    for (int o = T / 2; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int T>
__device__ __forceinline__ float sum_lanes_f(float x) {
#pragma unroll
    for (int o = T / 2; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Shared per-CTA tables.
struct SmemTabs {
    float fs2[64], fe4[64], fush[64], fc1[64];
    double de24[64], ds2[64], de4[64], dush[64];
    double dtm[MD_MAXT], hdtm[MD_MAXT], mass[MD_MAXT];
};

// The velocity-Verlet epilogue for component d of atom i; returns the new
// shadow coordinate (FUSED) and accumulates thermo terms.
template <bool THERMO, bool PRE>
__device__ __forceinline__ float epilogue(const ForceArgs &a, const SmemTabs &tb, int64_t i, int d,
                                          int ti, double F, double pv, double pr, double &ke,
                                          double &p, double &disp2) {
    const int64_t o = d * a.ns + i;
    float snew = 0.f;
    if (a.mode == MODE_FORCE_ONLY) {
        a.f[o] = F;
        if (THERMO) {
            const double vv = a.v[o];
            ke += 0.5 * tb.mass[ti] * vv * vv;
            p += tb.mass[ti] * vv;
            const double dd = a.r_in[o] - a.rbuild[o];
            disp2 += dd * dd;
        }
    } else if (a.mode == MODE_FINAL) {
        a.f[o] = F;
        const double vv = fma(tb.hdtm[ti], F, a.v[o]);
        a.v[o] = vv;
        if (THERMO) {
            ke += 0.5 * tb.mass[ti] * vv * vv;
            p += tb.mass[ti] * vv;
            const double dd = a.r_in[o] - a.rbuild[o];
            disp2 += dd * dd;
        }
    } else {
        // streaming accesses (read or written once per step): keep them out of
        // L1, which holds the neighbor shadows the gathers reuse
        double vv;
        const double v0 = PRE ? pv : __ldcs(a.v + o);
        const double r0 = PRE ? pr : __ldcs(a.r_in + o);
        if (THERMO) {
            const double vh = fma(tb.hdtm[ti], F, v0);
            ke += 0.5 * tb.mass[ti] * vh * vh;
            p += tb.mass[ti] * vh;
            const double dd = r0 - a.rbuild[o];
            disp2 += dd * dd;
            vv = fma(tb.hdtm[ti], F, vh);
        } else {
            vv = fma(tb.dtm[ti], F, v0);
        }
        __stcs(a.v + o, vv);
        const double rn = fma(a.pair->dt, vv, r0);
        __stcs(a.r_out + o, rn);
        snew = __double2float_rn(rn);
    }
    return snew;
}


// A lane's FP64 state for the FUSED velocity-Verlet epilogue: components
// d = sub + k T (k < NC) of velocity and position, loaded when a tile starts
// so that their DRAM latency overlaps the tile's list rows instead of
// stalling the epilogue.
template <int T>
struct TileState {
    static constexpr int NC = (3 + T - 1) / T;
    double v[NC], r[NC];
};

template <int T>
__device__ __forceinline__ void load_tile_state(const ForceArgs &a, int64_t i, bool valid,
                                                TileState<T> &st) {
    const int sub = (threadIdx.x & 31) % T;
#pragma unroll
    for (int k = 0; k < TileState<T>::NC; ++k) {
        const int d = sub + k * T;
        const bool on = valid && d < 3 && a.mode == MODE_FUSED;
        const int64_t o = (int64_t)(on ? d : 0) * a.ns + i;
        st.v[k] = on ? __ldcs(a.v + o) : 0.0;
        st.r[k] = on ? __ldcs(a.r_in + o) : 0.0;
    }
}

// The rest of a warp-tile once each atom's force is known in all its lanes:
// the velocity-Verlet epilogue (lane `sub` takes components sub, sub + T, ...;
// PRE: with the state `st` loaded at the tile's start), the atom's next
// shadow, and the tile's thermo partials.  Only the components a lane handles
// are widened to FP64.
template <int T, bool THERMO, bool PRE, typename FT>
__device__ __forceinline__ void finish_tile(const ForceArgs &a, const SmemTabs &tb, int64_t wt,
                                            int64_t i, bool valid, int ti, const FT (&F)[3],
                                            double ped, const TileState<T> &st) {
    const int lane = threadIdx.x & 31, sub = lane % T;
    double ke = 0.0, pd[3] = {0.0, 0.0, 0.0}, disp2 = 0.0;
    float snew[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < (3 + T - 1) / T; ++k) {
        const int d = sub + k * T;
        if (valid && d < 3) {
            const double Fc = (double)(d == 0 ? F[0] : (d == 1 ? F[1] : F[2]));
            double pp = 0.0;
            const float sn =
                epilogue<THERMO, PRE>(a, tb, i, d, ti, Fc, st.v[k], st.r[k], ke, pp, disp2);
#pragma unroll
            for (int dd = 0; dd < 3; ++dd)
                if (dd == d) { snew[dd] = sn; pd[dd] = pp; }
        }
    }
    if (a.mode == MODE_FUSED) {
        float s3[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            s3[d] = __shfl_sync(0xffffffffu, snew[d], (lane - sub) + d % T);
        if (valid && sub == 0) a.sh_out[i] = make_float4(s3[0], s3[1], s3[2], __int_as_float(ti));
    }
    if (THERMO) {
        // Five FP64 sums over the warp (PE, KE, Px, Py, Pz) by a butterfly
        // that halves the values each lane carries per level (9 adds instead
        // of 25); lane 4q ends with quantity q.  The largest displacement^2 of
        // an atom (its components summed over its lanes) in FP32.
        double q[8] = {(valid && sub == 0) ? ped : 0.0, ke, pd[0], pd[1], pd[2], 0.0, 0.0, 0.0};
#pragma unroll
        for (int h = 4, o = 16; h >= 1; h >>= 1, o >>= 1) {
            const bool up = lane & o;
#pragma unroll
            for (int k = 0; k < h; ++k) {
                const double give = up ? q[k] : q[k + h];
                const double keep = up ? q[k + h] : q[k];
                q[k] = keep + __shfl_xor_sync(0xffffffffu, give, o);
            }
        }
        q[0] += __shfl_xor_sync(0xffffffffu, q[0], 2);
        q[0] += __shfl_xor_sync(0xffffffffu, q[0], 1);
        const float dsum = sum_lanes_f<T>((float)disp2);
        const float dm = __uint_as_float(
            __reduce_max_sync(0xffffffffu, valid ? __float_as_uint(dsum) : 0u));
        double *tp = a.tpart + wt * TP;
        if ((lane & 3) == 0 && lane < 20) tp[lane >> 2] = q[0];
        if (lane == 0) tp[5] = (double)dm;
    }
}

// ---- FP64 kernel ----
//
// Warp w of the grid takes warp-tiles w, w + nwarps, ...; each lane walks its
// share of the atom's row (entries sub, sub + T, ...) kBatch entries at a time:
// the list words, then the neighbor positions, then the pair terms.
template <int T, bool ONE, bool THERMO, bool HALF>
__device__ __forceinline__ void force_body64(const ForceArgs &a, const SmemTabs &tb,
                                             double (*s_offd)[81], float (*s_offf)[81]) {
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = lane % T;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int nt = a.pair->nt;
    const double rc2 = a.pair->rc2;
    const double de24_0 = tb.de24[0], ds2_0 = tb.ds2[0], de4_0 = tb.de4[0], dush_0 = tb.dush[0];
    int curbox = -1;
    for (int64_t wt = gw; wt < a.nwt; wt += nw) {
        const int64_t i = wt * A + lane / T;
        const int b = a.tile_box[(wt * A) >> 5];
        const Box &B = a.boxes[b];
        if (b != curbox) {
            if (lane < 27) {
                const int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
                s_offd[wib][3 * lane + 0] = (double)ox * B.h[0];
                s_offd[wib][3 * lane + 1] = (double)oy * B.h[1];
                s_offd[wib][3 * lane + 2] = (double)oz * B.h[2];
                s_offf[wib][3 * lane + 0] = (float)ox * B.hf[0];
                s_offf[wib][3 * lane + 1] = (float)oy * B.hf[1];
                s_offf[wib][3 * lane + 2] = (float)oz * B.hf[2];
            }
            __syncwarp();
            curbox = b;
        }
        const bool valid = (i - B.slot_off) < B.n;
        const int ni = valid ? min(a.nn[i], a.pad) : 0;
        const uint32_t *row = a.nbr + (size_t)wt * a.R * 32 + lane;
        const double rix = a.r_in[i], riy = a.r_in[a.ns + i], riz = a.r_in[2 * a.ns + i];
        const int ti = ONE ? 0 : a.type[i];
        // the epilogue's velocities, in flight during the rows (positions: rix..)
        TileState<T> st;
#pragma unroll
        for (int k = 0; k < TileState<T>::NC; ++k) {
            const int d = sub + k * T;
            const bool on = !HALF && valid && d < 3 && a.mode == MODE_FUSED;
            st.v[k] = on ? __ldcs(a.v + (int64_t)(on ? d : 0) * a.ns + i) : 0.0;
            st.r[k] = d == 0 ? rix : (d == 1 ? riy : riz);
        }
        double fx = 0.0, fy = 0.0, fz = 0.0, pe = 0.0;
        const int nq = (ni - sub + T - 1) / T;
        // B300's FP64 pipe is charged per warp instruction, however many lanes
        // are active: the FP64 pass runs only over the entries that can lie
        // within rc, so that the warp loops over the longest such count rather
        // than over the longest row.  Pass 1 marks them (FP32 r^2 on the
        // cell-relative shadows below rc^2 (1 + 1e-4); the shadows' error in r^2
        // is below 1e-6 rc^2); pass 2 takes them in row order, so the FP64 sums
        // are those of the full row, term for term.
        const float4 si = a.sh_in[i];
        for (int c0 = 0; c0 < nq; c0 += 32) {
          const int cn = min(32, nq - c0);
          uint32_t near = 0u;
          for (int q0 = 0; q0 < cn; q0 += kBatch) {
            uint32_t e[kBatch];
            float4 sj[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                e[u] = (q0 + u < cn) ? __ldg(row + (size_t)(c0 + q0 + u) * 32) : kNoEntry;
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                sj[u] = e[u] != kNoEntry
                            ? __ldg(a.sh_in + chk_index(e[u] & MD_IDX_MASK, a.ns + 1,
                                                        CHK_FORCE64_GATHER, a.fl, a.ns))
                            : make_float4(1e4f, 1e4f, 1e4f, 0.f);
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const float *o = s_offf[wib] + 3 * ((e[u] >> MD_IDX_BITS) % 27);
                const float dx = (sj[u].x + o[0]) - si.x;
                const float dy = (sj[u].y + o[1]) - si.y;
                const float dz = (sj[u].z + o[2]) - si.z;
                if (e[u] != kNoEntry && dx * dx + dy * dy + dz * dz < a.pair->rc2f * 1.0001f)
                    near |= 1u << (q0 + u);
            }
          }
          while (near) {
            uint32_t e[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (near) {
                    const int k = __ffs(near) - 1;
                    near &= near - 1u;
                    e[u] = __ldg(row + (size_t)(c0 + k) * 32);
                } else {
                    e[u] = kNoEntry;
                }
            }
            double xj[kBatch], yj[kBatch], zj[kBatch];
            int64_t jj[kBatch];  // checked slot indices (half lists: the reactions' targets)
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const bool ok = e[u] != kNoEntry;
                const int64_t j =
                    ok ? chk_index(e[u] & MD_IDX_MASK, a.ns, CHK_FORCE64_GATHER, a.fl, 0) : 0;
                jj[u] = j;
                xj[u] = ok ? __ldg(a.r_in + j) : 1e4;
                yj[u] = ok ? __ldg(a.r_in + a.ns + j) : 1e4;
                zj[u] = ok ? __ldg(a.r_in + 2 * a.ns + j) : 1e4;
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const double *o = s_offd[wib] + 3 * ((e[u] >> MD_IDX_BITS) % 27);
                const double dx = (xj[u] + o[0]) - rix;
                const double dy = (yj[u] + o[1]) - riy;
                const double dz = (zj[u] + o[2]) - riz;
                const double r2 = (dx * dx + dy * dy) + dz * dz;
                if (r2 < rc2) {
                    double e24, s2, e4, ush;
                    if (ONE) {
                        e24 = de24_0; s2 = ds2_0; e4 = de4_0; ush = dush_0;
                    } else {
                        const int64_t j =
                            chk_index(e[u] & MD_IDX_MASK, a.ns, CHK_FORCE64_GATHER, a.fl, 0);
                        const int ab = ti * nt + __ldg(a.type + j);
                        e24 = tb.de24[ab]; s2 = tb.ds2[ab]; e4 = tb.de4[ab]; ush = tb.dush[ab];
                    }
                    const double r2inv = rcp_newton64(r2);
                    const double q2 = s2 * r2inv;
                    const double s6 = q2 * q2 * q2;
                    const double phi = e24 * r2inv * s6 * (2.0 * s6 - 1.0);
                    fx -= phi * dx;
                    fy -= phi * dy;
                    fz -= phi * dz;
                    const double up = THERMO ? 0.5 * (e4 * s6 * (s6 - 1.0) - ush) : 0.0;
                    if (THERMO) pe += up;
                    if (HALF) {
                        // the pair is listed once: its reaction (and the other
                        // half of its energy) goes to the partner's accumulator
                        double *pj = a.facc64 + 4 * jj[u];
                        atomicAdd(pj + 0, phi * dx);
                        atomicAdd(pj + 1, phi * dy);
                        atomicAdd(pj + 2, phi * dz);
                        if (THERMO) atomicAdd(pj + 3, up);
                    }
                }
            }
          }
        }
        const double Fd[3] = {sum_lanes_d<T>(fx), sum_lanes_d<T>(fy), sum_lanes_d<T>(fz)};
        const double ped = THERMO ? sum_lanes_d<T>(pe) : 0.0;
        if (HALF) {
            // the atom's own sums join the reactions in its accumulator; the
            // epilogue kernel integrates
            if (valid && sub == 0) {
                double *pi = a.facc64 + 4 * i;
                atomicAdd(pi + 0, Fd[0]);
                atomicAdd(pi + 1, Fd[1]);
                atomicAdd(pi + 2, Fd[2]);
                if (THERMO) atomicAdd(pi + 3, ped);
            }
        } else {
            finish_tile<T, THERMO, true>(a, tb, wt, i, valid, ti, Fd, ped, st);
        }
    }
}

// ---- mixed-precision kernel ----
//
// Each warp walks a contiguous run of warp-tiles (the CTA's chunk, warps
// interleaved, so the CTA's warps share neighbors in L1).  While it evaluates
// tile t it has tile t + 1's list rows in flight into the other half of a
// per-warp shared-memory double buffer: one bulk (TMA) copy per tile, only as
// many 128-byte rows as the tile's longest row, completing on an mbarrier.
// Neighbor shadows are gathered kBatch at a time per lane.  (Measured on B300
// and dropped: 16-byte cp.async copies of the rows, 2% slower; a 27-entry
// float4 offset table, read as one 16-byte load, 1-2% slower than three
// 4-byte arrays.)

// The list is read once per step: its copies carry an L2 evict-first policy so
// they do not push out the neighbor shadows (small enough to stay in L2).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// Rows [0, rows) of a list block (128 bytes each) -> shared dst as one bulk
// copy that completes on mbarrier `bar` (the arrival and the byte count are
// posted together).  `extra` adds bytes that never arrive: a test hook that
// makes the wait below run out.  One lane only.
__device__ __forceinline__ void bulk_rows(uint32_t dst, const uint32_t *src, int rows, uint32_t bar,
                                          uint64_t pol, uint32_t extra) {
    const uint32_t bytes = (uint32_t)rows * 128u;
    // the warp's earlier generic-proxy reads of dst come before the async-proxy write
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                 "r"(bytes + extra)
                 : "memory");
    if (bytes > 0)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
            "[%0], [%1], %2, [%3], %4;\n" ::"r"(dst),
            "l"(src), "r"(bytes), "r"(bar), "l"(pol)
            : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Wait for the mbarrier phase of the given parity; false after ~1 s (or 2^28
// polls), so a copy that never completes cannot hang the kernel.  The first
// poll is inlined (a tile's rows were requested a whole tile earlier and have
// nearly always landed); the bounded loop is a call.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t k = 1; k < (1u << 28); ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((k & 255u) == 0u && globaltimer_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity);
}

// List rows a warp-tile needs: its longest row (rows past an atom's count hold
// the sentinel entry).
template <int T>
__device__ __forceinline__ int tile_rows(int ni) {
    return __reduce_max_sync(0xffffffffu, (ni + T - 1) / T);
}

// Loop-invariant pair constants of the mixed kernels.
struct MixedConst {
    int nt;
    float rc2f, c1_0, c1x2_0, s2_0, e4_0, ush_0;
};

__device__ __forceinline__ MixedConst mixed_const(const ForceArgs &a, const SmemTabs &tb) {
    MixedConst k;
    k.nt = a.pair->nt;
    k.rc2f = a.pair->rc2f;
    k.c1_0 = tb.fc1[0];
    k.c1x2_0 = 2.0f * k.c1_0;
    k.s2_0 = tb.fs2[0];
    k.e4_0 = tb.fe4[0];
    k.ush_0 = tb.fush[0];
    return k;
}

// One lane's Kahan-compensated FP32 partial sums (value = s - c).
struct Acc {
    float fx = 0.f, fy = 0.f, fz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, pe = 0.f, cp = 0.f;
};

// The pair terms of one lane's share of a list block: rows [0, rows) of the
// block in shared memory (Lr: this lane's word of row 0, rows 32 words apart;
// a row's slots past its atom's count hold the sentinel entry up to the
// block's longest row), for the home atom with shadow si and type ti.  off:
// the warp's stencil offsets (off[d][code]).  HALF: each entry is a pair
// listed once; its reaction (and half its energy) goes to the partner's
// accumulator.
template <bool ONE, bool THERMO, bool HALF, int VL = 0>
__device__ __forceinline__ void lane_rows(const ForceArgs &a, const SmemTabs &tb,
                                          const MixedConst &k, const float (*off)[32],
                                          const uint32_t *Lr, int rows, const float4 &si, int ti,
                                          Acc &acc) {
    constexpr int G = MD_FORCE_GROUP;
    static_assert(kBatch % G == 0, "MD_FORCE_GROUP must divide MD_FORCE_BATCH");
    // One list entry: x_j - x_i from the shadows and the stencil offset,
    // the LJ term masked at rc (sentinel entries past an atom's count sit
    // far beyond it): t = -phi (x_j - x_i), tp = the pair energy half.
    auto terms = [&](const uint32_t en, const float4 &sj, float &tx, float &ty, float &tz,
                     float &tp) {
        const unsigned cd = en >> MD_IDX_BITS;
        const float dx = (sj.x + off[0][cd]) - si.x;
        const float dy = (sj.y + off[1][cd]) - si.y;
        const float dz = (sj.z + off[2][cd]) - si.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool in = r2 < k.rc2f;
        const float r2inv = rcp_approx(r2);
        float s2, e4, ush, w;
        if (ONE) {
            s2 = k.s2_0; e4 = k.e4_0; ush = k.ush_0;
        } else {
            const int ab = ti * k.nt + __float_as_int(sj.w);
            s2 = tb.fs2[ab]; e4 = tb.fe4[ab]; ush = tb.fush[ab];
        }
        const float q2 = s2 * r2inv;
        const float s6 = q2 * q2 * q2;
        // phi = 24 eps / r^2 (sigma/r)^6 [2 (sigma/r)^6 - 1] = c1 q2 s6 (2 s6 - 1),
        // c1 = 24 eps / sigma^2
        if (ONE) w = fmaf(k.c1x2_0, s6, -k.c1_0);
        else w = tb.fc1[ti * k.nt + __float_as_int(sj.w)] * fmaf(2.0f, s6, -1.0f);
        const float phi = in ? (q2 * s6) * w : 0.0f;
        tx = -phi * dx;
        ty = -phi * dy;
        tz = -phi * dz;
        tp = (THERMO && in) ? 0.5f * fmaf(e4 * s6, s6 - 1.0f, -ush) : 0.0f;
        if (HALF && in)
            red_add4(a.facc + chk_index(en & MD_IDX_MASK, a.ns + 1, CHK_FORCE_GATHER, a.fl, a.ns),
                     -tx, -ty, -tz, tp);
    };
    // groups of G consecutive terms are added by an FMA chain, each group
    // sum into the lane's partial by one Kahan step
    auto batch = [&](const uint32_t (&eb)[kBatch], const float4 (&sj)[kBatch]) {
        float gx = 0.f, gy = 0.f, gz = 0.f, gp = 0.f;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            float tx, ty, tz, tp;
            terms(eb[u], sj[u], tx, ty, tz, tp);
            if (u % G == 0) {
                gx = tx; gy = ty; gz = tz; gp = tp;
            } else {
                gx += tx; gy += ty; gz += tz; gp += tp;
            }
            if (u % G == G - 1) {
                kahan_add(acc.fx, acc.cx, gx);
                kahan_add(acc.fy, acc.cy, gy);
                kahan_add(acc.fz, acc.cz, gz);
                if (THERMO) kahan_add(acc.pe, acc.cp, gp);
            }
        }
    };
    // whole batches, then the remaining rows one at a time
    const int rows_full = rows / kBatch * kBatch;
    for (int q = 0; q < rows_full; q += kBatch) {
        uint32_t eb[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) eb[u] = Lr[(q + u) * 32];
        float4 sj[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) sj[u] = gather_shadow<VL, ONE>(a, eb[u]);
        batch(eb, sj);
    }
    for (int q = rows_full; q < rows; ++q) {
        const uint32_t en = Lr[q * 32];
        const float4 sj = gather_shadow<VL, ONE>(a, en);
        float tx, ty, tz, tp;
        terms(en, sj, tx, ty, tz, tp);
        kahan_add(acc.fx, acc.cx, tx);
        kahan_add(acc.fy, acc.cy, ty);
        kahan_add(acc.fz, acc.cz, tz);
        if (THERMO) kahan_add(acc.pe, acc.cp, tp);
    }
}

// The warp's stencil offsets (code `lane`; codes 27..31 unused: zero) for box B.
__device__ __forceinline__ void set_offsets(float (*off)[32], const Box &B, int lane) {
    const bool code = lane < 27;
    off[0][lane] = code ? (float)(lane % 3 - 1) * B.hf[0] : 0.f;
    off[1][lane] = code ? (float)((lane / 3) % 3 - 1) * B.hf[1] : 0.f;
    off[2][lane] = code ? (float)(lane / 9 - 1) * B.hf[2] : 0.f;
}

template <int T, bool ONE, bool THERMO, bool HALF, int VL>
__device__ __forceinline__ void mixed_body(const ForceArgs &a, const SmemTabs &tb,
                                           float (*s_off)[3][32], uint64_t (*s_bar)[2],
                                           uint32_t *lbuf) {
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwc = blockDim.x >> 5;
    const int64_t chunk = (a.nwt + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * chunk;
    const int64_t t1 = min(a.nwt, t0 + chunk);
    const MixedConst kc = mixed_const(a, tb);
    const size_t rowblk = (size_t)a.R * 32;  // words in one warp-tile's list block
    const uint64_t pol = l2_evict_first_policy();
    const uint32_t sbuf0 = (uint32_t)__cvta_generic_to_shared(lbuf + (size_t)wib * 2 * rowblk);
    const uint32_t bstride = (uint32_t)(rowblk * 4);  // bytes per buffer half
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[wib][0]);
    uint32_t phase = 0;  // bit k: parity of buffer k's next completion
    if (lane == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        fence_mbar_init();
    }
    __syncwarp();
    int64_t wt = t0 + wib;
    int rows_cur = 0;
    int nn_next = 0;  // the next tile's count for this lane's atom, loaded a tile ahead
    float4 si_next = make_float4(0.f, 0.f, 0.f, 0.f);  // the next tile's home shadow, likewise
    int b_next = 0;  // and its box
    int64_t box_slot = 0;
    int32_t box_n = 0;
    if (wt < t1) {
        b_next = a.tile_box[(wt * A) >> 5];
        rows_cur = tile_rows<T>(min(__ldg(a.nn + wt * A + lane / T), a.pad));
        if (lane == 0) bulk_rows(sbuf0, a.nbr + wt * rowblk, rows_cur, bar0, pol, a.tx_extra);
        if (wt + nwc < t1) nn_next = __ldg(a.nn + (wt + nwc) * A + lane / T);
        si_next = a.sh_in[wt * A + lane / T];
    }
    int cb = 0;
    int curbox = -1;
    for (; wt < t1; wt += nwc) {
        const int64_t wn = wt + nwc;
        const bool has_next = wn < t1;
        int rows_next = 0;
        if (has_next) {
            rows_next = tile_rows<T>(min(nn_next, a.pad));
            if (lane == 0)
                bulk_rows(sbuf0 + (cb ^ 1) * bstride, a.nbr + wn * rowblk, rows_next,
                          bar0 + 8 * (cb ^ 1), pol, a.tx_extra);
        }
        // the count of the tile after next, in flight while this tile runs
        nn_next = wn + nwc < t1 ? __ldg(a.nn + (wn + nwc) * A + lane / T) : 0;
        const int64_t i = wt * A + lane / T;
        const int b = b_next;
        if (has_next) b_next = a.tile_box[(wn * A) >> 5];
        if (b != curbox) {
            const Box &B = a.boxes[b];
            set_offsets(s_off[wib], B, lane);
            box_slot = B.slot_off;
            box_n = B.n;
            curbox = b;
        }
        const bool valid = (i - box_slot) < box_n;
        const float4 si = si_next;
        if (has_next) si_next = a.sh_in[wn * A + lane / T];
        const int ti = ONE ? 0 : __float_as_int(si.w);
        // one lane per atom holds three components: there the registers are
        // worth more to the rows (long ones) than the early loads (half lists:
        // the epilogue is another kernel's)
        constexpr bool kPre = T >= 2 && !HALF;
        TileState<T> st;
        if (kPre) load_tile_state<T>(a, i, valid, st);
        // the current tile's rows have landed; a wait that runs out abandons
        // the step with a timeout status (after waiting, again bounded, for
        // the copy in flight into the other half)
        if (!mbar_wait(bar0 + 8 * cb, (phase >> cb) & 1u)) {
            atomicOr(&a.fl->status, ST_TIMEOUT);
            if (has_next) mbar_wait(bar0 + 8 * (cb ^ 1), (phase >> (cb ^ 1)) & 1u);
            return;
        }
        phase ^= 1u << cb;
        __syncwarp();  // s_off is visible to the whole warp
        Acc acc;
        lane_rows<ONE, THERMO, HALF, VL>(a, tb, kc, s_off[wib],
                               lbuf + (size_t)wib * 2 * rowblk + cb * rowblk + lane, rows_cur, si,
                               ti, acc);
        __syncwarp();  // done reading this half; the next copy may refill it
        // each lane folds its compensation (value = s - c); the T lane
        // partials of an atom are then added in a fixed xor-shuffle order
        const float Ff[3] = {sum_lanes_f<T>(acc.fx - acc.cx), sum_lanes_f<T>(acc.fy - acc.cy),
                             sum_lanes_f<T>(acc.fz - acc.cz)};
        if (HALF) {
            // the atom's own sums join the reactions in its accumulator
            const float pf = THERMO ? sum_lanes_f<T>(acc.pe - acc.cp) : 0.0f;
            if (valid && lane % T == 0) red_add4(a.facc + i, Ff[0], Ff[1], Ff[2], pf);
        } else {
            const double ped = THERMO ? (double)sum_lanes_f<T>(acc.pe - acc.cp) : 0.0;
            finish_tile<T, THERMO, kPre>(a, tb, wt, i, valid, ti, Ff, ped, st);
        }
        cb ^= 1;
        rows_cur = rows_next;
    }
}

// Rows [0, r0) and [0, r1) of two list blocks (128 bytes a row) -> shared
// dst0 and dst1 as two bulk copies completing on one mbarrier (one arrival
// posting both byte counts).  One lane only.
__device__ __forceinline__ void bulk_rows2(uint32_t dst0, const uint32_t *src0, int r0,
                                           uint32_t dst1, const uint32_t *src1, int r1,
                                           uint32_t bar, uint64_t pol, uint32_t extra) {
    const uint32_t b0 = (uint32_t)r0 * 128u, b1 = (uint32_t)r1 * 128u;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                 "r"(b0 + b1 + extra)
                 : "memory");
    if (b0 > 0)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
            "[%0], [%1], %2, [%3], %4;\n" ::"r"(dst0),
            "l"(src0), "r"(b0), "r"(bar), "l"(pol)
            : "memory");
    if (b1 > 0)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
            "[%0], [%1], %2, [%3], %4;\n" ::"r"(dst1),
            "l"(src1), "r"(b1), "r"(bar), "l"(pol)
            : "memory");
}

// Eight lanes per atom on the 8-lane list layout (4 atoms per list block),
// walked in tiles of 8 atoms: the two blocks of a tile arrive by one pair of
// bulk copies, then the 8 lanes of each group take atom g of the first block
// and, in a second pass, atom 4 + g of the second.  One gather instruction
// then covers 4 atoms x 8 consecutive list entries instead of 8 atoms x 4: a
// quarter-warp (8 lanes) reads one atom's run of neighbors, which touches
// fewer distinct 128-byte lines.  The epilogue runs once per 8 atoms with 4
// lanes per atom (as the 4-lane traversal), the forces moved there by shuffles.
template <bool ONE, bool THERMO>
__device__ __forceinline__ void mixed_body_pairs(const ForceArgs &a, const SmemTabs &tb,
                                                 float (*s_off)[3][32], uint64_t (*s_bar)[2],
                                                 uint32_t *lbuf) {
    constexpr int T = 8;  // the list layout (4 atoms per block)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, g = lane >> 3;
    const int nwc = blockDim.x >> 5;
    const int64_t nst = a.nwt / 2;  // tiles of 8 atoms (block pairs)
    const int64_t chunk = (nst + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * chunk;
    const int64_t t1 = min(nst, t0 + chunk);
    const MixedConst kc = mixed_const(a, tb);
    const size_t rowblk = (size_t)a.R * 32;  // words in one list block
    const uint64_t pol = l2_evict_first_policy();
    uint32_t *wbuf = lbuf + (size_t)wib * 4 * rowblk;  // 2 halves x 2 blocks
    const uint32_t sbuf0 = (uint32_t)__cvta_generic_to_shared(wbuf);
    const uint32_t bbytes = (uint32_t)(rowblk * 4);  // bytes per block
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[wib][0]);
    uint32_t phase = 0;
    if (lane == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int64_t st, int half, int r0, int r1) {
        if (lane == 0)
            bulk_rows2(sbuf0 + (uint32_t)half * 2u * bbytes, a.nbr + (2 * st) * rowblk, r0,
                       sbuf0 + (uint32_t)half * 2u * bbytes + bbytes, a.nbr + (2 * st + 1) * rowblk,
                       r1, bar0 + 8 * half, pol, a.tx_extra);
    };
    int64_t st = t0 + wib;
    int rows0 = 0, rows1 = 0;
    int nn0_next = 0, nn1_next = 0;
    float4 s0_next = make_float4(0.f, 0.f, 0.f, 0.f), s1_next = s0_next;
    int b_next = 0;
    int64_t box_slot = 0;
    int32_t box_n = 0;
    if (st < t1) {
        b_next = a.tile_box[(st * 8) >> 5];
        rows0 = tile_rows<T>(min(__ldg(a.nn + st * 8 + g), a.pad));
        rows1 = tile_rows<T>(min(__ldg(a.nn + st * 8 + 4 + g), a.pad));
        issue(st, 0, rows0, rows1);
        if (st + nwc < t1) {
            nn0_next = __ldg(a.nn + (st + nwc) * 8 + g);
            nn1_next = __ldg(a.nn + (st + nwc) * 8 + 4 + g);
        }
        s0_next = a.sh_in[st * 8 + g];
        s1_next = a.sh_in[st * 8 + 4 + g];
    }
    int cb = 0;
    int curbox = -1;
    for (; st < t1; st += nwc) {
        const int64_t sn = st + nwc;
        const bool has_next = sn < t1;
        int r0n = 0, r1n = 0;
        if (has_next) {
            r0n = tile_rows<T>(min(nn0_next, a.pad));
            r1n = tile_rows<T>(min(nn1_next, a.pad));
            issue(sn, cb ^ 1, r0n, r1n);
        }
        if (sn + nwc < t1) {
            nn0_next = __ldg(a.nn + (sn + nwc) * 8 + g);
            nn1_next = __ldg(a.nn + (sn + nwc) * 8 + 4 + g);
        }
        const int b = b_next;
        if (has_next) b_next = a.tile_box[(sn * 8) >> 5];
        if (b != curbox) {
            const Box &B = a.boxes[b];
            set_offsets(s_off[wib], B, lane);
            box_slot = B.slot_off;
            box_n = B.n;
            curbox = b;
        }
        const float4 s0 = s0_next, s1 = s1_next;
        if (has_next) {
            s0_next = a.sh_in[sn * 8 + g];
            s1_next = a.sh_in[sn * 8 + 4 + g];
        }
        const int ti0 = ONE ? 0 : __float_as_int(s0.w), ti1 = ONE ? 0 : __float_as_int(s1.w);
        // the epilogue's atom: 4 lanes each, lane 4e + d takes component d
        const int64_t ie = st * 8 + (lane >> 2);
        const bool valid_e = (ie - box_slot) < box_n;
        TileState<4> ts;
        load_tile_state<4>(a, ie, valid_e, ts);
        if (!mbar_wait(bar0 + 8 * cb, (phase >> cb) & 1u)) {
            atomicOr(&a.fl->status, ST_TIMEOUT);
            if (has_next) mbar_wait(bar0 + 8 * (cb ^ 1), (phase >> (cb ^ 1)) & 1u);
            return;
        }
        phase ^= 1u << cb;
        __syncwarp();
        const uint32_t *Lb = wbuf + (size_t)cb * 2 * rowblk + lane;
        Acc acc0, acc1;
        lane_rows<ONE, THERMO, false>(a, tb, kc, s_off[wib], Lb, rows0, s0, ti0, acc0);
        lane_rows<ONE, THERMO, false>(a, tb, kc, s_off[wib], Lb + rowblk, rows1, s1, ti1, acc1);
        __syncwarp();  // done reading this half
        const float F0[3] = {sum_lanes_f<T>(acc0.fx - acc0.cx), sum_lanes_f<T>(acc0.fy - acc0.cy),
                             sum_lanes_f<T>(acc0.fz - acc0.cz)};
        const float F1[3] = {sum_lanes_f<T>(acc1.fx - acc1.cx), sum_lanes_f<T>(acc1.fy - acc1.cy),
                             sum_lanes_f<T>(acc1.fz - acc1.cz)};
        // atom e = lane / 4 of the tile: group e of the first pass (e < 4) or
        // group e - 4 of the second
        const int src = 8 * ((lane >> 2) & 3);
        const bool second = lane >= 16;
        float Fe[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float u0 = __shfl_sync(0xffffffffu, F0[d], src);
            const float u1 = __shfl_sync(0xffffffffu, F1[d], src);
            Fe[d] = second ? u1 : u0;
        }
        double ped = 0.0;
        if (THERMO) {
            const float p0 = __shfl_sync(0xffffffffu, sum_lanes_f<T>(acc0.pe - acc0.cp), src);
            const float p1 = __shfl_sync(0xffffffffu, sum_lanes_f<T>(acc1.pe - acc1.cp), src);
            ped = (double)(second ? p1 : p0);
        }
        int te = 0;
        if (!ONE) {
            const int u0 = __shfl_sync(0xffffffffu, ti0, src), u1 = __shfl_sync(0xffffffffu, ti1, src);
            te = second ? u1 : u0;
        }
        // thermo partials: the tile's in the slot of its first block, zero in
        // the second's
        finish_tile<4, THERMO, true>(a, tb, 2 * st, ie, valid_e, te, Fe, ped, ts);
        if (THERMO && lane < TP) a.tpart[(2 * st + 1) * TP + lane] = 0.0;
        cb ^= 1;
        rows0 = r0n;
        rows1 = r1n;
    }
}

// Frozen (a list overflowed, a position went non-finite or a wait ran out
// earlier in this run): keep the state and mirror it into the output buffers
// so the buffer flip stays valid.
__device__ __forceinline__ void mirror_state(const ForceArgs &a) {
    if (a.mode != MODE_FUSED) return;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.ns;
         t += (int64_t)gridDim.x * blockDim.x) {
        a.sh_out[t] = a.sh_in[t];
        for (int d = 0; d < 3; ++d) a.r_out[d * a.ns + t] = a.r_in[d * a.ns + t];
    }
}

__device__ __forceinline__ void load_tabs(const Pair &P, SmemTabs &tb) {
    for (int t = threadIdx.x; t < 64; t += blockDim.x) {
        tb.fs2[t] = P.fs2[t]; tb.fe4[t] = P.fe4[t]; tb.fush[t] = P.fush[t]; tb.fc1[t] = P.fc1[t];
        tb.de24[t] = P.e24[t]; tb.ds2[t] = P.s2[t]; tb.de4[t] = P.e4[t]; tb.dush[t] = P.ush[t];
        if (t < MD_MAXT) { tb.dtm[t] = P.dtm[t]; tb.hdtm[t] = P.hdtm[t]; tb.mass[t] = P.mass[t]; }
    }
}

// The last CTA to finish records which step the thermo partials describe and,
// in FUSED mode, advances the step clock (every CTA has read it).
__device__ __forceinline__ void kernel_done(const ForceArgs &a, int64_t clock, bool thermo) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(a.done, 1u);
        if (prev == gridDim.x - 1) {
            *a.done = 0u;
            a.fl->thermo = thermo ? 1u : 0u;
            if (a.mode == MODE_FUSED) a.fl->clock = clock + 1;
        }
    }
}

// Register budget: the share of MD_FORCE_MINB resident 128-thread CTAs per SM,
// rounded down to the allocation granule of 8 (80 at 6); CTAs of 64 to 768
// threads (kMaxWarpsMixed warps) fit it.
#define MD_FORCE_MAXREG (65536 / (MD_FORCE_MINB * 128) / 8 * 8)
static_assert(MD_FORCE_MAXREG * kMaxWarpsMixed * 32 <= 65536, "a full-size CTA must fit the SM");

template <int T, bool ONE, bool HALF, int VL>
__global__ void __maxnreg__(MD_FORCE_MAXREG) k_force_mixed(ForceArgs a) {
    if (a.fl->status & ST_FREEZE) {
        if (!HALF) mirror_state(a);  // half lists: the epilogue kernel mirrors
        return;
    }
    extern __shared__ __align__(128) uint32_t lbuf[];
    __shared__ SmemTabs tb;
    __shared__ __align__(16) float s_off[kMaxWarpsMixed][3][32];
    __shared__ __align__(8) uint64_t s_bar[kMaxWarpsMixed][2];
    load_tabs(*a.pair, tb);
    __syncthreads();
    const int64_t clock = a.fl->clock;
    const bool thermo = a.mode != MODE_FUSED || (a.thermo_every > 0 && clock % a.thermo_every == 0);
    if constexpr (T == 8) {
        if (thermo) mixed_body_pairs<ONE, true>(a, tb, s_off, s_bar, lbuf);
        else mixed_body_pairs<ONE, false>(a, tb, s_off, s_bar, lbuf);
    } else {
        if (thermo) mixed_body<T, ONE, true, HALF, VL>(a, tb, s_off, s_bar, lbuf);
        else mixed_body<T, ONE, false, HALF, VL>(a, tb, s_off, s_bar, lbuf);
    }
    if (!HALF) kernel_done(a, clock, thermo);
}

// The AoSoA copy of the shadows (slots 0..ns, the sentinel's included): slot i
// in block i / VL at lane i % VL of each component array.
template <int VL>
__global__ void k_shadow_aosoa(const float4 *__restrict__ sh, float *__restrict__ shv, int64_t m,
                               const Flags *fl) {
    if (fl->status & ST_FREEZE) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float4 s = sh[i];
    float *p = shv + (i / VL) * (4 * VL) + (i % VL);
    p[0] = s.x;
    p[VL] = s.y;
    p[2 * VL] = s.z;
    p[3 * VL] = s.w;
}

// Half lists, after k_force_mixed<4, ONE, true>: each slot's accumulator holds
// its force and half-energy sums (own terms and the reactions of the atoms
// that list it); the epilogue of the 4-lane traversal runs on them (warp-tiles
// of 8 atoms, lane 4e + d takes component d of atom e) and the accumulators
// are cleared for the next evaluation.
template <bool ONE>
__global__ void __launch_bounds__(256) k_half_epilogue(ForceArgs a) {
    if (a.fl->status & ST_FREEZE) {
        mirror_state(a);
        return;
    }
    __shared__ SmemTabs tb;
    load_tabs(*a.pair, tb);
    __syncthreads();
    const int64_t clock = a.fl->clock;
    const bool thermo = a.mode != MODE_FUSED || (a.thermo_every > 0 && clock % a.thermo_every == 0);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t wt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wt < a.nwt;
         wt += nw) {
        const int64_t i = wt * 8 + (lane >> 2);
        const Box &B = a.boxes[a.tile_box[(wt * 8) >> 5]];
        const bool valid = (i - B.slot_off) < B.n;
        const float4 fa = a.facc[i];
        __syncwarp();
        if ((lane & 3) == 0) a.facc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int ti = ONE ? 0 : a.type[i];
        const float F[3] = {fa.x, fa.y, fa.z};
        TileState<4> st;
        if (thermo) finish_tile<4, true, false>(a, tb, wt, i, valid, ti, F, (double)fa.w, st);
        else finish_tile<4, false, false>(a, tb, wt, i, valid, ti, F, 0.0, st);
    }
    kernel_done(a, clock, thermo);
}

template <int T, bool ONE, bool HALF>
__global__ void __launch_bounds__(kBlock64, 2) k_force64(ForceArgs a) {
    if (a.fl->status & ST_FREEZE) {
        if (!HALF) mirror_state(a);  // half lists: the epilogue kernel mirrors
        return;
    }
    __shared__ SmemTabs tb;
    __shared__ __align__(16) double s_offd[kMaxWarps][81];
    __shared__ float s_offf64[kMaxWarps][81];
    load_tabs(*a.pair, tb);
    __syncthreads();
    const int64_t clock = a.fl->clock;
    const bool thermo = a.mode != MODE_FUSED || (a.thermo_every > 0 && clock % a.thermo_every == 0);
    if (thermo) force_body64<T, ONE, true, HALF>(a, tb, s_offd, s_offf64);
    else force_body64<T, ONE, false, HALF>(a, tb, s_offd, s_offf64);
    if (!HALF) kernel_done(a, clock, thermo);
}

// Half lists in an FP64 context, after k_force64<4, ONE, true>: as
// k_half_epilogue, on the FP64 accumulators (x, y, z, energy per slot).
template <bool ONE>
__global__ void __launch_bounds__(256) k_half_epilogue64(ForceArgs a) {
    if (a.fl->status & ST_FREEZE) {
        mirror_state(a);
        return;
    }
    __shared__ SmemTabs tb;
    load_tabs(*a.pair, tb);
    __syncthreads();
    const int64_t clock = a.fl->clock;
    const bool thermo = a.mode != MODE_FUSED || (a.thermo_every > 0 && clock % a.thermo_every == 0);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t wt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wt < a.nwt;
         wt += nw) {
        const int64_t i = wt * 8 + (lane >> 2);
        const Box &B = a.boxes[a.tile_box[(wt * 8) >> 5]];
        const bool valid = (i - B.slot_off) < B.n;
        double *pi = a.facc64 + 4 * i;
        const double F[3] = {pi[0], pi[1], pi[2]};
        const double e = pi[3];
        __syncwarp();
        if ((lane & 3) == 0) {
            pi[0] = 0.0; pi[1] = 0.0; pi[2] = 0.0; pi[3] = 0.0;
        }
        const int ti = ONE ? 0 : a.type[i];
        TileState<4> st;
        if (thermo) finish_tile<4, true, false>(a, tb, wt, i, valid, ti, F, e, st);
        else finish_tile<4, false, false>(a, tb, wt, i, valid, ti, F, 0.0, st);
    }
    kernel_done(a, clock, thermo);
}

// v += dt/2 F/m; x += dt v; shadow refresh.  From a READY state.
__global__ void k_kick_drift(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                             const Pair *__restrict__ pair, int64_t ns,
                             const int32_t *__restrict__ type, const double *__restrict__ f,
                             double *__restrict__ v, const double *__restrict__ r_in,
                             double *__restrict__ r_out, float4 *__restrict__ sh_out, Flags *fl) {
    if (fl->status & ST_FREEZE) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) fl->clock += 1;
    if (i >= ns) return;
    const Box &B = boxes[tile_box[i >> 5]];
    const int ty = type[i];
    float s[3] = {0.f, 0.f, 0.f};
    if (i - B.slot_off < B.n) {
        const double hdtm = pair->hdtm[ty], dt = pair->dt;
        for (int d = 0; d < 3; ++d) {
            const int64_t o = d * ns + i;
            const double vv = fma(hdtm, f[o], v[o]);
            v[o] = vv;
            const double rn = fma(dt, vv, r_in[o]);
            r_out[o] = rn;
            s[d] = __double2float_rn(rn);
        }
    } else {
        for (int d = 0; d < 3; ++d) r_out[d * ns + i] = 0.0;
    }
    sh_out[i] = make_float4(s[0], s[1], s[2], __int_as_float(ty));
}

// Thermo reduction in two fixed-order levels: CTA (b, s) sums the s-th of
// `split` contiguous ranges of box b's warp-tile partials; then one CTA per box
// sums its `split` results in order.  Deterministic for a given split.
__global__ void __launch_bounds__(256) k_finalize_part(const Box *__restrict__ boxes, int A,
                                                       int split, const double *__restrict__ tpart,
                                                       double *__restrict__ fpart, const Flags *fl) {
    if (fl->status & ST_FREEZE) return;
    if (fl->thermo == 0u) return;  // the force kernel computed no thermo this step
    const int b = blockIdx.x / split, s = blockIdx.x % split;
    const Box &B = boxes[b];
    const int64_t w0 = B.slot_off / A, w1 = (B.slot_off + B.npad) / A;
    const int64_t chunk = (w1 - w0 + split - 1) / split;
    const int64_t lo = w0 + s * chunk, hi = min(w1, lo + chunk);
    __shared__ double red[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t w = lo + threadIdx.x; w < hi; w += blockDim.x) {
        const double *tp = tpart + w * TP;
        for (int q = 0; q < 5; ++q) acc[q] += tp[q];
        acc[5] = fmax(acc[5], tp[5]);
    }
    for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int h = 128; h >= 1; h >>= 1) {
        if (threadIdx.x < h) {
            for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
            red[5][threadIdx.x] = fmax(red[5][threadIdx.x], red[5][threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) fpart[(size_t)blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_finalize(int split, const double *__restrict__ fpart,
                           double *__restrict__ tbox, Flags *fl, double *__restrict__ tlog,
                           int32_t tlog_cap, int thermo_every, int mode) {
    if (fl->status & ST_FREEZE) return;
    if (fl->thermo == 0u) return;
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < split; ++s) {
        const double *p = fpart + ((size_t)b * split + s) * 6;
        for (int q = 0; q < 5; ++q) acc[q] += p[q];
        acc[5] = fmax(acc[5], p[5]);
    }
    // step the numbers describe: FUSED already advanced the clock
    const int64_t step = fl->clock - (mode == MODE_FUSED ? 1 : 0);
    double *tb = tbox + b * TB;
    for (int q = 0; q < 5; ++q) tb[q] = acc[q];
    tb[5] = sqrt(acc[5]);
    tb[6] = (double)step;
    if (b == 0 && thermo_every > 0 && step % thermo_every == 0) {
        const int64_t row = step / thermo_every;
        if (row < tlog_cap) {
            tlog[4 * row + 0] = (double)step;
            tlog[4 * row + 1] = acc[0];
            tlog[4 * row + 2] = acc[1];
            tlog[4 * row + 3] = acc[0] + acc[1];
        }
    }
}

__global__ void k_get_state(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                            const double *__restrict__ ctab, int64_t ns,
                            const double *__restrict__ r,
                            const int32_t *__restrict__ cellc, const double *__restrict__ v,
                            const double *__restrict__ f, const int32_t *__restrict__ img,
                            const int32_t *__restrict__ id, double *__restrict__ xo,
                            double *__restrict__ vo, double *__restrict__ fo,
                            int32_t *__restrict__ imgo, int32_t *__restrict__ ido,
                            const int32_t *__restrict__ ty, int32_t *__restrict__ tyo) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const Box &B = boxes[tile_box[k >> 5]];
    const int64_t loc = k - B.slot_off;
    if (loc >= B.n) return;
    const int64_t g = id[k];
    int cc[3];
    unpack_cell(cellc[k], cc[0], cc[1], cc[2]);
    for (int d = 0; d < 3; ++d) {
        if (xo) xo[3 * g + d] = __dadd_rn(cell_centre(ctab, B, d, cc[d]), r[d * ns + k]);
        if (vo) vo[3 * g + d] = v[d * ns + k];
        if (fo) fo[3 * g + d] = f[d * ns + k];
        if (imgo) imgo[3 * g + d] = img[d * ns + k];
    }
    if (ido) ido[B.atom_base + loc] = (int32_t)g;
    if (tyo) tyo[g] = ty[k];
}

__global__ void k_get_neighbors(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                                int64_t ns, int T, int R, int pad, const int32_t *__restrict__ nn,
                                const uint32_t *__restrict__ nbr, int pad_out,
                                int32_t *__restrict__ nn_out, int32_t *__restrict__ nbr_out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const Box &B = boxes[tile_box[i >> 5]];
    const int64_t loc = i - B.slot_off;
    if (loc >= B.n) return;
    const int64_t u = B.atom_base + loc;
    const int cnt = nn[i];
    if (nn_out) nn_out[u] = cnt;
    if (!nbr_out) return;
    const int A = 32 / T;
    const int m = min(cnt, min(pad, pad_out));
    for (int k = 0; k < m; ++k) {
        const uint32_t e = nbr[((size_t)(i / A) * R + k / T) * 32 + (i % A) * T + k % T];
        const int64_t j = e & MD_IDX_MASK;
        nbr_out[u * pad_out + k] = (int32_t)(B.atom_base + (j - B.slot_off));
    }
}

// Mixed-kernel CTA size when md_params.block_threads is 0.  Every size below
// keeps 24 warps per SM under the register cap (1 x 768, 2 x 384, 3 x 256,
// 6 x 128 threads); the largest is best on B300 (one CTA per SM walks one
// contiguous run of warp-tiles, so all 24 warps share neighbors in L1: 0.79 ms
// vs 0.81-0.83 ms at 256 for the 4M-atom melt), but a CTA must leave every SM
// some tiles and its list buffers must fit in shared memory.
constexpr size_t kSmemDyn = 200 * 1024;  // dynamic shared memory a mixed-kernel CTA may take

int auto_block_mixed(const md_ctx *c, int64_t nwt, size_t per_warp_smem) {
    static const int sizes[] = {768, 384, 256, 128, 64};
    for (int b : sizes) {
        const int w = b / 32;
        if ((size_t)w * per_warp_smem <= kSmemDyn && nwt >= (int64_t)w * c->nsm) return b;
    }
    return 64;
}

template <bool MIXED, int T, bool ONE, bool HALF = false, int VL = 0>
cudaError_t launch_force_t(md_ctx *c, const ForceArgs &a) {
    if constexpr (MIXED) {
        // Each warp has a double buffer of R list rows in shared memory (of two
        // list blocks with 8 lanes per atom).
        const int64_t units = T == 8 ? a.nwt / 2 : a.nwt;  // tiles a warp takes in turn
        const size_t per_warp = (size_t)(T == 8 ? 4 : 2) * a.R * 32 * sizeof(uint32_t);
        int block = c->block ? c->block : auto_block_mixed(c, units, per_warp);
        // an explicit size is an upper bound: fewer warps when their buffers
        // would not fit in shared memory
        while (block > 32 && (size_t)(block / 32) * per_warp > kSmemDyn) block -= 32;
        const int warps = block / 32;
        const size_t smem = (size_t)warps * per_warp;
        // process-wide: the kernel's shared-memory limit and the last occupancy query
        static std::mutex mu;
        static size_t smem_set = 0, occ_smem = 0;
        static int occ = 0, occ_block = 0;
        int per_sm;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (smem > smem_set) {
                cudaError_t e = cudaFuncSetAttribute(
                    k_force_mixed<T, ONE, HALF, VL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                smem_set = smem;
            }
            if (occ_smem != smem || occ_block != block) {
                int per = 0;
                cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, k_force_mixed<T, ONE, HALF, VL>, block, smem);
                if (e != cudaSuccess) return e;
                occ = per > 0 ? per : 1;
                occ_smem = smem;
                occ_block = block;
            }
            per_sm = occ;
        }
        int64_t grid = (int64_t)c->nsm * per_sm;
        const int64_t need = (units + warps - 1) / warps;
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        if constexpr (VL > 0) {
            const int64_t m = c->ns + 1;
            k_shadow_aosoa<VL><<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(a.sh_in, c->shv,
                                                                                   m, a.fl);
            c->kernels += 1;
        }
        k_force_mixed<T, ONE, HALF, VL><<<(unsigned)grid, block, smem, c->stream>>>(a);
        if constexpr (HALF) {
            const int64_t blocks = std::min<int64_t>((a.nwt + 7) / 8, (int64_t)c->nsm * 8);
            k_half_epilogue<ONE><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
            c->kernels += 1;
        }
    } else {
        const int block = c->block ? std::min(c->block, kBlock64) : kBlock64;
        static std::atomic<int> grid_cache[kMaxWarps + 1] = {};  // per CTA size
        int g = grid_cache[block / 32].load(std::memory_order_relaxed);
        if (g == 0) {
            int per = 0;
            cudaError_t e =
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_force64<T, ONE, HALF>, block, 0);
            if (e != cudaSuccess) return e;
            g = per > 0 ? per : 1;
            grid_cache[block / 32].store(g, std::memory_order_relaxed);
        }
        const int64_t warps_per_block = block / 32;
        int64_t grid = (int64_t)c->nsm * g;
        const int64_t need = (a.nwt + warps_per_block - 1) / warps_per_block;
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        k_force64<T, ONE, HALF><<<(unsigned)grid, block, 0, c->stream>>>(a);
        if constexpr (HALF) {
            const int64_t blocks = std::min<int64_t>((a.nwt + 7) / 8, (int64_t)c->nsm * 8);
            k_half_epilogue64<ONE><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
            c->kernels += 1;
        }
    }
    c->kernels += 1;
    return cudaGetLastError();
}

template <bool MIXED>
cudaError_t launch_force_m(md_ctx *c, const ForceArgs &a) {
    const bool one = c->hpair.nt == 1;
    if (c->params.half_list) {  // 4 lanes per atom (checked at create)
        return one ? launch_force_t<MIXED, 4, true, true>(c, a)
                   : launch_force_t<MIXED, 4, false, true>(c, a);
    }
    if (MIXED && c->params.shadow_vl == 8) {  // 4 lanes per atom (checked at create)
        return one ? launch_force_t<true, 4, true, false, 8>(c, a)
                   : launch_force_t<true, 4, false, false, 8>(c, a);
    }
    if (MIXED && c->params.shadow_vl == 32) {
        return one ? launch_force_t<true, 4, true, false, 32>(c, a)
                   : launch_force_t<true, 4, false, false, 32>(c, a);
    }
    switch (c->T) {
        case 1: return one ? launch_force_t<MIXED, 1, true>(c, a) : launch_force_t<MIXED, 1, false>(c, a);
        case 2: return one ? launch_force_t<MIXED, 2, true>(c, a) : launch_force_t<MIXED, 2, false>(c, a);
        case 4: return one ? launch_force_t<MIXED, 4, true>(c, a) : launch_force_t<MIXED, 4, false>(c, a);
        case 8: return one ? launch_force_t<MIXED, 8, true>(c, a) : launch_force_t<MIXED, 8, false>(c, a);
        default: return cudaErrorInvalidValue;
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_force(md_ctx *c, int mode) {
    ForceArgs a;
    a.boxes = c->dbox;
    a.tile_box = c->tile_box;
    a.pair = c->dpair;
    a.ns = c->ns;
    a.nwt = c->ns / (32 / c->T);
    a.pad = c->pad;
    a.R = c->R;
    a.sh_in = c->sh[c->pc];
    a.sh_out = c->sh[c->pc ^ 1];
    a.r_in = c->r[c->pc];
    a.r_out = c->r[c->pc ^ 1];
    a.v = c->v[c->oc];
    a.f = c->f;
    a.rbuild = c->rbuild;
    a.type = c->type[c->oc];
    a.nn = c->nn;
    a.nbr = c->nbr;
    a.tpart = c->tpart;
    a.fl = c->dflags;
    a.mode = mode;
    a.thermo_every = c->params.thermo_every;
    a.done = &c->dflags->done;
    a.tx_extra = c->debug_tx_extra;
    a.facc = c->facc;
    a.facc64 = c->facc64;
    a.shv = c->shv;
    cudaError_t e = c->params.precision == MD_MIXED ? launch_force_m<true>(c, a)
                                                    : launch_force_m<false>(c, a);
    if (e == cudaSuccess && mode == MODE_FUSED) c->pc ^= 1;
    return e;
}

cudaError_t launch_kick_drift(md_ctx *c) {
    const int t = 256;
    k_kick_drift<<<blocks_for(c->ns, t), t, 0, c->stream>>>(
        c->dbox, c->tile_box, c->dpair, c->ns, c->type[c->oc], c->f, c->v[c->oc], c->r[c->pc],
        c->r[c->pc ^ 1], c->sh[c->pc ^ 1], c->dflags);
    c->pc ^= 1;
    c->kernels += 1;
    return cudaGetLastError();
}

cudaError_t launch_finalize(md_ctx *c, int mode) {
    k_finalize_part<<<c->nbox * c->fsplit, 256, 0, c->stream>>>(c->dbox, 32 / c->T, c->fsplit,
                                                                 c->tpart, c->fpart, c->dflags);
    k_finalize<<<c->nbox, 32, 0, c->stream>>>(c->fsplit, c->fpart, c->tbox, c->dflags, c->tlog,
                                              c->tlog_cap, c->params.thermo_every, mode);
    c->kernels += 2;
    return cudaGetLastError();
}

cudaError_t launch_get_state(md_ctx *c, double *x_aos, double *v_aos, double *f_aos,
                             int32_t *img_aos, int32_t *ids, int32_t *types) {
    const int t = 256;
    k_get_state<<<blocks_for(c->ns, t), t, 0, c->stream>>>(
        c->dbox, c->tile_box, c->ctab, c->ns, c->r[c->pc], c->cellc[c->oc], c->v[c->oc], c->f,
        c->img[c->oc], c->id[c->oc], x_aos, v_aos, f_aos, img_aos, ids, c->type[c->oc], types);
    return cudaGetLastError();
}

cudaError_t launch_get_neighbors(md_ctx *c, int32_t *nn_out, int32_t *nbr_out, int pad_out) {
    const int t = 256;
    k_get_neighbors<<<blocks_for(c->ns, t), t, 0, c->stream>>>(
        c->dbox, c->tile_box, c->ns, c->T, c->R, c->pad, c->nn, c->nbr, pad_out, nn_out, nbr_out);
    return cudaGetLastError();
}

}  // namespace mdb

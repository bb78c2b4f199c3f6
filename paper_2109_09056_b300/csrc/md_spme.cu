// md_spme.cu -- long-range Coulomb by smooth particle mesh Ewald (SPME) on a
// single-box context (include/md_spme.h).
//
// The paper's CabanaMD section lists the steps: B-spline spreading of the
// charges onto a uniform grid, 3-D FFTs for the reciprocal-space energy and
// forces, a gradient gather back onto the atoms, and real-space pairs over the
// short-range neighbor list.  Definitions from Essmann et al., J. Chem. Phys.
// 103, 8577 (1995), Secs. 2-4.
//
// Grid precision R follows the context: FP64 for MD_FP64 contexts; FP32 for
// MD_MIXED (FP32 spline weights, grid, single-precision FFTs and gather, FP64
// energy sums and force output).  B300's FP64 pipe runs at ~1/64 of FP32, so
// the FP64 FFTs are bound there, the FP32 ones by memory.
//
// One md_spme_compute is these launches on the context's stream:
//   k_spme_charges  charge of each slot's atom, gathered by its original id
//                   (mixed: also the slot's shadow with the charge in w);
//   k_spme_spread   one thread per slot: scaled fractional coordinates from the
//                   FP64 cell-relative position, order-p spline weights by their
//                   recursion, p^3 atomic adds into the grid Q (FP32 grid: each
//                   stencil row's consecutive points as float4/float2 adds);
//   k_spme_real     the real-space erfc pairs over the context's Verlet list
//                   (same warp-transposed rows and lanes per atom as the LJ
//                   kernels), FP64 or FP32 + Kahan by the context's precision;
//   k_fft_x_r2c, k_fft_lines  the forward FFT's x and y passes: Q -> Qhat
//                   (half spectrum, K_z x K_y x (K_x/2+1));
//   k_fft_z_influence  the z pass: each z line forward, its energy terms
//                   theta |Qhat|^2 (weighted 2 for the elements that stand for
//                   a conjugate pair), Qhat *= theta, back along z;
//   k_fft_lines, k_fft_x_c2r  the inverse's y and x passes -> dE/dQ on the
//                   grid (unnormalised inverse) (md_fft.cu, hand-written);
//   k_spme_gather   one thread per slot: spline gradients against dE/dQ, plus the
//                   slot's real-space force, written in original atom order;
// then one single-CTA sum of the energy partials (fixed order, deterministic).
// The real-space pass depends only on the charges: it runs on a side stream,
// forked after k_spme_charges and joined before the gather, beside the
// reciprocal chain (it is issue-bound, the chain atomic- and memory-bound);
// mixed, as a persistent grid of MD_SPME_REAL_CTAS CTAs per SM.  With
// profiling on, the launches run in order on one stream instead.
//
// md_spme_step integrates Coulomb + LJ with velocity Verlet: the context's
// kick + drift and its re-sort and list at the rebuild cadence, then one SPME
// evaluation whose real-space pass is fused with the LJ pair terms (one walk
// of the list writes F_LJ + F_real; the gather adds F_recip), then
// k_spme_half_kick closes the step.
#include "md_fft.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "md_common.cuh"
#include "md_trace.h"
#include "md_spme.h"

namespace mdb {  // md_api.cu
md_status ensure_list(md_ctx *c);
bool is_device_pointer(const void *p);
md_status resort_and_build(md_ctx *c);
md_status check_run_flags(md_ctx *c);
}  // namespace mdb

using namespace mdb;

namespace {

thread_local std::string g_spme_error;

constexpr int kThreads = 256;       // spread / gather / influence CTAs
constexpr int kRealBlock = 256;     // real-space CTA (8 warps)
constexpr int kMaxGrid = 4096;
constexpr int kRealBatch = 4;       // list entries per lane in flight (mixed real space)
#ifndef MD_SPME_REAL_CTAS
#define MD_SPME_REAL_CTAS 4   // the real-space kernel's register-limited residency
#endif
// persistent mixed real-space grid: this many CTAs per SM, at most the
// variant's residency (the fused LJ + Coulomb variant holds more registers)
constexpr int kRealCtasPerSm = MD_SPME_REAL_CTAS;
#ifndef MD_SPME_FUSED_CTAS
#define MD_SPME_FUSED_CTAS 3
#endif
// the same for the fused LJ + Coulomb pass (its residency at 80 registers;
// 1/2/3 per SM measured 6.70/4.52/4.42 ms per Coulomb + LJ step at 4M atoms)
constexpr int kFusedCtasPerSm = MD_SPME_FUSED_CTAS;
// FP64 real-space pair functions erfc(alpha r) and exp(-alpha^2 r^2) as
// piecewise polynomials on [0, rc]: kPieces equal intervals, degree kDeg64 in
// the interval's local coordinate t in [0, 1).  (B300's FP64 pipe: the
// library erfc and exp were 78% of the FP64 pass; the tables cut it 70.7 ->
// 31.1 ms at 4M atoms.  In FP32 the same tables, read with divergent interval
// indices, were 2% slower than erfcf and the exp intrinsic, which stay.)
// 64 pieces of degree 8 meet the fit's 1e-14 bar wherever 32 of degree 10 did
// (alpha rc up to ~10; host check at create) with 4 fewer DFMAs per pair.
constexpr int kPieces = 64;
constexpr int kDeg64 = 8;
constexpr int kTab64 = 2 * kPieces * (kDeg64 + 1);
// Mixed pass: erfc(x) = exp(-x^2) t H(s) on [0, alpha rc], with t = 1 / (1 + p x)
// (the form of Hastings' erfc approximations, Abramowitz & Stegun 7.1.26),
// s = (t - t_min) / (1 - t_min) in [0, 1] and H of degree kErfcDeg interpolated
// at Chebyshev nodes on the host for the solver's own range; the kernel reuses
// the exp(-x^2) that the force needs.  (B300, 4M atoms: erfcf was ~0.3 ms of a
// 4.3 ms Coulomb + LJ step.)  Used when its FP32 evaluation is within
// kErfcTol of erfc over the range, else erfcf.
constexpr int kErfcDeg = 7;
constexpr double kErfcP = 0.47;
constexpr double kErfcTol = 1e-6;
constexpr int kEvents = 7;
enum { kSpread = 0, kGatherOut = 1, kGatherAcc = 2 };

struct Geom {
    int32_t K[3];
    int32_t Kh;          // K_x / 2 + 1
    double Kd[3];        // K_d as double
    double kl[3];        // K_d / L_d
};

}  // namespace

struct md_spme {
    md_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;  // the context's stream (kept: destroy never reads ctx)
    md_spme_params p{};
    Geom g{};
    int64_t ngrid = 0, nhalf = 0;
    double *q = nullptr;        // charges, original atom order (n)
    double *qs = nullptr;       // charge per slot (ns)
    float4 *shq = nullptr;      // mixed: per slot the context's FP32 shadow with w = charge
                                // (ns + 1: the list's sentinel slot ns, far away, w = 0)
    bool f32 = false;           // grid precision R: FP32 (mixed context) or FP64
    void *grid = nullptr;       // Q, then dE/dQ: K_z x K_y x K_x of R
    void *ghat = nullptr;       // half spectrum, complex R
    void *theta = nullptr;      // influence function on the half spectrum, R
    double *fs = nullptr;       // real-space forces per slot, SoA 3 x ns
    double *tab64 = nullptr;    // FP64 pair-function polynomials (kTab64)
    float erfc_c[kErfcDeg + 1] = {};  // mixed: H's coefficients in s (see kErfcDeg)
    float erfc_sa = 0.f, erfc_sb = 0.f;  // s = sa t + sb
    bool erfc_fit = false;      // use H (else erfcf): see fit_erfc_mixed
    double erfc_err[2] = {0, 0};  // device check: max relative error of H's form, of erfcf
    double *part = nullptr;     // energy partials: real [nreal], then recip [nrecip]
    double *lpart = nullptr;    // LJ energy partials of the fused pass [nreal]
    int64_t nreal = 0, nrecip = 0;
    double *dsum = nullptr;     // E_real, E_recip, KE, -, LJ PE, - (md_spme_step fills 2-5)
    double *hsum = nullptr;     // pinned mirror of dsum
    double *kpart = nullptr;    // kinetic-energy partials of the half-kick
    double *fstage = nullptr;   // n x 3 device output when the caller's f is host memory
    double e_const = 0.0;       // E_self + E_bg
    int64_t last_real_blocks = 0;  // real-space CTAs (energy partials) of the last pass
    // the state md_spme_step left the context's force array for (LJ + Coulomb
    // forces of that state): its step, launch count, buffer parities and pair
    // tables; any call that changes the state or the forces changes one of them
    int64_t f_step = -1, f_kernels = -1;
    int f_pc = -1, f_oc = -1;
    Pair f_pair{};
    Fft3 fft;                   // the hand-written 3-D FFT passes (md_fft.cu)
    bool prof = false;
    cudaEvent_t ev[kEvents] = {};
    cudaStream_t side = nullptr;        // real-space pass beside the reciprocal chain
    cudaEvent_t fork = nullptr, join = nullptr;
    double ms[6] = {0, 0, 0, 0, 0, 0};
    std::string err;
};

namespace {

md_status sfail(md_spme *s, md_status st, const std::string &msg) {
    if (s) s->err = msg;
    else g_spme_error = msg;
    return st;
}

md_status scuda(md_spme *s, cudaError_t e, const char *where) {
    return sfail(s, e == cudaErrorMemoryAllocation ? MD_ERR_NOMEM : MD_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define SCK(call)                                               \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return scuda(s, e_, #call);      \
    } while (0)

// ---- B-splines --------------------------------------------------------------

// w[j] = M_P(t + j), dw[j] = M_P'(t + j), j = 0..P-1, t in [0, 1): the
// recursion M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) / (n - 1) from
// M_1 = 1 on [0, 1), and M_n' (x) = M_{n-1}(x) - M_{n-1}(x - 1) (SPME paper,
// Sec. 4), on the P values that are nonzero.
template <typename R, int P, bool DERIV>
__device__ __forceinline__ void bspline(R t, R (&w)[P], R (&dw)[P]) {
    R a[P];
#pragma unroll
    for (int j = 0; j < P; ++j) a[j] = j == 0 ? R(1) : R(0);
#pragma unroll
    for (int n = 2; n <= P; ++n) {
        if (DERIV && n == P) {
#pragma unroll
            for (int j = 0; j < P; ++j) dw[j] = a[j] - (j ? a[j - 1] : R(0));
        }
        const R inv = R(1) / R(n - 1);
#pragma unroll
        for (int j = n - 1; j >= 0; --j)
            a[j] = ((t + R(j)) * a[j] + (R(n - j) - t) * (j ? a[j - 1] : R(0))) * inv;
    }
#pragma unroll
    for (int j = 0; j < P; ++j) w[j] = a[j];
}

// The P grid indices floor(u) - j (mod K) that atom coordinate x touches, and
// t = frac(u), for u = K x / L folded into [0, K).
template <int P>
__device__ __forceinline__ double grid_stencil(double x, double kl, double Kd, int K, int (&ix)[P]) {
    double u = x * kl;
    u = u - Kd * floor(u / Kd);
    const double fl = floor(u);
    int k0 = (int)fl;
    if (k0 >= K) k0 -= K;  // u rounded up to K
#pragma unroll
    for (int j = 0; j < P; ++j) {
        int k = k0 - j;
        ix[j] = k < 0 ? k + K : k;
    }
    return u - fl;
}

// ---- kernels ------------------------------------------------------------------

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic CTA sum of one double per thread into out (thread 0 writes).
template <int NT>
__device__ __forceinline__ void cta_sum_to(double v, double *out) {
    __shared__ double red[NT / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) *out = t;
    }
}


struct AtomArgs {
    const Box *box;
    const double *ctab;
    const double *r;          // cell-relative FP64 positions, SoA 3 x ns
    const int32_t *cellc;     // packed cell of each slot
    const int32_t *id;        // original id of each slot
    int64_t ns;
    Geom g;
};

// Adds v[0..P-1] to the P consecutive floats at p with vector atomics: H
// leading elements bring p to a 16-byte boundary (H = 0..3, from p's
// alignment), then float4 adds, then a float2 and/or a float for the rest.
template <int P, int H>
__device__ __forceinline__ void red_run_h(float *p, const float (&v)[P]) {
    static_assert(H >= 0 && H <= 3, "head");
    if (H == 1) atomicAdd(p, v[0]);
    if (H == 2) atomicAdd(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
    if (H == 3) {
        atomicAdd(p, v[0]);
        atomicAdd(reinterpret_cast<float2 *>(p + 1), make_float2(v[1], v[2]));
    }
    constexpr int h = H < P ? H : P;
    constexpr int rest = P - h;
#pragma unroll
    for (int k = 0; k < rest / 4; ++k)
        atomicAdd(reinterpret_cast<float4 *>(p + h + 4 * k),
                  make_float4(v[h + 4 * k], v[h + 4 * k + 1], v[h + 4 * k + 2], v[h + 4 * k + 3]));
    constexpr int t = h + 4 * (rest / 4);
    if ((rest % 4) >= 2) atomicAdd(reinterpret_cast<float2 *>(p + t), make_float2(v[t], v[t + 1]));
    if ((rest % 4) & 1) atomicAdd(p + P - 1, v[P - 1]);
}

template <int P>
__device__ __forceinline__ void red_run(float *p, const float (&v)[P]) {
    switch ((reinterpret_cast<uintptr_t>(p) >> 2) & 3) {
        case 0: red_run_h<P, 0>(p, v); break;
        case 1: red_run_h<P, 3>(p, v); break;
        case 2: red_run_h<P, 2>(p, v); break;
        default: red_run_h<P, 1>(p, v); break;
    }
}

// Charge of each slot's atom (gathered by its original id); for the mixed
// real-space pass also the slot's FP32 shadow with the charge in w, so that a
// neighbor costs one 16-byte gather.
__global__ void __launch_bounds__(kThreads) k_spme_charges(const Box *__restrict__ box, int64_t ns,
                                                           const int32_t *__restrict__ id,
                                                           const double *__restrict__ q_orig,
                                                           const float4 *__restrict__ sh,
                                                           double *__restrict__ qs,
                                                           float4 *__restrict__ shq) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns || i >= box[0].n) return;
    const double q = q_orig[id[i]];
    qs[i] = q;
    if (shq) {
        const float4 p = sh[i];
        shq[i] = make_float4(p.x, p.y, p.z, (float)q);
    }
}

template <int P, typename R>
__global__ void __launch_bounds__(kThreads) k_spme_spread(AtomArgs a, const double *__restrict__ qs,
                                                          R *__restrict__ grid) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.ns) return;
    const Box &B = a.box[0];
    if (i >= B.n) return;
    const double q = qs[i];
    if (q == 0.0) return;
    int cc[3];
    unpack_cell(a.cellc[i], cc[0], cc[1], cc[2]);
    int ix[3][P];
    R w[3][P], unused[P];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double x = __dadd_rn(cell_centre(a.ctab, B, d, cc[d]), a.r[d * a.ns + i]);
        const double t = grid_stencil<P>(x, a.g.kl[d], a.g.Kd[d], a.g.K[d], ix[d]);
        bspline<R, P, false>((R)t, w[d], unused);
    }
    const int64_t Kx = a.g.K[0], Ky = a.g.K[1];
    const R qr = (R)q;
    // FP32 grid: the P x-points of a stencil row are consecutive (k0 - P + 1
    // .. k0) unless the row wraps at the box edge; add them with vector atomics
    constexpr bool kVec = sizeof(R) == 4;
    const bool contiguous = kVec && ix[0][P - 1] + (P - 1) == ix[0][0];
#pragma unroll
    for (int c = 0; c < P; ++c) {
        const R qz = qr * w[2][c];
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const R qzy = qz * w[1][b];
            R *row = grid + ((int64_t)ix[2][c] * Ky + ix[1][b]) * Kx;
            if constexpr (kVec) {
                if (contiguous) {
                    float v[P];
#pragma unroll
                    for (int e = 0; e < P; ++e) v[e] = qzy * w[0][P - 1 - e];
                    red_run<P>(reinterpret_cast<float *>(row + ix[0][P - 1]), v);
                    continue;
                }
            }
#pragma unroll
            for (int e = 0; e < P; ++e) atomicAdd(row + ix[0][e], qzy * w[0][e]);
        }
    }
}

// Forces on the atoms: F = -q (K/L) sum over the P^3 stencil of the spline
// gradient times dE/dQ, plus the slot's real-space force; written to `out` in
// original order (n x 3), or with ACC added to the context's slot-order force
// array (SoA, 3 x ns).
template <int P, typename R, bool ACC>
__global__ void __launch_bounds__(kThreads) k_spme_gather(AtomArgs a, const double *__restrict__ qs,
                                                          const R *__restrict__ dEdQ,
                                                          const double *__restrict__ fs,
                                                          double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.ns) return;
    const Box &B = a.box[0];
    if (i >= B.n) return;
    const double q = qs[i];
    double fr[3] = {0.0, 0.0, 0.0};
    if (q != 0.0) {
        int cc[3];
        unpack_cell(a.cellc[i], cc[0], cc[1], cc[2]);
        int ix[3][P];
        R w[3][P], dw[3][P];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = __dadd_rn(cell_centre(a.ctab, B, d, cc[d]), a.r[d * a.ns + i]);
            const double t = grid_stencil<P>(x, a.g.kl[d], a.g.Kd[d], a.g.K[d], ix[d]);
            bspline<R, P, true>((R)t, w[d], dw[d]);
        }
        const int64_t Kx = a.g.K[0], Ky = a.g.K[1];
        R gx = 0, gy = 0, gz = 0;
#pragma unroll
        for (int c = 0; c < P; ++c) {
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const R *row = dEdQ + ((int64_t)ix[2][c] * Ky + ix[1][b]) * Kx;
                R sd = 0, sw = 0;
#pragma unroll
                for (int e = 0; e < P; ++e) {
                    const R ph = __ldg(row + ix[0][e]);
                    sd = fma(dw[0][e], ph, sd);
                    sw = fma(w[0][e], ph, sw);
                }
                gx = fma(w[2][c] * w[1][b], sd, gx);
                gy = fma(w[2][c] * dw[1][b], sw, gy);
                gz = fma(dw[2][c] * w[1][b], sw, gz);
            }
        }
        fr[0] = -q * a.g.kl[0] * (double)gx;
        fr[1] = -q * a.g.kl[1] * (double)gy;
        fr[2] = -q * a.g.kl[2] * (double)gz;
    }
    if (ACC) {
        // fs null: the real-space forces are in out already (fused LJ pass)
#pragma unroll
        for (int d = 0; d < 3; ++d) out[d * a.ns + i] += (fs ? fs[d * a.ns + i] : 0.0) + fr[d];
    } else {
        const int64_t g = a.id[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) out[3 * g + d] = fs[d * a.ns + i] + fr[d];
    }
}

// Closing half-kick of velocity Verlet, v += dt/2 F/m (kick = 1), and, with
// ke = 1, the kinetic energy of the resulting velocities summed per CTA (fixed
// order).  kick and ke are uniform over the grid.
__global__ void __launch_bounds__(kThreads) k_spme_half_kick(const Box *__restrict__ box,
                                                             const Pair *__restrict__ pair,
                                                             int64_t ns, int kick, int ke,
                                                             const int32_t *__restrict__ type,
                                                             const double *__restrict__ f,
                                                             double *__restrict__ v,
                                                             double *__restrict__ part) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < box[0].n) {
        const int ty = type[i];
        const double hdtm = pair->hdtm[ty], m = pair->mass[ty];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double vv = v[d * ns + i];
            if (kick) {
                vv = fma(hdtm, f[d * ns + i], vv);
                v[d * ns + i] = vv;
            }
            if (ke) e += 0.5 * m * vv * vv;
        }
    }
    if (ke) cta_sum_to<kThreads>(e, part + blockIdx.x);
}

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

// theta(m) = B(m) exp(-pi^2 |m|^2 / alpha^2) / (pi V |m|^2), theta(0) = 0, on
// the half spectrum; bmod holds |b_x|^2 (K_x), |b_y|^2 (K_y), |b_z|^2 (K_z).
template <typename R>
__global__ void k_spme_theta(R *__restrict__ theta, const double *__restrict__ bmod, Geom g,
                             double Lx, double Ly, double Lz, double alpha, int64_t nhalf) {
    const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= nhalf) return;
    const int mx = (int)(h % g.Kh);
    const int64_t rest = h / g.Kh;
    const int my = (int)(rest % g.K[1]);
    const int mz = (int)(rest / g.K[1]);
    const int sy = 2 * my <= g.K[1] ? my : my - g.K[1];
    const int sz = 2 * mz <= g.K[2] ? mz : mz - g.K[2];
    const double ux = mx / Lx, uy = sy / Ly, uz = sz / Lz;
    const double msq = ux * ux + uy * uy + uz * uz;
    if (h == 0) {
        theta[h] = R(0);
        return;
    }
    const double pi = 3.141592653589793;
    const double B = bmod[mx] * bmod[g.K[0] + my] * bmod[g.K[0] + g.K[1] + mz];
    theta[h] = (R)(B * exp(-pi * pi * msq / (alpha * alpha)) / (pi * (Lx * Ly * Lz) * msq));
}

struct RealArgs {
    const Box *box;
    const double *r;        // FP64 cell-relative positions (SoA)
    const float4 *shq;      // FP32 shadow with w = charge (mixed)
    const float4 *sh;       // the context's FP32 shadow (the FP64 pass's prefilter)
    const double *qs;
    const int32_t *nn;
    const uint32_t *nbr;
    double *fs;
    double *part;
    int64_t ns, nwt;
    int R, pad;
    double alpha, rc2, c2a;  // c2a = 2 alpha / sqrt(pi)
    float alphaf, rc2f, c2af;
    float ec[kErfcDeg + 1], esa, esb;  // erfc(x) = exp(-x^2) t H(sa t + sb) when efit
    int efit;
    const double *tab64;     // erfc(alpha r), exp(-alpha^2 r^2) pieces (FP64 pass)
    double pinv;             // kPieces / rc
    // fused LJ + Coulomb pass (md_spme_step): the context's pair tables and
    // types; fs is then the context's force array and lpart the LJ energy's
    // per-CTA partials
    const Pair *pair;
    const int32_t *type;
    double *lpart;
    Flags *fl;               // the context's flags (index checks of a checked build)
};

// 1/x from the approximate reciprocal and one Newton-Raphson step
// (r' = r + r (1 - x r)): within about an ulp, where the LJ powers of the fused
// pass need more than the approximation alone gives.
__device__ __forceinline__ float rcp_newton(float x) {
    const float r = __fdividef(1.0f, x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// erfc(x) for the mixed real-space pass, ex = exp(-x^2) from the caller: the
// host-fitted form when it met its accuracy check, else the library erfcf.
__device__ __forceinline__ float erfc_mixed(const RealArgs &a, float x, float ex) {
    if (!a.efit) return erfcf(x);
    const float t = __fdividef(1.0f, fmaf((float)kErfcP, x, 1.0f));
    const float sv = fmaf(a.esa, t, a.esb);
    float h = a.ec[kErfcDeg];
#pragma unroll
    for (int k = kErfcDeg - 1; k >= 0; --k) h = fmaf(h, sv, a.ec[k]);
    return ex * (t * h);
}

// The mixed pass's erfc(alpha r) as the real-space kernel evaluates it (the
// same FP32 operations and intrinsics, from r^2 in FP32), by the fitted form
// and by erfcf, against FP64 erfc of the same r: the largest relative errors
// over npts separations in (0, rc], into out[0] (fitted) and out[1] (erfcf)
// as the bit patterns of non-negative doubles (which order as integers).
__global__ void k_erfc_check(RealArgs a, double alpha, float rc, int npts,
                             unsigned long long *out) {
    double w_fit = 0.0, w_lib = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x + 1; q <= npts;
         q += gridDim.x * blockDim.x) {
        const float r = rc * (float)q / (float)npts;
        const float r2 = r * r;
        const float rinv = rsqrtf(r2);
        const float ex = __expf(-(a.alphaf * a.alphaf) * r2);
        const float x = a.alphaf * (r2 * rinv);
        const double ref = erfc(alpha * sqrt((double)r2));
        RealArgs f = a;
        f.efit = 1;
        w_fit = fmax(w_fit, fabs((double)erfc_mixed(f, x, ex) - ref) / ref);
        w_lib = fmax(w_lib, fabs((double)erfcf(x) - ref) / ref);
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(w_fit));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(w_lib));
}

// erfc(alpha r) and exp(-alpha^2 r^2) from the piecewise tables (Horner in
// the interval's local coordinate t = r kPieces / rc - k), D the degree.
template <typename V, int D>
__device__ __forceinline__ void pair_functions(const V *__restrict__ tab, V rr, V pinv, V &er,
                                               V &ex) {
    const V u = rr * pinv;
    const int k = min((int)u, kPieces - 1);
    const V t = u - (V)k;
    const V *c0 = tab + k * (D + 1);
    const V *c1 = tab + (kPieces + k) * (D + 1);
    er = c0[D];
    ex = c1[D];
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
        er = fma(er, t, c0[j]);
        ex = fma(ex, t, c1[j]);
    }
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Real-space pairs: U = q_i q_j erfc(alpha r) / r over r^2 < rc^2, full list.
// With LJ, the same walk of the list also takes the LJ 12-6 pair terms of the
// context (its cutoff, which is at least rc, its eps/sigma tables and shift)
// and writes F_LJ + F_real: the force pass of a Coulomb + LJ step.
//
// Half lists (HALF): each pair is listed once; fs starts at zero, the atom's
// own sums and each pair's reaction (FP64 atomics) are added into it, and the
// energy partials count each pair once (doubled below to the full-list
// convention of two halves per pair).
template <int T, bool MIXED, bool LJ, bool HALF>
__global__ void __launch_bounds__(kRealBlock) k_spme_real(RealArgs a) {
    constexpr int A = 32 / T;
    __shared__ double s_offd[81];
    __shared__ float s_offf[81];
    __shared__ double s_tab64[MIXED ? 1 : kTab64];
    // LJ tables per type pair: c1 = 24 eps / sigma^2 (FP32) or 24 eps (FP64),
    // sigma^2, 4 eps, U(rc)
    __shared__ double s_lj64[LJ && !MIXED ? 4 * 64 : 1];
    __shared__ float s_lj32[LJ && MIXED ? 4 * 64 : 1];
    const Box &B = a.box[0];
    if (!MIXED)
        for (int k = threadIdx.x; k < kTab64; k += blockDim.x) s_tab64[k] = a.tab64[k];
    if (LJ && threadIdx.x < 64) {
        const int k = threadIdx.x;
        if (MIXED) {
            s_lj32[k] = a.pair->fc1[k];
            s_lj32[64 + k] = a.pair->fs2[k];
            s_lj32[128 + k] = a.pair->fe4[k];
            s_lj32[192 + k] = a.pair->fush[k];
        } else {
            s_lj64[k] = a.pair->e24[k];
            s_lj64[64 + k] = a.pair->s2[k];
            s_lj64[128 + k] = a.pair->e4[k];
            s_lj64[192 + k] = a.pair->ush[k];
        }
    }
    const int nt = LJ ? a.pair->nt : 1;
    const double rc2lj = LJ ? a.pair->rc2 : 0.0;
    const float rc2ljf = LJ ? a.pair->rc2f : 0.f;
    if (threadIdx.x < 81) {
        const int code = threadIdx.x / 3, d = threadIdx.x % 3;
        const int o = (d == 0 ? code % 3 : (d == 1 ? (code / 3) % 3 : code / 9)) - 1;
        s_offd[threadIdx.x] = (double)o * B.h[d];
        s_offf[threadIdx.x] = o ? (float)o * B.hf[d] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane % T;
    double pe_lane = 0.0, pl_lane = 0.0;
    for (int64_t wt = (int64_t)blockIdx.x * (kRealBlock / 32) + (threadIdx.x >> 5); wt < a.nwt;
         wt += (int64_t)gridDim.x * (kRealBlock / 32)) {
        const int64_t i = wt * A + lane / T;
        const bool valid = i < B.n;
        const int ni = valid ? min(a.nn[i], a.pad) : 0;
        const uint32_t *row = a.nbr + (size_t)wt * a.R * 32 + lane;
        const int nq = (ni - sub + T - 1) / T;
        double F[3];
        if (MIXED) {
            const float4 si = a.shq[i];
            const float qi = si.w;
            const int ti = LJ && nt > 1 ? a.type[i] : 0;
            float fx = 0.f, fy = 0.f, fz = 0.f, pe = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;
            float pl = 0.f, cl = 0.f;
            // kRealBatch entries per lane at a time: their list words, then
            // their shadows and charges, are all in flight before the math.
            // Whole batches: a lane's entries past its count are replaced by
            // the sentinel, whose slot ns is far from every atom, uncharged.
            const int nqr = (nq + kRealBatch - 1) & ~(kRealBatch - 1);
            const uint32_t sent = sentinel_entry(a.ns);
            for (int k0 = 0; k0 < nqr; k0 += kRealBatch) {
                uint32_t e[kRealBatch];
#pragma unroll
                for (int u = 0; u < kRealBatch; ++u)
                    e[u] = k0 + u < nq ? __ldg(row + (size_t)(k0 + u) * 32) : sent;
                float4 sj[kRealBatch];
                float qj[kRealBatch];
                int tj[kRealBatch];
                int64_t jj[kRealBatch];  // checked slot indices (half lists: the reactions' targets)
#pragma unroll
                for (int u = 0; u < kRealBatch; ++u) {
                    const int64_t j =
                        chk_index(e[u] & MD_IDX_MASK, a.ns + 1, CHK_SPME_GATHER, a.fl, a.ns);
                    jj[u] = j;
                    sj[u] = __ldg(a.shq + j);
                    qj[u] = sj[u].w;
                    tj[u] = LJ && nt > 1 ? __ldg(a.type + j) : 0;
                }
                // the batch's terms are summed plainly, then added to the
                // per-atom sums with one compensated add per component
                float bx = 0.f, by = 0.f, bz = 0.f, be = 0.f, bl = 0.f;
#pragma unroll
                for (int u = 0; u < kRealBatch; ++u) {
                    const int cd = 3 * (int)(e[u] >> MD_IDX_BITS);
                    const float dx = (sj[u].x + s_offf[cd]) - si.x;
                    const float dy = (sj[u].y + s_offf[cd + 1]) - si.y;
                    const float dz = (sj[u].z + s_offf[cd + 2]) - si.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    if (LJ) {
                        // the LJ cutoff is at least rc: its test covers both
                        if (r2 < rc2ljf) {
                            const float rinv = rsqrtf(r2);
                            const float r2inv = rcp_newton(r2);  // s^6, s^12 amplify its error
                            const int ab = ti * nt + tj[u];
                            const float q2 = s_lj32[64 + ab] * r2inv;
                            const float s6 = q2 * q2 * q2;
                            float g = s_lj32[ab] * q2 * s6 * fmaf(2.f, s6, -1.f);
                            bl += 0.5f * fmaf(s_lj32[128 + ab] * s6, s6 - 1.f, -s_lj32[192 + ab]);
                            if (qj[u] != 0.f && r2 < a.rc2f) {
                                const float qq = qi * qj[u];
                                const float ex = __expf(-(a.alphaf * a.alphaf) * r2);
                                const float er = erfc_mixed(a, a.alphaf * (r2 * rinv), ex);
                                g = fmaf(qq * fmaf(er, rinv, a.c2af * ex), r2inv, g);
                                be = fmaf(0.5f * qq, er * rinv, be);
                            }
                            bx = fmaf(-g, dx, bx);
                            by = fmaf(-g, dy, by);
                            bz = fmaf(-g, dz, bz);
                            if (HALF && jj[u] < a.ns) {  // (slot ns: the far dummy)
                                const int64_t j = jj[u];
                                atomicAdd(a.fs + j, (double)(g * dx));
                                atomicAdd(a.fs + a.ns + j, (double)(g * dy));
                                atomicAdd(a.fs + 2 * a.ns + j, (double)(g * dz));
                            }
                        }
                    } else if (qj[u] != 0.f && r2 < a.rc2f) {
                        const float qq = qi * qj[u];
                        const float rinv = rsqrtf(r2);
                        const float ex = __expf(-(a.alphaf * a.alphaf) * r2);
                        const float er = erfc_mixed(a, a.alphaf * (r2 * rinv), ex);
                        const float g = qq * fmaf(er, rinv, a.c2af * ex) * (rinv * rinv);
                        bx = fmaf(-g, dx, bx);
                        by = fmaf(-g, dy, by);
                        bz = fmaf(-g, dz, bz);
                        be = fmaf(0.5f * qq, er * rinv, be);
                        if (HALF && jj[u] < a.ns) {  // (slot ns: the far dummy)
                            const int64_t j = jj[u];
                            atomicAdd(a.fs + j, (double)(g * dx));
                            atomicAdd(a.fs + a.ns + j, (double)(g * dy));
                            atomicAdd(a.fs + 2 * a.ns + j, (double)(g * dz));
                        }
                    }
                }
                kahan_add(fx, cx, bx);
                kahan_add(fy, cy, by);
                kahan_add(fz, cz, bz);
                kahan_add(pe, cp, be);
                if (LJ) kahan_add(pl, cl, bl);
            }
            F[0] = (double)(fx - cx);
            F[1] = (double)(fy - cy);
            F[2] = (double)(fz - cz);
            pe_lane += (double)(pe - cp);
            pl_lane += (double)(pl - cl);
        } else {
            const double rix = a.r[i], riy = a.r[a.ns + i], riz = a.r[2 * a.ns + i];
            const double qi = a.qs[i];
            const int ti = LJ && nt > 1 ? a.type[i] : 0;
            double fx = 0.0, fy = 0.0, fz = 0.0, pe = 0.0, pl = 0.0;
            // The FP64 pipe is charged per warp instruction: an FP32 pass on
            // the shadows first marks the entries that can lie within the
            // larger cutoff (r^2 below it by a 1e-4 margin; the shadows' error
            // in r^2 is below 1e-6 of it), and the FP64 pass takes those only,
            // in row order (the same sums).
            const float4 si = a.sh[i];
            const float cut2 = (float)(LJ ? rc2lj : a.rc2) * 1.0001f;
            for (int c0 = 0; c0 < nq; c0 += 32) {
              const int cn = min(32, nq - c0);
              uint32_t near = 0u;
              for (int k = 0; k < cn; ++k) {
                const uint32_t e = __ldg(row + (size_t)(c0 + k) * 32);
                const float4 sj = __ldg(
                    a.sh + chk_index(e & MD_IDX_MASK, a.ns + 1, CHK_SPME_GATHER, a.fl, a.ns));
                const int cd = 3 * (int)(e >> MD_IDX_BITS);
                const float dx = (sj.x + s_offf[cd]) - si.x;
                const float dy = (sj.y + s_offf[cd + 1]) - si.y;
                const float dz = (sj.z + s_offf[cd + 2]) - si.z;
                if (dx * dx + dy * dy + dz * dz < cut2) near |= 1u << k;
              }
              while (near) {
                const int k = c0 + __ffs(near) - 1;
                near &= near - 1u;
                const uint32_t e = __ldg(row + (size_t)k * 32);
                const int64_t j = chk_index(e & MD_IDX_MASK, a.ns, CHK_SPME_GATHER, a.fl, 0);
                const int cd = 3 * (int)(e >> MD_IDX_BITS);
                const double dx = (__ldg(a.r + j) + s_offd[cd]) - rix;
                const double dy = (__ldg(a.r + a.ns + j) + s_offd[cd + 1]) - riy;
                const double dz = (__ldg(a.r + 2 * a.ns + j) + s_offd[cd + 2]) - riz;
                const double r2 = (dx * dx + dy * dy) + dz * dz;
                double g = 0.0;
                if (LJ && r2 < rc2lj) {
                    const double r2inv = rcp_newton64(r2);
                    const int ab = ti * nt + (nt > 1 ? __ldg(a.type + j) : 0);
                    const double q2 = s_lj64[64 + ab] * r2inv;
                    const double s6 = q2 * q2 * q2;
                    g = s_lj64[ab] * r2inv * s6 * (2.0 * s6 - 1.0);
                    pl += 0.5 * (s_lj64[128 + ab] * s6 * (s6 - 1.0) - s_lj64[192 + ab]);
                }
                if (r2 < a.rc2) {
                    const double qq = qi * __ldg(a.qs + j);
                    const double rinv = rsqrt(r2);
                    double er, ex;
                    pair_functions<double, kDeg64>(s_tab64, r2 * rinv, a.pinv, er, ex);
                    g += qq * (er * rinv + a.c2a * ex) * (rinv * rinv);
                    pe += 0.5 * qq * er * rinv;
                }
                fx -= g * dx;
                fy -= g * dy;
                fz -= g * dz;
                if (HALF && g != 0.0) {
                    atomicAdd(a.fs + j, g * dx);
                    atomicAdd(a.fs + a.ns + j, g * dy);
                    atomicAdd(a.fs + 2 * a.ns + j, g * dz);
                }
              }
            }
            F[0] = fx;
            F[1] = fy;
            F[2] = fz;
            pe_lane += pe;
            pl_lane += pl;
        }
#pragma unroll
        for (int o = T / 2; o; o >>= 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) F[d] += __shfl_xor_sync(0xffffffffu, F[d], o);
        }
        if (valid && sub == 0) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (HALF) atomicAdd(a.fs + d * a.ns + i, F[d]);
                else a.fs[d * a.ns + i] = F[d];
            }
        }
    }
    if (HALF) {
        pe_lane *= 2.0;
        pl_lane *= 2.0;
    }
    cta_sum_to<kRealBlock>(pe_lane, a.part + blockIdx.x);
    if (LJ) {
        __syncthreads();
        cta_sum_to<kRealBlock>(pl_lane, a.lpart + blockIdx.x);
    }
}

__global__ void k_spme_sum(const double *__restrict__ part, int64_t nreal, int64_t nrecip,
                           double *__restrict__ out) {
    double er = 0.0, ek = 0.0;
    for (int64_t k = threadIdx.x; k < nreal; k += blockDim.x) er += part[k];
    for (int64_t k = threadIdx.x; k < nrecip; k += blockDim.x) ek += part[nreal + k];
    cta_sum_to<1024>(er, out);
    __syncthreads();
    cta_sum_to<1024>(ek, out + 1);
    if (threadIdx.x == 0) out[1] *= 0.5;
}

// ---- host helpers -------------------------------------------------------------

// |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K)|^2, m = 0..K-1
// (SPME paper, Sec. 4), with M_p at the integers by the spline recursion.
bool spline_moduli(int p, int K, double *out) {
    std::vector<double> a(p + 1, 0.0);  // a[j] = M_n(j), j = 0..n
    a[1] = 1.0;                          // M_2 at 0, 1, 2: 0, 1, 0
    for (int n = 3; n <= p; ++n) {
        std::vector<double> b(p + 1, 0.0);
        for (int j = 1; j < n; ++j) b[j] = (j * a[j] + (n - j) * a[j - 1]) / (n - 1);
        a.swap(b);
    }
    const double pi = 3.141592653589793;
    for (int m = 0; m < K; ++m) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k <= p - 2; ++k) {
            const double ang = 2.0 * pi * (double)m * (double)k / (double)K;
            re += a[k + 1] * std::cos(ang);
            im += a[k + 1] * std::sin(ang);
        }
        const double d = re * re + im * im;
        if (!(d > 1e-30)) return false;
        out[m] = 1.0 / d;
    }
    return true;
}

// Degree n - 1 interpolant of g on [0, 1] at the Chebyshev nodes, as
// monomial coefficients in t (out[0..n-1], Horner order out[n-1] ... out[0]).
template <typename G>
void cheb_fit01(G g, int n, double *out) {
    const double pi = 3.141592653589793;
    std::vector<double> y(n), c(n, 0.0), mono(n, 0.0);
    for (int m = 0; m < n; ++m) {
        const double x = std::cos(pi * (m + 0.5) / n);        // node in [-1, 1]
        y[m] = g(0.5 * (x + 1.0));
    }
    for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) acc += y[m] * std::cos(pi * j * (m + 0.5) / n);
        c[j] = (j == 0 ? 1.0 : 2.0) * acc / n;
    }
    // T_j(2t - 1) as polynomials in t: T_0 = 1, T_1 = 2t - 1,
    // T_{j+1} = (4t - 2) T_j - T_{j-1}
    std::vector<double> tm(n, 0.0), t0(n, 0.0), t1(n, 0.0);
    t0[0] = 1.0;
    if (n > 1) {
        t1[0] = -1.0;
        t1[1] = 2.0;
    }
    for (int i = 0; i < n; ++i) mono[i] += c[0] * t0[i];
    for (int j = 1; j < n; ++j) {
        for (int i = 0; i < n; ++i) mono[i] += c[j] * t1[i];
        std::fill(tm.begin(), tm.end(), 0.0);
        for (int i = 0; i < n; ++i) {
            tm[i] += -2.0 * t1[i] - t0[i];
            if (i + 1 < n) tm[i + 1] += 4.0 * t1[i];
        }
        t0.swap(t1);
        t1.swap(tm);
    }
    for (int i = 0; i < n; ++i) out[i] = mono[i];
}

// Piecewise polynomial of f on [0, rc]: on each of kPieces equal intervals,
// Chebyshev interpolation at the deg + 1 first-kind nodes, re-expressed in the
// monomial basis of the local coordinate t in [0, 1) (out[piece * (deg + 1) +
// j]).  Returns the largest absolute deviation from f on a check grid of 64
// points per interval.
template <typename F>
double fit_pieces(F f, double rc, int deg, double *out) {
    const double w = rc / kPieces;
    const int n = deg + 1;
    double worst = 0.0;
    for (int k = 0; k < kPieces; ++k) {
        double *mono = out + k * n;
        cheb_fit01([&](double t) { return f((k + t) * w); }, n, mono);
        for (int q = 0; q <= 64; ++q) {
            const double t = q / 64.0;
            double v = mono[n - 1];
            for (int i = n - 2; i >= 0; --i) v = v * t + mono[i];
            worst = std::max(worst, std::fabs(v - f((k + t) * w)));
        }
    }
    return worst;
}

// Mixed real-space pass: H(s) of erfc(x) = exp(-x^2) t H(s) on [0, alpha rc]
// (kErfcDeg), then the check of its FP32 evaluation against erfc.
void fit_erfc_mixed(md_spme *s, double alpha, double rc) {
    const double X = alpha * rc * (1.0 + 1e-6);
    const double tmin = 1.0 / (1.0 + kErfcP * X);
    const int n = kErfcDeg + 1;
    std::vector<double> mono(n);
    cheb_fit01(
        [&](double sv) {
            const double t = tmin + (1.0 - tmin) * sv;
            const double x = (1.0 / t - 1.0) / kErfcP;
            return std::erfc(x) * std::exp(x * x) / t;
        },
        n, mono.data());
    for (int k = 0; k < n; ++k) s->erfc_c[k] = (float)mono[k];
    s->erfc_sa = (float)(1.0 / (1.0 - tmin));
    s->erfc_sb = (float)(-tmin / (1.0 - tmin));
    double worst = 0.0;
    for (int q = 0; q <= 4000; ++q) {
        const float xf = (float)(X * q / 4000.0);
        const float t = 1.0f / std::fmaf((float)kErfcP, xf, 1.0f);
        const float sv = std::fmaf(s->erfc_sa, t, s->erfc_sb);
        float h = s->erfc_c[kErfcDeg];
        for (int k = kErfcDeg - 1; k >= 0; --k) h = std::fmaf(h, sv, s->erfc_c[k]);
        const float ex = (float)std::exp(-(double)xf * (double)xf);
        const double ref = std::erfc((double)xf);
        worst = std::max(worst, std::fabs((double)(ex * (t * h)) - ref) / ref);
    }
    s->erfc_fit = worst <= kErfcTol;
}

// The device check of the fit (k_erfc_check): H's form is used when, as the
// kernel evaluates it (__fdividef, __expf, FP32 arguments), it is within
// kErfcTol of erfc or no worse than erfcf on the same inputs.
md_status check_erfc_on_device(md_spme *s) {
    if (!s->erfc_fit) return MD_OK;  // the host check already chose erfcf
    RealArgs ra{};
    ra.alphaf = (float)s->p.alpha;
    for (int k = 0; k <= kErfcDeg; ++k) ra.ec[k] = s->erfc_c[k];
    ra.esa = s->erfc_sa;
    ra.esb = s->erfc_sb;
    ra.efit = 1;
    unsigned long long *d = nullptr;
    SCK(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemset(d, 0, sizeof(h));
    if (e == cudaSuccess) {
        k_erfc_check<<<16, 256, 0, s->stream>>>(ra, s->p.alpha, (float)s->p.rc, 4000, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d);
    SCK(e);
    std::memcpy(&s->erfc_err[0], &h[0], sizeof(double));
    std::memcpy(&s->erfc_err[1], &h[1], sizeof(double));
    s->erfc_fit = s->erfc_err[0] <= std::max(kErfcTol, s->erfc_err[1]);
    return MD_OK;
}

template <int T, bool MIXED, bool LJ, bool HALF = false>
cudaError_t launch_real_t(const RealArgs &ra, int blocks, cudaStream_t st) {
    k_spme_real<T, MIXED, LJ, HALF><<<blocks, kRealBlock, 0, st>>>(ra);
    return cudaGetLastError();
}

// half lists: 4 lanes per atom (checked when the context is created)
template <bool MIXED, bool LJ>
cudaError_t launch_real_l(int T, bool half, const RealArgs &ra, int blocks, cudaStream_t st) {
    if (half) return T == 4 ? launch_real_t<4, MIXED, LJ, true>(ra, blocks, st) : cudaErrorInvalidValue;
    switch (T) {
        case 1: return launch_real_t<1, MIXED, LJ>(ra, blocks, st);
        case 2: return launch_real_t<2, MIXED, LJ>(ra, blocks, st);
        case 4: return launch_real_t<4, MIXED, LJ>(ra, blocks, st);
        case 8: return launch_real_t<8, MIXED, LJ>(ra, blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

// Resident CTAs per SM of a real-space kernel variant (occupancy API, cached).
template <int T, bool MIXED, bool LJ, bool HALF = false>
int real_residency() {
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (v == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_spme_real<T, MIXED, LJ, HALF>,
                                                          kRealBlock, 0) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        cached.store(v);
    }
    return v;
}

template <bool MIXED, bool LJ>
int real_residency_l(int T, bool half) {
    if (half) return real_residency<4, MIXED, LJ, true>();
    switch (T) {
        case 1: return real_residency<1, MIXED, LJ>();
        case 2: return real_residency<2, MIXED, LJ>();
        case 4: return real_residency<4, MIXED, LJ>();
        default: return real_residency<8, MIXED, LJ>();
    }
}

int real_residency_any(bool mixed, bool lj, int T, bool half) {
    if (mixed) return lj ? real_residency_l<true, true>(T, half) : real_residency_l<true, false>(T, half);
    return lj ? real_residency_l<false, true>(T, half) : real_residency_l<false, false>(T, half);
}

cudaError_t launch_real(bool mixed, bool lj, int T, bool half, const RealArgs &ra, int blocks,
                        cudaStream_t st) {
    if (mixed) return lj ? launch_real_l<true, true>(T, half, ra, blocks, st)
                         : launch_real_l<true, false>(T, half, ra, blocks, st);
    return lj ? launch_real_l<false, true>(T, half, ra, blocks, st)
              : launch_real_l<false, false>(T, half, ra, blocks, st);
}

template <int P, typename R>
cudaError_t launch_atoms(int mode, const AtomArgs &aa, const double *qs, void *grid,
                         const double *fs, double *out, cudaStream_t st) {
    const int blocks = (int)((aa.ns + kThreads - 1) / kThreads);
    if (mode == kGatherOut)
        k_spme_gather<P, R, false><<<blocks, kThreads, 0, st>>>(aa, qs, (const R *)grid, fs, out);
    else if (mode == kGatherAcc)
        k_spme_gather<P, R, true><<<blocks, kThreads, 0, st>>>(aa, qs, (const R *)grid, fs, out);
    else
        k_spme_spread<P, R><<<blocks, kThreads, 0, st>>>(aa, qs, (R *)grid);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_atoms_p(int p, int mode, const AtomArgs &aa, const double *qs, void *grid,
                           const double *fs, double *out, cudaStream_t st) {
    switch (p) {
        case 4: return launch_atoms<4, R>(mode, aa, qs, grid, fs, out, st);
        case 6: return launch_atoms<6, R>(mode, aa, qs, grid, fs, out, st);
        case 8: return launch_atoms<8, R>(mode, aa, qs, grid, fs, out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_atoms_any(bool f32, int p, int mode, const AtomArgs &aa, const double *qs,
                             void *grid, const double *fs, double *out, cudaStream_t st) {
    return f32 ? launch_atoms_p<float>(p, mode, aa, qs, grid, fs, out, st)
               : launch_atoms_p<double>(p, mode, aa, qs, grid, fs, out, st);
}

void destroy(md_spme *s) {
    auto F = [](void *p) { if (p) cudaFree(p); };
    F(s->q); F(s->qs); F(s->shq); F(s->grid); F(s->ghat); F(s->theta); F(s->fs); F(s->part); F(s->lpart);
    F(s->dsum); F(s->fstage); F(s->kpart); F(s->tab64);
    if (s->hsum) cudaFreeHost(s->hsum);
    fft3_free(&s->fft);
    for (auto e : s->ev)
        if (e) cudaEventDestroy(e);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->join) cudaEventDestroy(s->join);
    if (s->side) cudaStreamDestroy(s->side);
}

md_status load_charges(md_spme *s, const double *q) {
    md_ctx *c = s->ctx;
    const int64_t n = c->n_total;
    std::vector<double> hq(n);
    if (is_device_pointer(q))
        SCK(cudaMemcpy(hq.data(), q, n * sizeof(double), cudaMemcpyDeviceToHost));
    else
        std::copy(q, q + n, hq.begin());
    double sq = 0.0, sum = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        if (!std::isfinite(hq[k])) return sfail(s, MD_ERR_NONFINITE, "non-finite charge");
        sq += hq[k] * hq[k];
        sum += hq[k];
    }
    const Box &B = c->hbox[0];
    const double V = B.L[0] * B.L[1] * B.L[2];
    const double pi = 3.141592653589793;
    const double al = s->p.alpha;
    s->e_const = -al / std::sqrt(pi) * sq - pi * sum * sum / (2.0 * V * al * al);
    SCK(cudaMemcpyAsync(s->q, hq.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    return MD_OK;
}

template <typename T>
cudaError_t salloc(T **p, size_t count) {
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T));
}

md_status init(md_spme *s, md_ctx *c, const double *q, const md_spme_params *p) {
    s->ctx = c;
    s->stream = c->stream;
    s->p = *p;
    const Box &B = c->hbox[0];
    Geom &g = s->g;
    for (int d = 0; d < 3; ++d) {
        g.K[d] = p->K[d];
        g.Kd[d] = (double)p->K[d];
        g.kl[d] = (double)p->K[d] / B.L[d];
    }
    g.Kh = g.K[0] / 2 + 1;
    s->ngrid = (int64_t)g.K[0] * g.K[1] * g.K[2];
    s->nhalf = (int64_t)g.Kh * g.K[1] * g.K[2];
    const int64_t ns = c->ns, n = c->n_total;
    // real-space CTAs: ns / (32 / T) warp tiles, kRealBlock / 32 per CTA; at most
    // (T = MD_MAXT = 8) ns / 4 tiles
    s->nreal = (ns / (32 / MD_MAXT) + kRealBlock / 32 - 1) / (kRealBlock / 32) + 1;
    s->nrecip = 4 * (int64_t)c->nsm;
    SCK(salloc(&s->q, n));
    SCK(salloc(&s->qs, ns));
    if (c->params.precision == MD_MIXED) SCK(salloc(&s->shq, ns + 1));
    SCK(cudaMemset(s->qs, 0, ns * sizeof(double)));   // padding slots stay uncharged
    if (s->shq) {
        // the sentinel slot ns of the list's padding entries: far away, uncharged
        SCK(cudaMemset(s->shq, 0, ns * sizeof(float4)));
        const float4 far = make_float4(1e4f, 1e4f, 1e4f, 0.f);
        SCK(cudaMemcpy(s->shq + ns, &far, sizeof(float4), cudaMemcpyHostToDevice));
    }
    s->f32 = c->params.precision == MD_MIXED;
    const size_t rb = s->f32 ? sizeof(float) : sizeof(double);
    SCK(cudaMalloc(&s->grid, s->ngrid * rb));
    SCK(cudaMalloc(&s->ghat, s->nhalf * 2 * rb));
    SCK(cudaMalloc(&s->theta, s->nhalf * rb));
    SCK(salloc(&s->fs, 3 * ns));
    SCK(salloc(&s->part, s->nreal + s->nrecip));
    SCK(salloc(&s->lpart, s->nreal));
    SCK(salloc(&s->dsum, 6));
    SCK(cudaMallocHost(reinterpret_cast<void **>(&s->hsum), 6 * sizeof(double)));
    for (auto &e : s->ev) SCK(cudaEventCreate(&e));
    SCK(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
    SCK(cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming));
    SCK(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
    // influence table, built once
    std::vector<double> bm(g.K[0] + g.K[1] + g.K[2]);
    if (!spline_moduli(p->order, g.K[0], bm.data()) ||
        !spline_moduli(p->order, g.K[1], bm.data() + g.K[0]) ||
        !spline_moduli(p->order, g.K[2], bm.data() + g.K[0] + g.K[1]))
        return sfail(s, MD_ERR_ARG, "Euler spline modulus vanishes for this order and grid");
    double *dbm = nullptr;
    SCK(salloc(&dbm, bm.size()));
    cudaError_t e = cudaMemcpyAsync(dbm, bm.data(), bm.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        const int tb = (int)((s->nhalf + 255) / 256);
        if (s->f32)
            k_spme_theta<float><<<tb, 256, 0, c->stream>>>((float *)s->theta, dbm, g, B.L[0], B.L[1],
                                                           B.L[2], p->alpha, s->nhalf);
        else
            k_spme_theta<double><<<tb, 256, 0, c->stream>>>((double *)s->theta, dbm, g, B.L[0],
                                                            B.L[1], B.L[2], p->alpha, s->nhalf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dbm);
    if (e != cudaSuccess) return scuda(s, e, "influence table");
    // real-space pair functions (host libm values, Chebyshev interpolation)
    {
        const double al = p->alpha, rc = p->rc;
        auto f_erfc = [al](double r) { return std::erfc(al * r); };
        auto f_gauss = [al](double r) { return std::exp(-al * al * r * r); };
        std::vector<double> h64(kTab64);
        const double e64 = std::max(fit_pieces(f_erfc, rc, kDeg64, h64.data()),
                                    fit_pieces(f_gauss, rc, kDeg64, h64.data() + kTab64 / 2));
        if (!(e64 <= 1e-14))
            return sfail(s, MD_ERR_ARG, "real-space pair-function fit not accurate for this alpha, rc");
        SCK(salloc(&s->tab64, kTab64));
        SCK(cudaMemcpy(s->tab64, h64.data(), kTab64 * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (s->f32) {
        fit_erfc_mixed(s, p->alpha, p->rc);
        const md_status se = check_erfc_on_device(s);
        if (se != MD_OK) return se;
    }
    SCK(fft3_plan(&s->fft, g.K, s->f32));
    return load_charges(s, q);
}

}  // namespace

extern "C" {

md_status md_spme_create(md_ctx *c, const double *q, const md_spme_params *p, md_spme **out) {
    MD_TRACE("md_spme_create");
    if (!out) return sfail(nullptr, MD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!c || !q || !p) return sfail(nullptr, MD_ERR_ARG, "NULL argument");
    if (c->nbox != 1) return sfail(nullptr, MD_ERR_ARG, "SPME needs a single-box context");
    if (!(p->alpha > 0.0) || !std::isfinite(p->alpha))
        return sfail(nullptr, MD_ERR_ARG, "alpha must be positive and finite");
    if (!(p->rc > 0.0) || !(p->rc <= c->params.rc))
        return sfail(nullptr, MD_ERR_ARG, "rc must satisfy 0 < rc <= the context's pair cutoff");
    if (p->order != 4 && p->order != 6 && p->order != 8)
        return sfail(nullptr, MD_ERR_ARG, "order must be 4, 6 or 8");
    for (int d = 0; d < 3; ++d) {
        if (p->K[d] < p->order || p->K[d] > kMaxGrid)
            return sfail(nullptr, MD_ERR_ARG, "grid size K out of [order, 4096]");
        int rad[kFftMaxStages], nst = 0;
        if (!fft_factor(p->K[d], true, rad, &nst))
            return sfail(nullptr, MD_ERR_ARG, "grid size K must factor into 2, 3, 5 and 7");
    }
    md_spme *s = new (std::nothrow) md_spme();
    if (!s) return sfail(nullptr, MD_ERR_NOMEM, "host allocation failed");
    md_status st = init(s, c, q, p);
    if (st != MD_OK) {
        g_spme_error = s->err;
        destroy(s);
        delete s;
        cudaGetLastError();   // a failed allocation's error is reported, not left pending
        return st;
    }
    *out = s;
    return MD_OK;
}

md_status md_spme_set_charges(md_spme *s, const double *q) {
    if (!s) return sfail(nullptr, MD_ERR_ARG, "NULL solver");
    if (!q) return sfail(s, MD_ERR_ARG, "q is NULL");
    // the total forces a previous md_spme_step left belong to the old charges
    s->f_step = -1;
    return load_charges(s, q);
}

}  // extern "C"

namespace {

// Enqueues one SPME evaluation at the context's current positions on its
// stream: forces to `out` (original order, n x 3) or, with acc, added to the
// context's slot-order forces; E_real and E_recip to s->dsum.  With lj (a
// Coulomb + LJ step, acc set), the real-space pass is the fused LJ + Coulomb
// pass: it writes F_LJ + F_real to the context's force array and the LJ
// energy's partials to s->lpart, and the gather adds F_recip.  No host sync.
md_status enqueue(md_spme *s, double *out, bool acc, bool lj) {
    md_ctx *c = s->ctx;
    const bool mixed = c->params.precision == MD_MIXED;
    cudaStream_t stream = c->stream;
    auto mark = [&](int k) -> cudaError_t {
        return s->prof ? cudaEventRecord(s->ev[k], stream) : cudaSuccess;
    };
    AtomArgs aa;
    aa.box = c->dbox;
    aa.ctab = c->ctab;
    aa.r = c->r[c->pc];
    aa.cellc = c->cellc[c->oc];
    aa.id = c->id[c->oc];
    aa.ns = c->ns;
    aa.g = s->g;
    const int A = 32 / c->T;
    RealArgs ra;
    ra.box = c->dbox;
    ra.r = c->r[c->pc];
    ra.shq = s->shq;
    ra.sh = c->sh[c->pc];
    ra.qs = s->qs;
    ra.nn = c->nn;
    ra.nbr = c->nbr;
    ra.fs = s->fs;
    ra.part = s->part;
    ra.ns = c->ns;
    ra.nwt = c->ns / A;
    ra.R = c->R;
    ra.pad = c->pad;
    ra.alpha = s->p.alpha;
    ra.rc2 = s->p.rc * s->p.rc;
    ra.c2a = 2.0 * s->p.alpha / std::sqrt(3.141592653589793);
    ra.alphaf = (float)ra.alpha;
    ra.rc2f = (float)ra.rc2;
    ra.c2af = (float)ra.c2a;
    ra.tab64 = s->tab64;
    for (int k = 0; k <= kErfcDeg; ++k) ra.ec[k] = s->erfc_c[k];
    ra.esa = s->erfc_sa;
    ra.esb = s->erfc_sb;
    ra.efit = s->erfc_fit ? 1 : 0;
    ra.pinv = kPieces / s->p.rc;
    ra.pair = c->dpair;
    ra.type = c->type[c->oc];
    ra.lpart = s->lpart;
    ra.fl = c->dflags;
    if (lj) ra.fs = c->f;
    // beside the reciprocal chain the mixed real-space pass takes a persistent
    // grid of kRealCtasPerSm CTAs per SM (grid-stride over warp tiles), leaving
    // room on every SM for the chain's kernels; the FP64 pass (which dominates
    // its call) and a profiled pass take one warp per tile
    const bool overlap = !s->prof;
    const int64_t tiles_blocks = (ra.nwt + kRealBlock / 32 - 1) / (kRealBlock / 32);
    const bool half = c->params.half_list != 0;
    const int per_sm =
        std::min(lj ? kFusedCtasPerSm : kRealCtasPerSm, real_residency_any(mixed, lj, c->T, half));
    const int real_blocks = (int)std::min<int64_t>(
        tiles_blocks, overlap && mixed ? (int64_t)per_sm * c->nsm : tiles_blocks);
    if (real_blocks > s->nreal) return sfail(s, MD_ERR_ARG, "internal: real-space partials");

    SCK(mark(0));
    k_spme_charges<<<(int)((c->ns + kThreads - 1) / kThreads), kThreads, 0, stream>>>(
        c->dbox, c->ns, c->id[c->oc], s->q, c->sh[c->pc], s->qs, s->shq);
    SCK(cudaGetLastError());
    if (overlap) {
        SCK(cudaEventRecord(s->fork, stream));
        SCK(cudaStreamWaitEvent(s->side, s->fork, 0));
        if (half) SCK(cudaMemsetAsync(ra.fs, 0, 3 * (size_t)c->ns * sizeof(double), s->side));
        SCK(launch_real(mixed, lj, c->T, half, ra, real_blocks, s->side));
        SCK(cudaEventRecord(s->join, s->side));
    }
    const size_t rb = s->f32 ? sizeof(float) : sizeof(double);
    s->last_real_blocks = real_blocks;
    SCK(cudaMemsetAsync(s->grid, 0, s->ngrid * rb, stream));
    SCK(launch_atoms_any(s->f32, s->p.order, kSpread, aa, s->qs, s->grid, nullptr, nullptr,
                         stream));
    SCK(mark(1));
    if (!overlap) {
        if (half) SCK(cudaMemsetAsync(ra.fs, 0, 3 * (size_t)c->ns * sizeof(double), stream));
        SCK(launch_real(mixed, lj, c->T, half, ra, real_blocks, stream));
    }
    SCK(mark(2));
    SCK(fft3_forward_xy(s->fft, s->grid, s->ghat, stream));
    SCK(mark(3));
    SCK(fft3_z_influence(s->fft, s->ghat, s->theta, s->part + real_blocks, (int)s->nrecip,
                         stream));
    SCK(mark(4));
    SCK(fft3_inverse_yx(s->fft, s->ghat, s->grid, stream));
    SCK(mark(5));
    if (overlap) SCK(cudaStreamWaitEvent(stream, s->join, 0));
    SCK(launch_atoms_any(s->f32, s->p.order, acc ? kGatherAcc : kGatherOut, aa, s->qs, s->grid,
                         lj ? nullptr : s->fs, out, stream));
    SCK(mark(6));
    k_spme_sum<<<1, 1024, 0, stream>>>(s->part, real_blocks, s->nrecip, s->dsum);
    SCK(cudaGetLastError());
    // charges, real space, spread, 2 forward FFT passes, the z pass with the
    // influence function, 2 inverse passes, gather, sum
    c->kernels += 10;
    return MD_OK;
}

md_status read_profile(md_spme *s) {
    if (!s->prof) return MD_OK;
    // event k -> k+1 brackets: spread, real, fwd FFT, influence, inv FFT, gather
    static const int slot[6] = {0, 5, 1, 2, 3, 4};
    for (int k = 0; k < 6; ++k) {
        float ms = 0.f;
        SCK(cudaEventElapsedTime(&ms, s->ev[k], s->ev[k + 1]));
        s->ms[slot[k]] = ms;
    }
    return MD_OK;
}

// LJ forces (force-only mode) at the context's current positions, then the
// SPME forces added to them: the total force of a Coulomb + LJ state.
md_status total_forces(md_spme *s) { return enqueue(s, s->ctx->f, true, true); }

}  // namespace

extern "C" {

md_status md_spme_compute(md_spme *s, double *f, double *energy) {
    MD_TRACE("md_spme_compute");
    if (!s) return sfail(nullptr, MD_ERR_ARG, "NULL solver");
    md_ctx *c = s->ctx;
    md_status st = ensure_list(c);
    if (st != MD_OK) return sfail(s, st, c->err);
    const int64_t n = c->n_total;
    double *out = nullptr;
    if (f && is_device_pointer(f)) {
        out = f;
    } else {
        if (!s->fstage) SCK(salloc(&s->fstage, 3 * n));
        out = s->fstage;
    }
    st = enqueue(s, out, false, false);
    if (st != MD_OK) return st;
    cudaStream_t stream = c->stream;
    SCK(cudaMemcpyAsync(s->hsum, s->dsum, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    if (f && out != f)
        SCK(cudaMemcpyAsync(f, out, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    SCK(cudaStreamSynchronize(stream));
    st = read_profile(s);
    if (st != MD_OK) return st;
    if (energy) {
        energy[0] = s->hsum[0];
        energy[1] = s->hsum[1];
        energy[2] = s->e_const;
        energy[3] = (s->hsum[0] + s->hsum[1]) + s->e_const;
    }
    return MD_OK;
}

md_status md_spme_step(md_spme *s, int32_t nsteps, double *energy) {
    MD_TRACE("md_spme_step");
    if (!s) return sfail(nullptr, MD_ERR_ARG, "NULL solver");
    if (nsteps < 0) return sfail(s, MD_ERR_ARG, "nsteps must be >= 0");
    md_ctx *c = s->ctx;
    md_status st = ensure_list(c);
    if (st != MD_OK) return sfail(s, st, c->err);
    cudaStream_t stream = c->stream;
    const int every = c->params.rebuild_every;
    // per-stage events are for md_spme_compute; steps run the overlapped path
    struct ProfOff {
        md_spme *s;
        bool was;
        ~ProfOff() { s->prof = was; }
    } prof_off{s, s->prof};
    s->prof = false;
    // the opening half-kick needs the total force of the current state: the
    // one this call's predecessor left, if nothing has touched the context since
    const bool cached = s->f_step == c->step && s->f_kernels == c->kernels && s->f_pc == c->pc &&
                        s->f_oc == c->oc && c->ready &&
                        std::memcmp(&s->f_pair, &c->hpair, sizeof(Pair)) == 0;
    if (!cached) {
        st = total_forces(s);
        if (st != MD_OK) return st;
    }
    c->forces_valid = false;   // c->f holds LJ + Coulomb, not what md_step expects
    const int kb = (int)((c->ns + kThreads - 1) / kThreads);
    if (!s->kpart) SCK(salloc(&s->kpart, kb));
    for (int32_t k = 0; k < nsteps; ++k) {
        SCK(launch_kick_drift(c));
        c->ready = false;
        const int64_t n = c->step + 1;
        c->step = n;
        if (n % every == 0) {
            st = resort_and_build(c);
            if (st != MD_OK) return sfail(s, st, c->err);
            c->sorted_at = n;
            c->built_at = n;
        }
        st = total_forces(s);
        if (st != MD_OK) return st;
        k_spme_half_kick<<<kb, kThreads, 0, stream>>>(c->dbox, c->dpair, c->ns, 1,
                                                       k == nsteps - 1 ? 1 : 0, c->type[c->oc],
                                                       c->f, c->v[c->oc], s->kpart);
        SCK(cudaGetLastError());
        c->kernels += 1;
        c->ready = true;
    }
    // energies of the final state: Coulomb and LJ from the last fused pass and
    // SPME sums, KE from the last half-kick (or the current velocities when no
    // step ran)
    const int64_t real_blocks = s->last_real_blocks;
    if (nsteps == 0) {
        k_spme_half_kick<<<kb, kThreads, 0, stream>>>(c->dbox, c->dpair, c->ns, 0, 1,
                                                       c->type[c->oc], c->f, c->v[c->oc], s->kpart);
        c->kernels += 1;
    }
    k_spme_sum<<<1, 1024, 0, stream>>>(s->kpart, kb, 0, s->dsum + 2);
    k_spme_sum<<<1, 1024, 0, stream>>>(s->lpart, real_blocks, 0, s->dsum + 4);
    SCK(cudaGetLastError());
    c->kernels += 2;
    SCK(cudaMemcpyAsync(s->hsum, s->dsum, 6 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    st = check_run_flags(c);
    if (st != MD_OK) return sfail(s, st, c->err);
    s->f_step = c->step;
    s->f_kernels = c->kernels;
    s->f_pc = c->pc;
    s->f_oc = c->oc;
    std::memcpy(&s->f_pair, &c->hpair, sizeof(Pair));
    if (energy) {
        const double ecoul = (s->hsum[0] + s->hsum[1]) + s->e_const;
        energy[0] = s->hsum[4];
        energy[1] = ecoul;
        energy[2] = s->hsum[2];
        energy[3] = (energy[0] + energy[1]) + energy[2];
    }
    return MD_OK;
}

md_status md_spme_profile(md_spme *s, int32_t on) {
    if (!s) return sfail(nullptr, MD_ERR_ARG, "NULL solver");
    s->prof = on != 0;
    return MD_OK;
}

md_status md_spme_profile_read(md_spme *s, double *ms) {
    if (!s || !ms) return sfail(s, MD_ERR_ARG, "NULL argument");
    for (int k = 0; k < 6; ++k) ms[k] = s->ms[k];
    return MD_OK;
}

const char *md_spme_last_error(const md_spme *s) {
    return s ? s->err.c_str() : g_spme_error.c_str();
}

void md_spme_destroy(md_spme *s) {
    if (!s) return;
    // the context may already be gone: only the stream handles are used here
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->side) cudaStreamSynchronize(s->side);
    cudaGetLastError();
    destroy(s);
    delete s;
}

}  // extern "C"

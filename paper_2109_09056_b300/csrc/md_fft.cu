// md_fft.cu -- hand-written 3-D FFT passes of the SPME reciprocal chain (see
// md_fft.cuh for the conventions and the pass structure).
//
// A tile holds lp whole lines of one axis in shared memory, element (k, l) of
// line l at tile[k * ls + l] (ls = lp + 1 for lp > 1: consecutive lines sit in
// consecutive banks, and a line's points an odd number of slots apart).  The
// lines are transformed by Stockham's autosort formulation of the mixed-radix
// FFT: with Ns the length of the sub-transforms done so far and r the stage's
// radix, butterfly j (of n / r per line) reads the r points j + t n / r,
// multiplies point t by the twiddle W^(k t n / (Ns r)), k = j mod Ns,
// W = exp(-+ 2 pi i / n), transforms them with a radix-r DFT and writes them
// to (j - k) r + k + t Ns of the other buffer; after the last stage the line
// is in natural order (no digit reversal).  Twiddles come from a per-axis
// table computed in FP64 on the host.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "md_common.cuh"
#include "md_fft.cuh"

namespace mdb {
namespace {

constexpr int kFftThreads = 256;


template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename C>
__device__ __forceinline__ C c_add(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C c_sub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C c_mul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a times (DIR i): DIR = -1 forward (-i), +1 inverse (+i)
template <int DIR, typename C>
__device__ __forceinline__ C c_rot(C a) {
    C r;
    if (DIR < 0) { r.x = a.y; r.y = -a.x; }
    else { r.x = -a.y; r.y = a.x; }
    return r;
}

// cos and sin of 2 pi e / r for the radices done as a direct DFT (exact values
// of the roots of unity, rounded once to double)
__device__ __forceinline__ double root_cos(int r, int e) {
    if (r == 3) return e == 0 ? 1.0 : -0.5;
    if (r == 6) {
        const double c[6] = {1.0, 0.5, -0.5, -1.0, -0.5, 0.5};
        return c[e];
    }
    if (r == 5) {
        const double c[5] = {1.0, 0.30901699437494742410, -0.80901699437494742410,
                             -0.80901699437494742410, 0.30901699437494742410};
        return c[e];
    }
    const double c[7] = {1.0, 0.62348980185873353053, -0.22252093395631440429,
                         -0.90096886790241912624, -0.90096886790241912624,
                         -0.22252093395631440429, 0.62348980185873353053};
    return c[e];
}
__device__ __forceinline__ double root_sin(int r, int e) {
    if (r == 3) return e == 0 ? 0.0 : (e == 1 ? 0.86602540378443864676 : -0.86602540378443864676);
    if (r == 6) {
        const double s[6] = {0.0, 0.86602540378443864676, 0.86602540378443864676, 0.0,
                             -0.86602540378443864676, -0.86602540378443864676};
        return s[e];
    }
    if (r == 5) {
        const double s[5] = {0.0, 0.95105651629515357212, 0.58778525229247312917,
                             -0.58778525229247312917, -0.95105651629515357212};
        return s[e];
    }
    const double s[7] = {0.0, 0.78183148246802980871, 0.97492791218182360702,
                         0.43388373911755812048, -0.43388373911755812048,
                         -0.97492791218182360702, -0.78183148246802980871};
    return s[e];
}

// In-register radix-r DFT, X_m = sum_t v_t exp(DIR 2 pi i m t / r).
template <typename R, int RAD, int DIR>
__device__ __forceinline__ void dft(typename CT<R>::T (&v)[RAD]) {
    using C = typename CT<R>::T;
    if constexpr (RAD == 2) {
        const C a = v[0], b = v[1];
        v[0] = c_add(a, b);
        v[1] = c_sub(a, b);
    } else if constexpr (RAD == 4) {
        const C y0 = c_add(v[0], v[2]), y1 = c_sub(v[0], v[2]);
        const C y2 = c_add(v[1], v[3]), y3 = c_rot<DIR>(c_sub(v[1], v[3]));
        v[0] = c_add(y0, y2);
        v[2] = c_sub(y0, y2);
        v[1] = c_add(y1, y3);
        v[3] = c_sub(y1, y3);
    } else if constexpr (RAD == 8) {
        // even and odd points by radix 4, joined by the eighth roots
        C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        dft<R, 4, DIR>(e);
        dft<R, 4, DIR>(o);
        const R h = (R)0.70710678118654752440;
        C w1, w3;
        w1.x = h; w1.y = (R)DIR * h;
        w3.x = -h; w3.y = (R)DIR * h;
        const C t0 = o[0], t1 = c_mul(o[1], w1), t2 = c_rot<DIR>(o[2]), t3 = c_mul(o[3], w3);
        v[0] = c_add(e[0], t0); v[4] = c_sub(e[0], t0);
        v[1] = c_add(e[1], t1); v[5] = c_sub(e[1], t1);
        v[2] = c_add(e[2], t2); v[6] = c_sub(e[2], t2);
        v[3] = c_add(e[3], t3); v[7] = c_sub(e[3], t3);
    } else if constexpr (RAD == 16) {
        // four radix-4 DFTs over t = 4 a + b (b fixed), twiddles W16^(b m1),
        // then radix 4 across b: X[m1 + 4 m2]
        C g[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            C u[4] = {v[b], v[b + 4], v[b + 8], v[b + 12]};
            dft<R, 4, DIR>(u);
#pragma unroll
            for (int m1 = 0; m1 < 4; ++m1) g[b][m1] = u[m1];
        }
        // W16^e = exp(DIR 2 pi i e / 16), e = b m1 <= 9
        const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;
        const R h = (R)0.70710678118654752440;
        auto w16 = [&](int e, C a) -> C {
            R c, sn;
            switch (e) {
                case 0: return a;
                case 1: c = c1; sn = s1; break;
                case 2: c = h; sn = h; break;
                case 3: c = s1; sn = c1; break;
                case 4: return c_rot<DIR>(a);
                case 6: c = -h; sn = h; break;
                default: c = -c1; sn = -s1; break;  // e = 9
            }
            C w;
            w.x = c;
            w.y = (R)DIR * sn;
            return c_mul(a, w);
        };
#pragma unroll
        for (int m1 = 0; m1 < 4; ++m1) {
            C u[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) u[b] = w16(b * m1, g[b][m1]);
            dft<R, 4, DIR>(u);
#pragma unroll
            for (int m2 = 0; m2 < 4; ++m2) v[m1 + 4 * m2] = u[m2];
        }
    } else {
        C o[RAD];
#pragma unroll
        for (int m = 0; m < RAD; ++m) {
            R re = v[0].x, im = v[0].y;
#pragma unroll
            for (int t = 1; t < RAD; ++t) {
                const int e = (m * t) % RAD;
                const R c = (R)root_cos(RAD, e), s = (R)DIR * (R)root_sin(RAD, e);
                re += v[t].x * c - v[t].y * s;
                im += v[t].x * s + v[t].y * c;
            }
            o[m].x = re;
            o[m].y = im;
        }
#pragma unroll
        for (int m = 0; m < RAD; ++m) v[m] = o[m];
    }
}

// j / d for j < 2^16 and 1 < d <= 4096 by a multiply-high with m = ceil(2^32 / d)
// (exact: the rounding up adds less than j d / 2^32 < 1 / d to j / d).
__device__ __forceinline__ uint32_t divm(uint32_t j, uint32_t m) { return __umulhi(j, m); }

// One Stockham stage of radix RAD over the tile's LP lines (lines past the
// tile's real ones, in the last tile of a pass, transform garbage that is
// never stored).  tw: the axis's twiddle table in shared memory.
template <typename R, int LP, int RAD, int DIR>
__device__ __forceinline__ void stage(const typename CT<R>::T *in, typename CT<R>::T *out,
                                      const typename CT<R>::T *tw, int n, int ls, int Ns,
                                      uint32_t mg) {
    using C = typename CT<R>::T;
    const int nb = n / RAD, step = n / (Ns * RAD);
    for (int w = threadIdx.x; w < nb * LP; w += blockDim.x) {
        const int l = w % LP, j = w / LP;
        const int q = Ns > 1 ? (int)divm((uint32_t)j, mg) : j;
        const int k = j - q * Ns;
        C v[RAD];
#pragma unroll
        for (int t = 0; t < RAD; ++t) v[t] = in[(j + t * nb) * ls + l];
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < RAD; ++t) {
                C W = tw[k * t * step];
                if (DIR > 0) W.y = -W.y;
                v[t] = c_mul(v[t], W);
            }
        }
        dft<R, RAD, DIR>(v);
        const int base = q * Ns * RAD + k;
#pragma unroll
        for (int t = 0; t < RAD; ++t) out[(base + t * Ns) * ls + l] = v[t];
    }
}

// Transforms the tile's LP lines through every stage of the axis; returns the
// buffer holding the result.
template <typename R, int LP, int DIR>
__device__ typename CT<R>::T *fft_tile(typename CT<R>::T *b0, typename CT<R>::T *b1,
                                        const typename CT<R>::T *tw, const FftAxis &ax) {
    using C = typename CT<R>::T;
    C *in = b0, *out = b1;
    int Ns = 1;
    const int n = ax.n, ls = ax.ls;
    for (int s = 0; s < ax.nst; ++s) {
        const int r = ax.rad[s];
        const uint32_t mg = ax.mg[s];
        switch (r) {
            case 16:
                if constexpr (sizeof(R) == 8) stage<R, LP, 16, DIR>(in, out, tw, n, ls, Ns, mg);
                break;
            case 8: stage<R, LP, 8, DIR>(in, out, tw, n, ls, Ns, mg); break;
            case 6: stage<R, LP, 6, DIR>(in, out, tw, n, ls, Ns, mg); break;
            case 4: stage<R, LP, 4, DIR>(in, out, tw, n, ls, Ns, mg); break;
            case 2: stage<R, LP, 2, DIR>(in, out, tw, n, ls, Ns, mg); break;
            case 3: stage<R, LP, 3, DIR>(in, out, tw, n, ls, Ns, mg); break;
            case 5: stage<R, LP, 5, DIR>(in, out, tw, n, ls, Ns, mg); break;
            default: stage<R, LP, 7, DIR>(in, out, tw, n, ls, Ns, mg); break;
        }
        __syncthreads();
        C *t = in;
        in = out;
        out = t;
        Ns *= r;
    }
    return in;
}

// Shared memory of a pass: the axis's twiddles (n), then two tile buffers of
// n * ls elements.
template <typename C>
__device__ __forceinline__ C *load_twiddles(unsigned char *smem, const FftAxis &ax) {
    C *tw = reinterpret_cast<C *>(smem);
    const C *g = static_cast<const C *>(ax.tw);
    for (int k = threadIdx.x; k < ax.n; k += blockDim.x) tw[k] = __ldg(g + k);
    return tw;
}

// Each thread moves at most kFftElems elements of a tile (tiles hold at most
// kFftThreads * kFftElems points: lp * n <= 3072).  A CTA loads its next
// tile into registers while it transforms the current one, so that the DRAM
// latency of the loads overlaps the Stockham stages.
constexpr int kFftElems = 12;

// x passes: two real rows share one complex line (row 2 l in the real part,
// row 2 l + 1 in the imaginary part), so a tile of LP lines carries 2 LP rows.
// Forward: Z = FFT(a + i b) gives A_m = (Z_m + conj Z_{n-m}) / 2 and
// B_m = (Z_m - conj Z_{n-m}) / (2 i).  Inverse: Z_k = A_k + i B_k over the
// whole spectrum (each half extended by X_{n-k} = conj X_k, the imaginary
// parts of X_0 and, for even n, X_{n/2} dropped as a real inverse does), and
// a = Re IFFT(Z), b = Im IFFT(Z).

// x pass, forward: rows (z, y) of K_x reals -> K_x / 2 + 1 complex.
template <typename R, int LP>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 1) k_fft_x_r2c(const R *__restrict__ grid,
                                                           typename CT<R>::T *__restrict__ ghat,
                                                           FftAxis ax, int64_t nrows, int Kh,
                                                           uint32_t mkh) {
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = ax.n, ls = ax.ls;
    C *tw = load_twiddles<C>(smem, ax);
    C *b0 = tw + n, *b1 = b0 + (size_t)n * ls;
    constexpr int RT = 2 * LP;  // rows per tile
    R pre[2 * kFftElems];
    auto fetch = [&](int64_t r0) {
        const int nr = (int)(nrows - r0 < RT ? nrows - r0 : RT);
        const R *src = grid + r0 * n;
#pragma unroll
        for (int e = 0; e < 2 * kFftElems; ++e) {
            const int idx = threadIdx.x + e * kFftThreads;
            if (idx < nr * n) pre[e] = src[idx];
        }
    };
    int64_t r0 = (int64_t)blockIdx.x * RT;
    if (r0 < nrows) fetch(r0);
    for (; r0 < nrows; r0 += (int64_t)gridDim.x * RT) {
        const int nr = (int)(nrows - r0 < RT ? nrows - r0 : RT);
        R *bs = reinterpret_cast<R *>(b0);
#pragma unroll
        for (int e = 0; e < 2 * kFftElems; ++e) {
            const int idx = threadIdx.x + e * kFftThreads;
            if (idx < nr * n) {
                const int row = (int)divm((uint32_t)idx, ax.mn), k = idx - row * n;
                bs[2 * (k * ls + (row >> 1)) + (row & 1)] = pre[e];
            }
        }
        if (nr & 1)  // a lone last row: its partner is zero
            for (int k = threadIdx.x; k < n; k += blockDim.x) bs[2 * (k * ls + (nr >> 1)) + 1] = (R)0;
        __syncthreads();
        const int64_t rn = r0 + (int64_t)gridDim.x * RT;
        if (rn < nrows) fetch(rn);
        const C *res = fft_tile<R, LP, -1>(b0, b1, tw, ax);
        C *dst = ghat + r0 * Kh;
        for (int idx = threadIdx.x; idx < nr * Kh; idx += blockDim.x) {
            const int row = (int)divm((uint32_t)idx, mkh), m = idx - row * Kh;
            const int l = row >> 1;
            const C z = res[m * ls + l], w = res[(m == 0 ? 0 : n - m) * ls + l];
            C o;
            if (row & 1) {  // (Z_m - conj Z_{n-m}) / (2 i)
                o.x = (R)0.5 * (z.y + w.y);
                o.y = (R)0.5 * (w.x - z.x);
            } else {        // (Z_m + conj Z_{n-m}) / 2
                o.x = (R)0.5 * (z.x + w.x);
                o.y = (R)0.5 * (z.y - w.y);
            }
            dst[idx] = o;
        }
        __syncthreads();
    }
}

// x pass, inverse: rows of K_x / 2 + 1 complex (a Hermitian spectrum's half)
// -> K_x reals (the unnormalised inverse of the whole spectrum).
template <typename R, int LP>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 1) k_fft_x_c2r(const typename CT<R>::T *__restrict__ ghat,
                                                           R *__restrict__ grid, FftAxis ax,
                                                           int64_t nrows, int Kh, uint32_t mkh) {
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = ax.n, ls = ax.ls;
    C *tw = load_twiddles<C>(smem, ax);
    C *b0 = tw + n, *b1 = b0 + (size_t)n * ls;
    constexpr int RT = 2 * LP;
    // 2 lp rows of K_x / 2 + 1 <= lp n + 2 lp <= kFftThreads (kFftElems + 2) elements
    constexpr int E = kFftElems + 2;
    C pre[E];
    auto fetch = [&](int64_t r0) {
        const int nr = (int)(nrows - r0 < RT ? nrows - r0 : RT);
        const C *src = ghat + r0 * Kh;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = threadIdx.x + e * kFftThreads;
            if (idx < nr * Kh) pre[e] = src[idx];
        }
    };
    // row's element k of the half (k < Kh) as its terms of Z at k and n - k
    // (the even row gives X, the odd one i X), added into the line
    auto put = [&](int row, int k, C v, bool add) {
        const int l = row >> 1;
        if (k == 0 || 2 * k == n) v.y = (R)0;  // real for a real row
        C a = v, c = v;                        // Z_k and Z_{n-k} terms
        c.y = -c.y;                            // conj
        if (row & 1) {                         // times i
            a.x = -v.y; a.y = v.x;
            c.x = v.y;  c.y = v.x;
        }
        C *p = b0 + k * ls + l;
        if (add) { p->x += a.x; p->y += a.y; }
        else *p = a;
        if (k > 0 && n - k >= Kh) {
            C *q = b0 + (n - k) * ls + l;
            if (add) { q->x += c.x; q->y += c.y; }
            else *q = c;
        }
    };
    int64_t r0 = (int64_t)blockIdx.x * RT;
    if (r0 < nrows) fetch(r0);
    for (; r0 < nrows; r0 += (int64_t)gridDim.x * RT) {
        const int nr = (int)(nrows - r0 < RT ? nrows - r0 : RT);
        // even rows set the lines, then odd rows add theirs
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = threadIdx.x + e * kFftThreads;
            if (idx < nr * Kh) {
                const int row = (int)divm((uint32_t)idx, mkh), k = idx - row * Kh;
                if (!(row & 1)) put(row, k, pre[e], false);
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = threadIdx.x + e * kFftThreads;
            if (idx < nr * Kh) {
                const int row = (int)divm((uint32_t)idx, mkh), k = idx - row * Kh;
                if (row & 1) put(row, k, pre[e], true);
            }
        }
        __syncthreads();
        const int64_t rn = r0 + (int64_t)gridDim.x * RT;
        if (rn < nrows) fetch(rn);
        const C *res = fft_tile<R, LP, 1>(b0, b1, tw, ax);
        R *dst = grid + r0 * n;
        for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
            const int row = (int)divm((uint32_t)idx, ax.mn), k = idx - row * n;
            const C z = res[k * ls + (row >> 1)];
            dst[idx] = (row & 1) ? z.y : z.x;
        }
        __syncthreads();
    }
}

// Lines along an axis of the half spectrum with stride `stride` between their
// points: tile t covers lines of `plane` (the outer index) and LP consecutive
// m_x.  Element (k, line l) of tile (o, x0) is at
// ghat[o * ostride + k * stride + x0 + l].
struct LineTiles {
    int64_t ostride, stride;  // complex elements
    int nouter;               // outer planes
    int xt;                   // tiles per plane along m_x
    int Kh;
};

// A tile of lines: its origin in the half spectrum and its real line count.
struct LineTile {
    int64_t off;
    int x0, lp;
};

template <int LP>
__device__ __forceinline__ LineTile line_tile(const LineTiles &lt, int64_t t) {
    const int o = (int)(t / lt.xt);
    LineTile r;
    r.x0 = (int)(t - (int64_t)o * lt.xt) * LP;
    r.lp = min(LP, lt.Kh - r.x0);
    r.off = o * lt.ostride + r.x0;
    return r;
}

// Registers <- a tile's points (element e of this thread: idx = tid + e T,
// point k = idx / LP of line l = idx % LP).
template <typename C, int LP>
__device__ __forceinline__ void fetch_lines(C (&pre)[kFftElems], const C *g, int n, int lp,
                                            int64_t stride) {
#pragma unroll
    for (int e = 0; e < kFftElems; ++e) {
        const int idx = threadIdx.x + e * kFftThreads;
        const int k = idx / LP, l = idx % LP;
        if (k < n && l < lp) pre[e] = g[k * stride + l];
    }
}

template <typename C, int LP>
__device__ __forceinline__ void commit_lines(C *b0, const C (&pre)[kFftElems], int n, int ls,
                                             int lp) {
#pragma unroll
    for (int e = 0; e < kFftElems; ++e) {
        const int idx = threadIdx.x + e * kFftThreads;
        const int k = idx / LP, l = idx % LP;
        if (k < n && l < lp) b0[k * ls + l] = pre[e];
    }
}

template <typename C, int LP>
__device__ __forceinline__ void store_lines(C *g, const C *res, int n, int ls, int lp,
                                            int64_t stride) {
    for (int idx = threadIdx.x; idx < LP * n; idx += blockDim.x) {
        const int k = idx / LP, l = idx % LP;
        if (l < lp) g[k * stride + l] = res[k * ls + l];
    }
}

template <typename R, int LP, int DIR>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 1) k_fft_lines(typename CT<R>::T *__restrict__ ghat,
                                                           FftAxis ax, LineTiles lt) {
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = ax.n, ls = ax.ls;
    C *tw = load_twiddles<C>(smem, ax);
    C *b0 = tw + n, *b1 = b0 + (size_t)n * ls;
    const int64_t ntiles = (int64_t)lt.nouter * lt.xt;
    C pre[kFftElems];
    int64_t t = blockIdx.x;
    if (t < ntiles) {
        const LineTile f = line_tile<LP>(lt, t);
        fetch_lines<C, LP>(pre, ghat + f.off, n, f.lp, lt.stride);
    }
    for (; t < ntiles; t += gridDim.x) {
        const LineTile cur = line_tile<LP>(lt, t);
        commit_lines<C, LP>(b0, pre, n, ls, cur.lp);
        __syncthreads();
        if (t + gridDim.x < ntiles) {
            const LineTile f = line_tile<LP>(lt, t + gridDim.x);
            fetch_lines<C, LP>(pre, ghat + f.off, n, f.lp, lt.stride);
        }
        const C *res = fft_tile<R, LP, DIR>(b0, b1, tw, ax);
        store_lines<C, LP>(ghat + cur.off, res, n, ls, cur.lp, lt.stride);
        __syncthreads();
    }
}

template <int NT>
__device__ __forceinline__ void block_sum_to(double v, double *out) {
    __shared__ double red[NT / 32];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (threadIdx.x == 0) *out = u;
    }
}

// z pass fused with the influence function: lines along m_z at fixed (m_y,
// m_x-tile) go forward, are multiplied by theta (their energy terms summed on
// the way), and come back.  CTA b takes tiles b, b + nparts, ... and writes its
// energy partial to part[b] (a fixed order: deterministic).
template <typename R, int LP>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 1) k_fft_z_influence(typename CT<R>::T *__restrict__ ghat,
                                                                 const R *__restrict__ theta,
                                                                 FftAxis ax, LineTiles lt, int Kx,
                                                                 double *__restrict__ part) {
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = ax.n, ls = ax.ls;
    C *tw = load_twiddles<C>(smem, ax);
    C *b0 = tw + n, *b1 = b0 + (size_t)n * ls;
    const int64_t ntiles = (int64_t)lt.nouter * lt.xt;
    double e = 0.0;
    C pre[kFftElems];
    int64_t t = blockIdx.x;
    if (t < ntiles) {
        const LineTile f = line_tile<LP>(lt, t);
        fetch_lines<C, LP>(pre, ghat + f.off, n, f.lp, lt.stride);
    }
    for (; t < ntiles; t += gridDim.x) {
        const LineTile cur = line_tile<LP>(lt, t);
        commit_lines<C, LP>(b0, pre, n, ls, cur.lp);
        __syncthreads();
        if (t + gridDim.x < ntiles) {
            const LineTile f = line_tile<LP>(lt, t + gridDim.x);
            fetch_lines<C, LP>(pre, ghat + f.off, n, f.lp, lt.stride);
        }
        // the tile's theta, in flight during the forward transform
        R th[kFftElems];
#pragma unroll
        for (int q = 0; q < kFftElems; ++q) {
            const int idx = threadIdx.x + q * kFftThreads;
            const int k = idx / LP, l = idx % LP;
            if (k < n && l < cur.lp) th[q] = __ldg(theta + cur.off + k * lt.stride + l);
        }
        C *res = fft_tile<R, LP, -1>(b0, b1, tw, ax);
#pragma unroll
        for (int q = 0; q < kFftElems; ++q) {
            const int idx = threadIdx.x + q * kFftThreads;
            const int k = idx / LP, l = idx % LP;
            if (k < n && l < cur.lp) {
                const int mx = cur.x0 + l;
                C v = res[k * ls + l];
                const R wgt = (mx == 0 || 2 * mx == Kx) ? (R)1 : (R)2;
                e += (double)(wgt * th[q] * (v.x * v.x + v.y * v.y));
                v.x *= th[q];
                v.y *= th[q];
                res[k * ls + l] = v;
            }
        }
        __syncthreads();
        C *other = res == b0 ? b1 : b0;
        const C *back = fft_tile<R, LP, 1>(res, other, tw, ax);
        store_lines<C, LP>(ghat + cur.off, back, n, ls, cur.lp, lt.stride);
        __syncthreads();
    }
    block_sum_to<kFftThreads>(e, part + blockIdx.x);
}

size_t tile_bytes(const FftAxis &ax, bool f32) {
    return (size_t)ax.n * (1 + 2 * (size_t)ax.ls) * (f32 ? sizeof(float2) : sizeof(double2));
}

// Raises a kernel's dynamic shared-memory limit (per kernel and device, once
// per size above the default 48 KB).
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = set[{reinterpret_cast<const void *>(kernel), dev}];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

// Persistent grids: at most 8 CTAs per SM of the current device.
int fft_blocks(int64_t tiles) {
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nsm = 148;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)nsm * 8));
}

uint32_t magic(int d) { return (uint32_t)(((1ull << 32) + (uint64_t)d - 1) / (uint64_t)d); }

LineTiles y_lines(const Fft3 &p) {
    LineTiles lt;
    lt.stride = p.Kh;                              // along m_y
    lt.ostride = (int64_t)p.K[1] * p.Kh;           // planes m_z
    lt.nouter = p.K[2];
    lt.xt = (p.Kh + p.ax[1].lp - 1) / p.ax[1].lp;
    lt.Kh = p.Kh;
    return lt;
}

LineTiles z_lines(const Fft3 &p) {
    LineTiles lt;
    lt.stride = (int64_t)p.K[1] * p.Kh;            // along m_z
    lt.ostride = p.Kh;                             // planes m_y
    lt.nouter = p.K[1];
    lt.xt = (p.Kh + p.ax[2].lp - 1) / p.ax[2].lp;
    lt.Kh = p.Kh;
    return lt;
}

template <typename R, int LP>
cudaError_t x_pass(const Fft3 &p, const void *in, void *out, bool forward, cudaStream_t st) {
    using C = typename CT<R>::T;
    const FftAxis &ax = p.ax[0];
    const int64_t rows = (int64_t)p.K[1] * p.K[2];
    const size_t sm = tile_bytes(ax, sizeof(R) == 4);
    const int blocks = fft_blocks((rows + 2 * LP - 1) / (2 * LP));
    const uint32_t mkh = magic(p.Kh);
    cudaError_t e;
    if (forward) {
        e = allow_smem(k_fft_x_r2c<R, LP>, sm);
        if (e != cudaSuccess) return e;
        k_fft_x_r2c<R, LP><<<blocks, kFftThreads, sm, st>>>(static_cast<const R *>(in),
                                                            static_cast<C *>(out), ax, rows, p.Kh,
                                                            mkh);
    } else {
        e = allow_smem(k_fft_x_c2r<R, LP>, sm);
        if (e != cudaSuccess) return e;
        k_fft_x_c2r<R, LP><<<blocks, kFftThreads, sm, st>>>(static_cast<const C *>(in),
                                                            static_cast<R *>(out), ax, rows, p.Kh,
                                                            mkh);
    }
    return cudaGetLastError();
}

template <typename R, int LP, int DIR>
cudaError_t line_pass(const Fft3 &p, void *ghat, int axis, cudaStream_t st) {
    using C = typename CT<R>::T;
    const LineTiles lt = axis == 1 ? y_lines(p) : z_lines(p);
    const size_t sm = tile_bytes(p.ax[axis], sizeof(R) == 4);
    cudaError_t e = allow_smem(k_fft_lines<R, LP, DIR>, sm);
    if (e != cudaSuccess) return e;
    k_fft_lines<R, LP, DIR><<<fft_blocks((int64_t)lt.nouter * lt.xt), kFftThreads, sm, st>>>(
        static_cast<C *>(ghat), p.ax[axis], lt);
    return cudaGetLastError();
}

template <typename R, int LP>
cudaError_t z_pass(const Fft3 &p, void *ghat, const void *theta, double *part, int nparts,
                   cudaStream_t st) {
    using C = typename CT<R>::T;
    const LineTiles lt = z_lines(p);
    const size_t sm = tile_bytes(p.ax[2], sizeof(R) == 4);
    cudaError_t e = allow_smem(k_fft_z_influence<R, LP>, sm);
    if (e != cudaSuccess) return e;
    k_fft_z_influence<R, LP><<<nparts, kFftThreads, sm, st>>>(
        static_cast<C *>(ghat), static_cast<const R *>(theta), p.ax[2], lt, p.K[0], part);
    return cudaGetLastError();
}

// The tile width as a template argument.
#define MD_FFT_LP_DISPATCH(lp, call_lp)       \
    switch (lp) {                             \
        case 16: return call_lp(16);          \
        case 8: return call_lp(8);            \
        case 4: return call_lp(4);            \
        case 2: return call_lp(2);            \
        default: return call_lp(1);           \
    }

template <typename R>
cudaError_t x_any(const Fft3 &p, const void *in, void *out, bool fwd, cudaStream_t st) {
#define MD_X(L) x_pass<R, L>(p, in, out, fwd, st)
    MD_FFT_LP_DISPATCH(p.ax[0].lp, MD_X)
#undef MD_X
}

template <typename R, int DIR>
cudaError_t lines_any(const Fft3 &p, void *ghat, int axis, cudaStream_t st) {
#define MD_L(L) line_pass<R, L, DIR>(p, ghat, axis, st)
    MD_FFT_LP_DISPATCH(p.ax[axis].lp, MD_L)
#undef MD_L
}

template <typename R>
cudaError_t z_any(const Fft3 &p, void *ghat, const void *theta, double *part, int nparts,
                  cudaStream_t st) {
#define MD_Z(L) z_pass<R, L>(p, ghat, theta, part, nparts, st)
    MD_FFT_LP_DISPATCH(p.ax[2].lp, MD_Z)
#undef MD_Z
}

template <typename R>
cudaError_t forward_xy(const Fft3 &p, const void *grid, void *ghat, cudaStream_t st) {
    cudaError_t e = x_any<R>(p, grid, ghat, true, st);
    if (e != cudaSuccess) return e;
    return lines_any<R, -1>(p, ghat, 1, st);
}

template <typename R>
cudaError_t inverse_yx(const Fft3 &p, void *ghat, void *grid, cudaStream_t st) {
    cudaError_t e = lines_any<R, 1>(p, ghat, 1, st);
    if (e != cudaSuccess) return e;
    return x_any<R>(p, ghat, grid, false, st);
}

}  // namespace

bool fft_factor(int n, bool f32, int *rad, int *nst) {
    int k = 0;
    if (n < 2) return false;
    for (int r : {16, 8, 6, 4, 2, 3, 5, 7}) {
        if (r == 16 && f32) continue;
        while (n % r == 0) {
            if (k == kFftMaxStages) return false;
            rad[k++] = r;
            n /= r;
        }
    }
    *nst = k;
    return n == 1;
}

cudaError_t fft3_plan(Fft3 *p, const int K[3], bool f32) {
    p->f32 = f32;
    for (int d = 0; d < 3; ++d) p->K[d] = K[d];
    p->Kh = K[0] / 2 + 1;
    // shared-memory budget of one tile (two buffers), per precision
    const size_t budget = f32 ? 64 * 1024 : 128 * 1024;
    const size_t csize = f32 ? sizeof(float2) : sizeof(double2);
    for (int d = 0; d < 3; ++d) {
        FftAxis &ax = p->ax[d];
        ax.n = K[d];
        if (!fft_factor(ax.n, f32, ax.rad, &ax.nst)) return cudaErrorInvalidValue;
        ax.mn = ax.n > 1 ? (uint32_t)(((1ull << 32) + ax.n - 1) / ax.n) : 0u;
        for (int st = 0, Ns = 1; st < ax.nst; Ns *= ax.rad[st], ++st)
            ax.mg[st] = Ns > 1 ? (uint32_t)(((1ull << 32) + Ns - 1) / Ns) : 0u;
        ax.lp = 1;
        ax.ls = 1;
        // the x pass takes whole rows; the y and z passes up to 16 m_x at once
        for (int lp : {16, 8, 4, 2}) {
            if (d == 0 && lp > 8) continue;
            if (lp * ax.n > kFftThreads * kFftElems) continue;  // a thread's share in registers
            if ((size_t)ax.n * (1 + 2 * (size_t)(lp + 1)) * csize <= budget) {
                ax.lp = lp;
                ax.ls = lp + 1;
                break;
            }
        }
        if ((size_t)ax.n * (1 + 2 * (size_t)ax.ls) * csize > 200 * 1024) return cudaErrorInvalidValue;
        // twiddles exp(-2 pi i k / n) in FP64, rounded once
        std::vector<double> tw(2 * (size_t)ax.n);
        const double pi = 3.141592653589793238462643;
        for (int k = 0; k < ax.n; ++k) {
            tw[2 * k] = std::cos(2.0 * pi * k / ax.n);
            tw[2 * k + 1] = -std::sin(2.0 * pi * k / ax.n);
        }
        cudaError_t e = cudaMalloc(&ax.tw, (size_t)ax.n * csize);
        if (e != cudaSuccess) return e;
        if (f32) {
            std::vector<float> t32(tw.begin(), tw.end());
            e = cudaMemcpy(ax.tw, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
        } else {
            e = cudaMemcpy(ax.tw, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void fft3_free(Fft3 *p) {
    for (auto &ax : p->ax) {
        if (ax.tw) cudaFree(ax.tw);
        ax.tw = nullptr;
    }
}

cudaError_t fft3_forward_xy(const Fft3 &p, const void *grid, void *ghat, cudaStream_t st) {
    return p.f32 ? forward_xy<float>(p, grid, ghat, st) : forward_xy<double>(p, grid, ghat, st);
}

cudaError_t fft3_z_influence(const Fft3 &p, void *ghat, const void *theta, double *part,
                             int nparts, cudaStream_t st) {
    return p.f32 ? z_any<float>(p, ghat, theta, part, nparts, st)
                 : z_any<double>(p, ghat, theta, part, nparts, st);
}

cudaError_t fft3_inverse_yx(const Fft3 &p, void *ghat, void *grid, cudaStream_t st) {
    return p.f32 ? inverse_yx<float>(p, ghat, grid, st) : inverse_yx<double>(p, ghat, grid, st);
}

}  // namespace mdb

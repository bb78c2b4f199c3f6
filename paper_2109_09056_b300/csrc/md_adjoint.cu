// md_adjoint.cu -- force-matching adjoint of the LJ force kernel (FP64).
//
// Upstream gradients G = dL/dF (per atom) and gE = dL/dPE.  With d = x_i - x_j
// (nearest image), u = |d|^2 < rc^2, s6 = (sigma^2/u)^3, s12 = s6^2:
//   phi = (24 eps/u)(2 s12 - s6)          (F_i = sum_j phi d)
//   psi = 2 dphi/du = (48 eps/u^2)(4 s6 - 14 s12)
//   dL/dx_i = sum_j [phi (G_i - G_j) + psi d (d . (G_i - G_j))] - gE F_i
// (the Jacobian block M_ij = phi I + psi d d^T is symmetric and the list is
// full, so the gather form needs no atomics), and for the type pair (a, b) of
// each ordered pair
//   dL/deps_ab   += (G_i . d) phi/eps + gE/2 dU/deps
//   dL/dsigma_ab += (G_i . d) (24 eps/u)(24 s12 - 6 s6)/sigma + gE/2 dU/dsigma
// with dU/deps = 4(s12 - s6), dU/dsigma = 4 eps (12 s12 - 6 s6)/sigma, minus the
// same at rc when energies are shifted.  Ordered-pair partials are kept per
// lane in shared memory, reduced per warp-tile in lane order and then over
// warp-tiles in tile order, so the result is deterministic.
#include "md_common.cuh"

namespace mdb {
namespace {

constexpr int kAdjThreads = 128;

struct AdjArgs {
    const Box *boxes;
    const int32_t *tile_box;
    const Pair *pair;
    int64_t ns, nwt;
    int pad, R;
    const double *r;
    const int32_t *type;
    const int32_t *id;
    const int32_t *nn;
    const uint32_t *nbr;
    const double *G;   // slot order SoA (3*ns)
    double gE;
    double *dx_aos;    // original order
    double *part;      // nwt * NP
    int NP;
    Flags *fl;
};

__global__ void k_gather_G(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                           int64_t ns, const int32_t *__restrict__ id,
                           const double *__restrict__ G_aos, double *__restrict__ Gs) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const Box &B = boxes[tile_box[k >> 5]];
    const bool valid = k - B.slot_off < B.n;
    const int64_t g = valid ? id[k] : 0;
    for (int d = 0; d < 3; ++d) Gs[d * ns + k] = valid ? G_aos[3 * g + d] : 0.0;
}

template <int T>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint(AdjArgs a) {
    if (a.fl->status & ST_FREEZE) return;
    constexpr int A = 32 / T;
    extern __shared__ double s_acc[];          // blockDim * NP
    __shared__ double s_off[kAdjThreads / 32][81];
    __shared__ double t_e24[64], t_s2[64], t_ie[64], t_is[64], t_she[64], t_shs[64], t_eps[64];
    const Pair &P = *a.pair;
    for (int t = threadIdx.x; t < 64; t += blockDim.x) {
        t_e24[t] = P.e24[t];
        t_s2[t] = P.s2[t];
        t_eps[t] = P.eps[t];
        const double e = P.eps[t], s = P.sig[t];
        t_ie[t] = e != 0.0 ? 1.0 / e : 0.0;
        t_is[t] = s != 0.0 ? 1.0 / s : 0.0;
        if (P.shift && s != 0.0) {
            const double c2 = (s * s) / P.rc2, c6 = c2 * c2 * c2, c12 = c6 * c6;
            t_she[t] = 4.0 * (c12 - c6);
            t_shs[t] = 4.0 * e * (12.0 * c12 - 6.0 * c6) / s;
        } else {
            t_she[t] = 0.0;
            t_shs[t] = 0.0;
        }
    }
    const int NP = a.NP;
    double *acc = s_acc + (size_t)threadIdx.x * NP;
    for (int q = 0; q < NP; ++q) acc[q] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, sub = lane % T;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int nt = P.nt;
    const double rc2 = P.rc2, gE = a.gE;
    int curbox = -1;
    for (int64_t wt = gw; wt < a.nwt; wt += nw) {
        const int64_t i = wt * A + lane / T;
        const int b = a.tile_box[(wt * A) >> 5];
        const Box &B = a.boxes[b];
        if (b != curbox) {
            if (lane < 27) {
                s_off[wib][3 * lane + 0] = (double)(lane % 3 - 1) * B.h[0];
                s_off[wib][3 * lane + 1] = (double)((lane / 3) % 3 - 1) * B.h[1];
                s_off[wib][3 * lane + 2] = (double)(lane / 9 - 1) * B.h[2];
            }
            __syncwarp();
            curbox = b;
        }
        const bool valid = (i - B.slot_off) < B.n;
        const int ni = valid ? min(a.nn[i], a.pad) : 0;
        const uint32_t *row = a.nbr + (size_t)wt * a.R * 32 + lane;
        const double rix = a.r[i], riy = a.r[a.ns + i], riz = a.r[2 * a.ns + i];
        const double gix = a.G[i], giy = a.G[a.ns + i], giz = a.G[2 * a.ns + i];
        const int ti = a.type[i];
        double gx = 0.0, gy = 0.0, gz = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        int q = 0;
        for (int k = sub; k < ni; k += T, ++q) {
            const uint32_t e = row[(size_t)q * 32];
            const int64_t j = chk_index(e & MD_IDX_MASK, a.ns, CHK_ADJ_GATHER, a.fl, 0);
            const double *o = s_off[wib] + 3 * (e >> MD_IDX_BITS);
            // d = x_i - x_j
            const double dx = rix - (a.r[j] + o[0]);
            const double dy = riy - (a.r[a.ns + j] + o[1]);
            const double dz = riz - (a.r[2 * a.ns + j] + o[2]);
            const double u = (dx * dx + dy * dy) + dz * dz;
            if (!(u < rc2)) continue;
            const int ab = ti * nt + a.type[j];
            const double iu = rcp_newton64(u);
            const double q2 = t_s2[ab] * iu;
            const double s6 = q2 * q2 * q2, s12 = s6 * s6;
            const double e24u = t_e24[ab] * iu;
            const double phi = e24u * (2.0 * s12 - s6);
            const double psi = 2.0 * (e24u * iu) * (4.0 * s6 - 14.0 * s12);
            const double Gdx = gix - a.G[j], Gdy = giy - a.G[a.ns + j], Gdz = giz - a.G[2 * a.ns + j];
            const double dG = dx * Gdx + dy * Gdy + dz * Gdz;
            gx += phi * Gdx + psi * dx * dG;
            gy += phi * Gdy + psi * dy * dG;
            gz += phi * Gdz + psi * dz * dG;
            fx += phi * dx;
            fy += phi * dy;
            fz += phi * dz;
            const double dGi = dx * gix + dy * giy + dz * giz;
            const double eps = t_eps[ab];
            const double dphide = phi * t_ie[ab];
            const double dphids = e24u * (24.0 * s12 - 6.0 * s6) * t_is[ab];
            const double dUde = 4.0 * (s12 - s6) - t_she[ab];
            const double dUds = 4.0 * eps * (12.0 * s12 - 6.0 * s6) * t_is[ab] - t_shs[ab];
            acc[2 * ab] += dGi * dphide + 0.5 * gE * dUde;
            acc[2 * ab + 1] += dGi * dphids + 0.5 * gE * dUds;
        }
#pragma unroll
        for (int o = T / 2; o >= 1; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (valid && sub == 0) {
            const int64_t g = a.id[i];
            a.dx_aos[3 * g + 0] = gx - gE * fx;
            a.dx_aos[3 * g + 1] = gy - gE * fy;
            a.dx_aos[3 * g + 2] = gz - gE * fz;
        }
        __syncwarp();
        for (int p = lane; p < NP; p += 32) {
            double s = 0.0;
            for (int l = 0; l < 32; ++l) s += s_acc[(size_t)(wib * 32 + l) * NP + p];
            a.part[wt * NP + p] = s;
        }
        __syncwarp();
        for (int p = 0; p < NP; ++p) acc[p] = 0.0;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_adj_reduce(const double *__restrict__ part, int64_t nwt,
                                                    int NP, double *__restrict__ out) {
    __shared__ double red[256];
    for (int p = 0; p < NP; ++p) {
        double s = 0.0;
        for (int64_t w = threadIdx.x; w < nwt; w += blockDim.x) s += part[w * NP + p];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = 128; h >= 1; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[p] = red[0];
        __syncthreads();
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <int T>
cudaError_t launch_adj_t(md_ctx *c, const AdjArgs &a) {
    const size_t smem = (size_t)kAdjThreads * a.NP * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_adjoint<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adjoint<T>, kAdjThreads, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)c->nsm * (per > 0 ? per : 1);
    const int64_t need = (a.nwt + 3) / 4;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_adjoint<T><<<(unsigned)grid, kAdjThreads, smem, c->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

// G_aos, dx_aos: device pointers in original order; the scratch holds the slot
// order G (3*ns) followed by the warp-tile partials (nwt*NP) and totals (NP).
cudaError_t launch_adjoint(md_ctx *c, const double *G_aos, double gE, double *dx_aos,
                           double *totals_out, double *scratch) {
    const int T = c->T;
    const int NP = 2 * c->hpair.nt * c->hpair.nt;
    const int64_t nwt = c->ns / (32 / T);
    double *Gs = scratch;
    double *part = Gs + 3 * c->ns;
    const int t = 256;
    k_gather_G<<<blocks_for(c->ns, t), t, 0, c->stream>>>(c->dbox, c->tile_box, c->ns,
                                                           c->id[c->oc], G_aos, Gs);
    AdjArgs a;
    a.boxes = c->dbox;
    a.tile_box = c->tile_box;
    a.pair = c->dpair;
    a.ns = c->ns;
    a.nwt = nwt;
    a.pad = c->pad;
    a.R = c->R;
    a.r = c->r[c->pc];
    a.type = c->type[c->oc];
    a.id = c->id[c->oc];
    a.nn = c->nn;
    a.nbr = c->nbr;
    a.G = Gs;
    a.gE = gE;
    a.dx_aos = dx_aos;
    a.part = part;
    a.NP = NP;
    a.fl = c->dflags;
    cudaError_t e;
    switch (T) {
        case 1: e = launch_adj_t<1>(c, a); break;
        case 2: e = launch_adj_t<2>(c, a); break;
        case 4: e = launch_adj_t<4>(c, a); break;
        case 8: e = launch_adj_t<8>(c, a); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    k_adj_reduce<<<1, 256, 0, c->stream>>>(part, nwt, NP, totals_out);
    return cudaGetLastError();
}

size_t adjoint_scratch_doubles(md_ctx *c) {
    const int NP = 2 * c->hpair.nt * c->hpair.nt;
    const int64_t nwt = c->ns / (32 / c->T);
    return (size_t)(3 * c->ns + nwt * NP + NP);
}

}  // namespace mdb

// md_sort.cu -- the resort step: wrap, geometric binning, stable cell-order
// permutation and the gather of all per-atom state into the new order
// (paper, Section "Particle Sorting": sorting by geometric binning; the
// Introduction's timestep ends with "the particles are then resorted").
//
//   k_bin      : x = O + r (or raw input), wrap into [0, L), cell id, atomic
//                histogram; each atom takes a slot rank inside its cell.
//   k_scan_sum, k_scan_out : exclusive prefix sum of the per-cell counts
//                (block sums, then per-block scans), plus the per-build
//                bookkeeping (dangerous-build test, counter resets).
//   k_scatter  : atom -> slot (cell start + atomic rank).
//   k_segsort  : per cell, order the slots by prior index, which makes the
//                permutation stable: new order = sort by (cell, prior index).
//   k_permute  : gather r, v, type, id, image counts into the new order, with
//                r re-expressed relative to the new cell's centre and the FP32
//                shadow refreshed.
//
// Every FP64 operation that decides a cell or a wrapped coordinate is an
// explicitly rounded intrinsic (no FMA contraction), so the wrapped positions
// and cell ids are bit-identical to the textbook definition.
#include "md_common.cuh"

namespace mdb {
namespace {

__global__ void k_unpack(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                         int64_t ns, const double *__restrict__ x, const double *__restrict__ v,
                         const int32_t *__restrict__ types, double *__restrict__ xraw,
                         double *__restrict__ vout, int32_t *__restrict__ tout,
                         int32_t *__restrict__ idout, int32_t *__restrict__ imgout,
                         int32_t *__restrict__ cellc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const Box &B = boxes[tile_box[i >> 5]];
    int64_t loc = i - B.slot_off;
    if (loc < B.n) {
        int64_t g = B.atom_base + loc;
        for (int d = 0; d < 3; ++d) {
            if (x) xraw[d * ns + i] = x[3 * g + d];
            vout[d * ns + i] = v ? v[3 * g + d] : 0.0;
            imgout[d * ns + i] = 0;
        }
        tout[i] = types ? types[g] : 0;
        idout[i] = (int32_t)g;
    } else {
        for (int d = 0; d < 3; ++d) {
            if (x) xraw[d * ns + i] = 0.0;
            vout[d * ns + i] = 0.0;
            imgout[d * ns + i] = 0;
        }
        tout[i] = 0;
        idout[i] = -1;
    }
    cellc[i] = 0;
}

__global__ void k_bin(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                      const double *__restrict__ ctab, int64_t ns, int raw,
                      const double *__restrict__ r,
                      const double *__restrict__ xraw, const int32_t *__restrict__ cellc,
                      int32_t *__restrict__ img, const double *__restrict__ rbuild,
                      double *__restrict__ xw, int32_t *__restrict__ cell,
                      int32_t *__restrict__ rank, int32_t *__restrict__ count, Flags *fl) {
    if (fl->status & ST_FREEZE) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool live = i < ns;
    const Box &B = boxes[tile_box[(live ? i : 0) >> 5]];
    live = live && i - B.slot_off < B.n;
    float disp2 = 0.f;
    int32_t gc = -1;
    if (live) {
        double x[3];
        if (raw) {
            for (int d = 0; d < 3; ++d) x[d] = xraw[d * ns + i];
        } else {
            int cc[3];
            unpack_cell(cellc[i], cc[0], cc[1], cc[2]);
            for (int d = 0; d < 3; ++d) {
                const double rd = r[d * ns + i];
                x[d] = __dadd_rn(cell_centre(ctab, B, d, cc[d]), rd);
                const float dd = (float)(rd - rbuild[d * ns + i]);
                disp2 += dd * dd;
            }
        }
        if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]))) {
            atomicOr(&fl->status, ST_NONFINITE);
            live = false;
        } else {
            int c[3];
            for (int d = 0; d < 3; ++d) {
                const double L = B.L[d];
                double w;
                // 0 <= x < L by the bit patterns (non-negative doubles order as
                // integers; -0.0 takes the general rule, which gives +0.0)
                const long long xb = __double_as_longlong(x[d]);
                if (xb >= 0 && xb < __double_as_longlong(L)) {
                    // inside the box: the general rule below gives w = x, k = 0
                    // (x/L may round to 1, then w = (x - L) + L = x exactly);
                    // + 0.0 maps -0.0 to +0.0 as it does
                    w = __dadd_rn(x[d], 0.0);
                } else {
                    const double q = floor(__ddiv_rn(x[d], L));
                    w = __dsub_rn(x[d], __dmul_rn(L, q));
                    int k = (int)q;
                    if (w < 0.0) { w = __dadd_rn(w, L); k -= 1; }
                    if (w >= L) { w = __dsub_rn(w, L); k += 1; }
                    img[d * ns + i] += k;
                }
                xw[d * ns + i] = w;
                int cd = __double2int_rz(__dmul_rn(w, B.inv[d]));
                cd = cd < 0 ? 0 : (cd > B.nc[d] - 1 ? B.nc[d] - 1 : cd);
                c[d] = cd;
            }
            gc = B.cell_off + (c[2] * B.nc[1] + c[1]) * B.nc[0] + c[0];
        }
    }
    // Slot ranks inside each cell: one atomic per run of lanes with the same
    // cell (atoms still in the previous cell order mostly share cells).
    const unsigned grp = __match_any_sync(0xffffffffu, gc);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (live && lane == leader) base = atomicAdd(&count[gc], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (live) {
        cell[i] = gc;
        rank[i] = base + __popc(grp & ((1u << lane) - 1u));
    }
    if (!raw) {
        const unsigned m = __reduce_max_sync(0xffffffffu, live ? __float_as_uint(sqrtf(disp2)) : 0u);
        if (lane == 0 && m != 0u) atomicMax(&fl->maxdisp_bits, m);
    }
}

// Exclusive scan of count[0..ncell) into cstart[0..ncell] in two passes over
// blocks of kScanCells cells: block sums, then each block adds the sums of
// the blocks before it (in order) to its own scan.
constexpr int kScanThreads = 256, kScanPer = 4, kScanCells = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) k_scan_sum(const int32_t *__restrict__ count,
                                                           int32_t ncell, int32_t *__restrict__ part,
                                                           const Flags *fl) {
    if (fl->status & ST_FREEZE) return;
    __shared__ int32_t red[kScanThreads / 32];
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * kScanCells;
    int32_t s = 0;
    for (int k = 0; k < kScanPer; ++k) {
        const int c = c0 + k * kScanThreads + tid;
        if (c < ncell) s += count[c];
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        int32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_out(const int32_t *__restrict__ count,
                                                           int32_t *__restrict__ cstart,
                                                           int32_t ncell,
                                                           const int32_t *__restrict__ part,
                                                           Flags *fl, double half_skin, int raw) {
    if (fl->status & ST_FREEZE) return;
    __shared__ int32_t wsum[kScanThreads / 32];
    __shared__ int32_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // sums of the blocks before this one, in block order
    if (w == 0) {
        int32_t b = 0;
        for (int k = lane; k < (int)blockIdx.x; k += 32) b += part[k];
        b = __reduce_add_sync(0xffffffffu, b);
        if (lane == 0) s_base = b;
    }
    // this thread's kScanPer consecutive cells
    const int c0 = blockIdx.x * kScanCells + tid * kScanPer;
    int32_t v[kScanPer];
    int32_t s = 0;
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = c0 + k < ncell ? count[c0 + k] : 0;
        s += v[k];
    }
    int32_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int32_t before = s_base;
    for (int k = 0; k < w; ++k) before += wsum[k];
    int32_t run = before + incl - s;
    for (int k = 0; k < kScanPer; ++k) {
        if (c0 + k < ncell) cstart[c0 + k] = run;
        run += v[k];
    }
    // the grid's last thread has summed every cell (zeros past ncell)
    if (blockIdx.x == gridDim.x - 1 && tid == kScanThreads - 1) cstart[ncell] = run;
    if (blockIdx.x == 0 && tid == 0) {
        if (!raw && __uint_as_float(fl->maxdisp_bits) > (float)half_skin) fl->dangerous += 1;
        fl->builds += 1;
        fl->maxdisp_bits = 0u;
        fl->maxnn = 0;
        fl->sumnn = 0ull;
    }
}

__global__ void k_scatter(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                          int64_t ns, const int32_t *__restrict__ cell,
                          const int32_t *__restrict__ rank, const int32_t *__restrict__ cstart,
                          int32_t *__restrict__ ptmp, Flags *fl) {
    if (fl->status & ST_FREEZE) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const Box &B = boxes[tile_box[i >> 5]];
    if (i - B.slot_off >= B.n) return;
    int32_t c = cell[i];
    int64_t slot = B.slot_off + ((int64_t)cstart[c] - B.atom_base) + rank[i];
    if (chk_ok(slot, B.slot_off, (int64_t)B.slot_off + B.n, CHK_SORT_SCATTER, fl))
        ptmp[slot] = (int32_t)i;
}

// One warp per cell: rank each slot's prior index among the cell's slots.
__global__ void k_segsort(const Box *__restrict__ boxes, const int32_t *__restrict__ cell_box,
                          int32_t ncell, const int32_t *__restrict__ cstart,
                          const int32_t *__restrict__ ptmp, int32_t *__restrict__ perm,
                          const Flags *fl) {
    if (fl->status & ST_FREEZE) return;
    int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= ncell) return;
    const int32_t c = (int32_t)wg;
    const Box &B = boxes[cell_box[c]];
    const int32_t m = cstart[c + 1] - cstart[c];
    const int64_t s0 = B.slot_off + ((int64_t)cstart[c] - B.atom_base);
    for (int e = lane; e < m; e += 32) {
        int32_t val = ptmp[s0 + e];
        int32_t rk = 0;
        for (int u = 0; u < m; ++u) rk += (ptmp[s0 + u] < val);
        perm[s0 + rk] = val;
    }
}

__global__ void k_permute(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                          const double *__restrict__ ctab, int64_t ns,
                          const int32_t *__restrict__ perm,
                          const int32_t *__restrict__ cell, const double *__restrict__ xw,
                          const double *__restrict__ v_in, const int32_t *__restrict__ t_in,
                          const int32_t *__restrict__ id_in, const int32_t *__restrict__ img_in,
                          double *__restrict__ r_out, double *__restrict__ v_out,
                          int32_t *__restrict__ t_out, int32_t *__restrict__ id_out,
                          int32_t *__restrict__ img_out, int32_t *__restrict__ cellc_out,
                          const int32_t *__restrict__ cellc_in,
                          float4 *__restrict__ sh_out, double *__restrict__ rbuild,
                          double *__restrict__ xws, int32_t *__restrict__ nn, Flags *fl) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= ns) return;
    if (fl->status & ST_FREEZE) {
        // Frozen: keep the order; mirror the order-buffered arrays so the
        // buffer flip that follows every re-sort stays valid.
        for (int d = 0; d < 3; ++d) {
            v_out[d * ns + k] = v_in[d * ns + k];
            img_out[d * ns + k] = img_in[d * ns + k];
        }
        t_out[k] = t_in[k];
        id_out[k] = id_in[k];
        cellc_out[k] = cellc_in[k];
        return;
    }
    const Box &B = boxes[tile_box[k >> 5]];
    if (k - B.slot_off >= B.n) {
        for (int d = 0; d < 3; ++d) {
            r_out[d * ns + k] = 0.0;
            v_out[d * ns + k] = 0.0;
            img_out[d * ns + k] = 0;
            rbuild[d * ns + k] = 0.0;
            xws[d * ns + k] = 0.0;
        }
        t_out[k] = 0;
        id_out[k] = -1;
        cellc_out[k] = 0;
        sh_out[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        nn[k] = 0;
        return;
    }
    const int32_t old = (int32_t)(B.slot_off + chk_index((int64_t)perm[k] - B.slot_off, B.n,
                                                         CHK_SORT_PERMUTE, fl, k - B.slot_off));
    const int32_t loc = cell[old] - B.cell_off;
    const int cx = loc % B.nc[0], cy = (loc / B.nc[0]) % B.nc[1], cz = loc / (B.nc[0] * B.nc[1]);
    const int cc[3] = {cx, cy, cz};
    float s[3];
    for (int d = 0; d < 3; ++d) {
        double w = xw[d * ns + old];
        double rd = __dsub_rn(w, cell_centre(ctab, B, d, cc[d]));
        r_out[d * ns + k] = rd;
        rbuild[d * ns + k] = rd;
        xws[d * ns + k] = w;
        s[d] = __double2float_rn(rd);
        v_out[d * ns + k] = v_in[d * ns + old];
        img_out[d * ns + k] = img_in[d * ns + old];
    }
    const int32_t ty = t_in[old];
    t_out[k] = ty;
    id_out[k] = id_in[old];
    cellc_out[k] = pack_cell(cx, cy, cz);
    sh_out[k] = make_float4(s[0], s[1], s[2], __int_as_float(ty));
}

// Velocities by original id into the current slot order (md_set_state, once
// the new positions are sorted); padding slots keep their zeros.
__global__ void k_load_v(const Box *__restrict__ boxes, const int32_t *__restrict__ tile_box,
                         int64_t ns, const int32_t *__restrict__ id,
                         const double *__restrict__ v_aos, double *__restrict__ v) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const Box &B = boxes[tile_box[k >> 5]];
    if (k - B.slot_off >= B.n) return;
    const int64_t g = id[k];
    for (int d = 0; d < 3; ++d) v[d * ns + k] = v_aos[3 * g + d];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_load_velocities(md_ctx *c, const double *v_aos) {
    const int t = 256;
    k_load_v<<<blocks_for(c->ns, t), t, 0, c->stream>>>(c->dbox, c->tile_box, c->ns,
                                                        c->id[c->oc], v_aos, c->v[c->oc]);
    c->kernels += 1;
    return cudaGetLastError();
}

cudaError_t launch_unpack_input(md_ctx *c, const double *x_aos, const double *v_aos,
                                const int32_t *types) {
    const int t = 256;
    k_unpack<<<blocks_for(c->ns, t), t, 0, c->stream>>>(
        c->dbox, c->tile_box, c->ns, x_aos, v_aos, types, c->xraw, c->v[c->oc], c->type[c->oc],
        c->id[c->oc], c->img[c->oc], c->cellc[c->oc]);
    c->kernels += 1;
    return cudaGetLastError();
}

cudaError_t launch_bin_sort(md_ctx *c, bool raw_input) {
    const int t = 256;
    const int oc = c->oc, pc = c->pc;
    cudaError_t e = cudaMemsetAsync(c->count, 0, sizeof(int32_t) * (size_t)c->ncell_tot, c->stream);
    if (e != cudaSuccess) return e;
    k_bin<<<blocks_for(c->ns, t), t, 0, c->stream>>>(
        c->dbox, c->tile_box, c->ctab, c->ns, raw_input ? 1 : 0, c->r[pc], c->xraw, c->cellc[oc],
        c->img[oc], c->rbuild, c->xw, c->cell, c->rank, c->count, c->dflags);
    const unsigned nsb = blocks_for(c->ncell_tot, kScanCells);
    k_scan_sum<<<nsb, kScanThreads, 0, c->stream>>>(c->count, c->ncell_tot, c->scan_part,
                                                    c->dflags);
    k_scan_out<<<nsb, kScanThreads, 0, c->stream>>>(c->count, c->cstart, c->ncell_tot,
                                                    c->scan_part, c->dflags, c->hpair.half_skin,
                                                    raw_input ? 1 : 0);
    k_scatter<<<blocks_for(c->ns, t), t, 0, c->stream>>>(c->dbox, c->tile_box, c->ns, c->cell,
                                                          c->rank, c->cstart, c->ptmp,
                                                          c->dflags);
    k_segsort<<<blocks_for((int64_t)c->ncell_tot * 32, t), t, 0, c->stream>>>(
        c->dbox, c->cell_box, c->ncell_tot, c->cstart, c->ptmp, c->perm, c->dflags);
    k_permute<<<blocks_for(c->ns, t), t, 0, c->stream>>>(
        c->dbox, c->tile_box, c->ctab, c->ns, c->perm, c->cell, c->xw, c->v[oc], c->type[oc], c->id[oc],
        c->img[oc], c->r[pc], c->v[oc ^ 1], c->type[oc ^ 1], c->id[oc ^ 1], c->img[oc ^ 1],
        c->cellc[oc ^ 1], c->cellc[oc], c->sh[pc], c->rbuild, c->xws, c->nn, c->dflags);
    c->oc ^= 1;
    c->kernels += 6;
    return cudaGetLastError();
}

}  // namespace mdb

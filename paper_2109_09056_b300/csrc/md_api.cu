// md_api.cu -- the C ABI (include/md.h): context set-up, argument checks,
// host/device pointer handling, and the orchestration of the timestep
// (paper, Introduction / Fig. 1: neighbor list -> forces -> propagate ->
// resort; Fig. 4 re-expresses that step as library calls, one call per stage).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "md_common.cuh"
#include "md_trace.h"

using namespace mdb;

namespace {

thread_local std::string g_create_error;

const double kUnit[1] = {1.0};

md_status fail(md_ctx *c, md_status s, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

md_status timeout_fail(md_ctx *c) {
    return fail(c, MD_ERR_TIMEOUT, "a bounded device wait expired (a list copy did not complete)");
}

md_status cuda_fail(md_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? MD_ERR_NOMEM : MD_ERR_CUDA, m);
}

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

void free_all(md_ctx *c) {
    auto F = [](void *p) { if (p) cudaFree(p); };
    for (int k = 0; k < 2; ++k) {
        F(c->r[k]); F(c->v[k]); F(c->sh[k]); F(c->type[k]); F(c->id[k]); F(c->img[k]); F(c->cellc[k]);
    }
    F(c->f); F(c->rbuild); F(c->xw); F(c->xws); F(c->xraw);
    F(c->cell); F(c->rank); F(c->perm); F(c->ptmp); F(c->count); F(c->cstart); F(c->nn);
    F(c->nbr); F(c->dbox); F(c->tile_box); F(c->cell_box); F(c->dpair); F(c->dflags);
    F(c->tpart); F(c->tbox); F(c->fpart); F(c->tlog); F(c->dscratch); F(c->stage);
    F(c->restage); F(c->scan_part); F(c->ctab); F(c->facc); F(c->facc64); F(c->shv);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->htbox) cudaFreeHost(c->htbox);
    for (auto &g : c->gexec)
        if (g) cudaGraphExecDestroy(g);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->ev_main) cudaEventDestroy(c->ev_main);
    if (c->ev_side) cudaEventDestroy(c->ev_side);
    if (c->side) cudaStreamDestroy(c->side);
}

void* stage_buffer(md_ctx *c, size_t bytes) {
    if (bytes > c->stage_bytes) {
        if (c->stage) cudaFree(c->stage);
        c->stage = nullptr;
        c->stage_bytes = 0;
        if (cudaMalloc(&c->stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c->stage_bytes = bytes;
    }
    return c->stage;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Pad after an overflow that needed `maxnn` slots: with an automatic pad, 15%
// + 16 slack; with an explicit md_params.neigh_pad, just enough (rounded to 8).
int grown_pad(const md_ctx *c, int maxnn) {
    return c->params.neigh_pad > 0 ? maxnn : (int)(maxnn * 1.05) + 8;
}

void invalidate_graphs(md_ctx *c) {
    for (auto &g : c->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Pair tables, validated.
md_status setup_pair(md_ctx *c, const double *eps, const double *sigma) {
    const md_params &p = c->params;
    const int nt = p.ntypes;
    Pair &P = c->hpair;
    std::memset(&P, 0, sizeof(P));
    P.nt = nt;
    P.shift = p.shift_energy ? 1 : 0;
    P.rc2 = p.rc * p.rc;
    const double rs = p.rc + p.skin;
    P.rs2 = rs * rs;
    P.dt = p.dt;
    P.half_skin = 0.5 * p.skin;
    P.rc2f = (float)P.rc2;
    P.rs2f = (float)P.rs2;
    P.bandf = (float)(3e-5 * P.rs2);  // > 3.9x the FP32 r^2 error bound (md_neigh.cu)
    c->eps.assign(eps, eps + nt * nt);
    c->sigma.assign(sigma, sigma + nt * nt);
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nt; ++b) {
            const int ab = a * nt + b;
            const double e = eps[ab], s = sigma[ab];
            if (!(std::isfinite(e) && std::isfinite(s) && s > 0.0 && e >= 0.0) ||
                e != eps[b * nt + a] || s != sigma[b * nt + a])
                return fail(c, MD_ERR_ARG, "eps/sigma must be finite, sigma > 0, eps >= 0, symmetric");
            P.eps[ab] = e;
            P.sig[ab] = s;
            P.e24[ab] = 24.0 * e;
            P.s2[ab] = s * s;
            P.e4[ab] = 4.0 * e;
            if (P.shift) {
                const double c2 = (s * s) / P.rc2, c6 = c2 * c2 * c2;
                P.ush[ab] = 4.0 * e * (c6 * c6 - c6);
            }
            P.fs2[ab] = (float)P.s2[ab];
            P.fe4[ab] = (float)P.e4[ab];
            P.fush[ab] = (float)P.ush[ab];
            P.fc1[ab] = (float)(P.e24[ab] / P.s2[ab]);
        }
    for (int a = 0; a < nt; ++a) {
        P.mass[a] = c->mass[a];
        P.dtm[a] = p.dt / c->mass[a];
        P.hdtm[a] = 0.5 * p.dt / c->mass[a];
    }
    return MD_OK;
}

md_status alloc_list(md_ctx *c, int pad) {
    // a multiple of 4 T keeps R = pad / T a multiple of the force kernel's
    // 4-entry batch
    c->pad = round_up(pad, std::max(8, MD_FORCE_BATCH * c->T));
    c->R = c->pad / c->T;
    const size_t words = (size_t)c->ns * c->pad;
    if (words > c->nbr_words) {
        if (c->nbr) cudaFree(c->nbr);
        c->nbr = nullptr;
        c->nbr_words = 0;
        CK(dalloc(&c->nbr, words));
        c->nbr_words = words;
    }
    CK(fill_list_sentinel(c));
    invalidate_graphs(c);
    c->list_valid = false;
    return MD_OK;
}

md_status read_flags(md_ctx *c) {
    CK(cudaMemcpyAsync(c->hflags, c->dflags, sizeof(Flags), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->hflags->check_site != CHK_NONE) {
        // only a checked build (-DMD_CHECKED) records these
        static const char *const names[CHK_SITES] = {
            "none", "sort scatter", "sort permute", "build home atom", "build candidate",
            "mixed force gather", "FP64 force gather", "adjoint gather", "SPME real-space gather"};
        const uint32_t k = c->hflags->check_site;
        return fail(c, MD_ERR_CUDA,
                    std::string("index check failed: ") + (k < CHK_SITES ? names[k] : "?") +
                        " (index " + std::to_string(c->hflags->check_index) + ")");
    }
    return MD_OK;
}

md_status clear_status(md_ctx *c) {
    CK(cudaMemsetAsync(&c->dflags->status, 0, sizeof(uint32_t), c->stream));
    return MD_OK;
}

// Build the list; on overflow grow the pad and rebuild (state must be sorted).
md_status build_with_retry(md_ctx *c) {
    for (int attempt = 0; attempt < 8; ++attempt) {
        CK(launch_build(c));
        md_status s = read_flags(c);
        if (s) return s;
        if (c->hflags->status & ST_NONFINITE) return fail(c, MD_ERR_NONFINITE, "non-finite position");
        if (!(c->hflags->status & ST_OVERFLOW)) {
            c->list_valid = true;
            return MD_OK;
        }
        s = clear_status(c);
        if (s) return s;
        s = alloc_list(c, grown_pad(c, c->hflags->maxnn));
        if (s) return s;
    }
    return fail(c, MD_ERR_NEIGH_OVERFLOW, "neighbor list kept overflowing");
}

md_status sort_build(md_ctx *c, bool raw) {
    CK(launch_bin_sort(c, raw));
    c->sorted_at = c->step;
    c->built_at = c->step;
    return build_with_retry(c);
}

// Forces (and thermo) of a freshly sorted and listed state.
md_status forces_at_build(md_ctx *c) {
    CK(launch_force(c, MODE_FORCE_ONLY));
    CK(launch_finalize(c, MODE_FORCE_ONLY));
    md_status s = read_flags(c);
    if (s) return s;
    if (c->hflags->status & ST_TIMEOUT) return timeout_fail(c);
    if (c->hflags->status & ST_NONFINITE) return fail(c, MD_ERR_NONFINITE, "non-finite position");
    c->forces_valid = true;
    c->ready = true;
    return MD_OK;
}

md_status sort_build_forces(md_ctx *c, bool raw) {
    md_status s = sort_build(c, raw);
    if (s) return s;
    return forces_at_build(c);
}

void fill_thermo(md_ctx *c, int b, md_thermo *t) {
    const double *tb = c->htbox + b * TB;
    std::memset(t, 0, sizeof(*t));
    t->step = c->step;
    t->pe = tb[0];
    t->ke = tb[1];
    t->etot = tb[0] + tb[1];
    const int64_t n = c->hbox[b].n;
    t->temperature = n > 1 ? 2.0 * tb[1] / (3.0 * (double)n - 3.0) : 0.0;
    t->momentum[0] = tb[2];
    t->momentum[1] = tb[3];
    t->momentum[2] = tb[4];
    t->max_displacement = tb[5];
    t->nn_max = c->hflags->maxnn;
    t->pad = c->pad;
    t->builds = c->hflags->builds;
    t->dangerous_builds = c->hflags->dangerous;
}

md_status pull_thermo(md_ctx *c) {
    CK(cudaMemcpyAsync(c->htbox, c->tbox, sizeof(double) * TB * c->nbox, cudaMemcpyDeviceToHost,
                       c->stream));
    return read_flags(c);
}

md_status ensure_forces(md_ctx *c) {
    if (c->forces_valid && c->ready) return MD_OK;
    if (!c->ready) return fail(c, MD_ERR_ARG, "internal: state between half-steps");
    if (!c->list_valid) {
        md_status s = build_with_retry(c);
        if (s) return s;
    }
    CK(launch_force(c, MODE_FORCE_ONLY));
    CK(launch_finalize(c, MODE_FORCE_ONLY));
    md_status s = read_flags(c);
    if (s) return s;
    c->forces_valid = true;
    return MD_OK;
}

md_status init_ctx(md_ctx *c, int32_t nbox, const int64_t *n_per_box, const md_box *boxes,
                   const md_params *params, void *stream) {
    if (!params || !boxes || !n_per_box || nbox < 1) return fail(c, MD_ERR_ARG, "NULL argument");
    c->params = *params;
    md_params &p = c->params;
    if (p.ntypes < 1 || p.ntypes > MD_MAXT) return fail(c, MD_ERR_ARG, "ntypes must be 1..8");
    if (!p.eps || !p.sigma || !p.mass) return fail(c, MD_ERR_ARG, "eps/sigma/mass NULL");
    if (!(p.rc > 0.0) || !(p.skin >= 0.0) || !(p.dt > 0.0) || !std::isfinite(p.rc + p.skin + p.dt))
        return fail(c, MD_ERR_ARG, "rc, skin, dt must be positive and finite");
    if (p.rebuild_every < 1) return fail(c, MD_ERR_ARG, "rebuild_every must be >= 1");
    if (p.precision != MD_FP64 && p.precision != MD_MIXED) return fail(c, MD_ERR_ARG, "precision");
    c->mass.assign(p.mass, p.mass + p.ntypes);
    for (double m : c->mass)
        if (!(m > 0.0) || !std::isfinite(m)) return fail(c, MD_ERR_ARG, "mass must be > 0");
    c->T = p.lanes_per_atom ? p.lanes_per_atom : 4;  // automatic: see below for FP64
    if (c->T != 1 && c->T != 2 && c->T != 4 && c->T != 8)
        return fail(c, MD_ERR_ARG, "lanes_per_atom must be 1, 2, 4 or 8");
    if (p.half_list && c->T != 4)
        return fail(c, MD_ERR_ARG, "half_list needs 4 lanes per atom");
    if (p.shadow_vl != 0 && ((p.shadow_vl != 8 && p.shadow_vl != 32) || p.precision != MD_MIXED ||
                             c->T != 4 || p.half_list))
        return fail(c, MD_ERR_ARG, "shadow_vl must be 0, or 8 or 32 with MD_MIXED, 4 lanes, full lists");
    c->block = p.block_threads;  // 0: chosen per launch (md_force.cu)
    if (c->block != 0 && (c->block < 64 || c->block > 768 || c->block % 32))
        return fail(c, MD_ERR_ARG, "block_threads must be 0 or 64..768, a multiple of 32");
    md_status s = setup_pair(c, p.eps, p.sigma);
    if (s) return s;
    c->stream = static_cast<cudaStream_t>(stream);
    c->nbox = nbox;
    const double rs = p.rc + p.skin;
    int64_t slot = 0, base = 0;
    int64_t cells = 0;
    double max_rho = 0.0;
    c->hbox.resize(nbox);
    for (int b = 0; b < nbox; ++b) {
        Box &B = c->hbox[b];
        std::memset(&B, 0, sizeof(B));
        if (n_per_box[b] < 1) return fail(c, MD_ERR_ARG, "every box needs n >= 1");
        for (int d = 0; d < 3; ++d) {
            const double L = boxes[b].L[d];
            if (!std::isfinite(L) || !(L > 2.0 * rs))
                return fail(c, MD_ERR_BOX_TOO_SMALL, "box edge must exceed 2*(rc+skin)");
            B.L[d] = L;
            B.nc[d] = (int32_t)std::floor(L / rs);
            if (B.nc[d] > 1023) return fail(c, MD_ERR_ARG, "more than 1023 cells along an axis");
            B.h[d] = L / B.nc[d];
            B.inv[d] = (double)B.nc[d] / L;
            B.hf[d] = (float)B.h[d];
        }
        B.ncell = B.nc[0] * B.nc[1] * B.nc[2];
        B.cell_off = (int32_t)cells;
        cells += B.ncell;
        B.n = (int32_t)n_per_box[b];
        B.npad = round_up(B.n, 32);
        B.slot_off = (int32_t)slot;
        B.atom_base = base;
        slot += B.npad;
        base += B.n;
        const double rho = B.n / (B.L[0] * B.L[1] * B.L[2]);
        if (rho > max_rho) max_rho = rho;
    }
    if (slot >= (int64_t)MD_IDX_MASK || cells > INT32_MAX / 2)
        return fail(c, MD_ERR_ARG, "too many atoms or cells for one context");
    c->ns = slot;
    c->n_total = base;
    c->ncell_tot = (int32_t)cells;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev));
    // Automatic lanes per atom for FP64 contexts: the FP64 pass loops over the
    // longest per-lane count of entries within rc, which long single-lane rows
    // balance best, once there are atoms enough for many waves of 32-atom warps
    // (B300: 4M atoms 2.98e8 atom-steps/s at 1 lane vs 2.86e8 at 4; 131k atoms
    // 2.44e8 vs 2.71e8, 4,000 atoms 2.6e7 vs 7.8e7).
    if (!p.lanes_per_atom && p.precision == MD_FP64 && !p.half_list && c->n_total >= 8192LL * c->nsm)
        c->T = 1;

    const size_t ns = (size_t)c->ns;
    for (int k = 0; k < 2; ++k) {
        CK(dalloc(&c->r[k], 3 * ns));
        CK(dalloc(&c->v[k], 3 * ns));
        CK(dalloc(&c->sh[k], ns + 1));   // slot ns: the dummy the sentinel entry points at
        // slot ns: type 0 for the sentinel entry (read by whole-batch gathers)
        CK(dalloc(&c->type[k], ns + 1));
        CK(cudaMemset(c->type[k], 0, (ns + 1) * sizeof(int32_t)));
        CK(dalloc(&c->id[k], ns));
        CK(dalloc(&c->img[k], 3 * ns));
        CK(dalloc(&c->cellc[k], ns));
        CK(cudaMemset(c->r[k], 0, 3 * ns * sizeof(double)));
        CK(cudaMemset(c->sh[k], 0, ns * sizeof(float4)));
        const float4 far = make_float4(1e4f, 1e4f, 1e4f, 0.f);
        CK(cudaMemcpy(c->sh[k] + ns, &far, sizeof(float4), cudaMemcpyHostToDevice));
    }
    CK(dalloc(&c->f, 3 * ns));
    CK(cudaMemset(c->f, 0, 3 * ns * sizeof(double)));
    if (p.shadow_vl) {
        const size_t blocks = (ns + 1 + p.shadow_vl - 1) / p.shadow_vl;
        CK(dalloc(&c->shv, blocks * 4 * (size_t)p.shadow_vl));
    }
    if (p.half_list && p.precision == MD_MIXED) {  // kept at zero between force evaluations
        CK(dalloc(&c->facc, ns + 1));
        CK(cudaMemset(c->facc, 0, (ns + 1) * sizeof(float4)));
    }
    if (p.half_list && p.precision == MD_FP64) {
        CK(dalloc(&c->facc64, 4 * (ns + 1)));
        CK(cudaMemset(c->facc64, 0, 4 * (ns + 1) * sizeof(double)));
    }
    CK(dalloc(&c->rbuild, 3 * ns));
    CK(dalloc(&c->xw, 3 * ns));
    CK(dalloc(&c->xws, 3 * ns));
    CK(dalloc(&c->xraw, 3 * ns));
    CK(dalloc(&c->cell, ns));
    CK(dalloc(&c->rank, ns));
    CK(dalloc(&c->perm, ns));
    CK(dalloc(&c->ptmp, ns));
    CK(dalloc(&c->nn, ns));
    CK(cudaMemset(c->nn, 0, ns * sizeof(int32_t)));
    CK(dalloc(&c->count, (size_t)c->ncell_tot));
    CK(cudaMemset(c->count, 0, (size_t)c->ncell_tot * sizeof(int32_t)));
    CK(dalloc(&c->cstart, (size_t)c->ncell_tot + 1));
    CK(dalloc(&c->scan_part, (size_t)c->ncell_tot / 1024 + 1));
    // cell centres (c + 1/2) h per box and axis, rounded as the device would
    std::vector<double> ctab;
    for (int b = 0; b < nbox; ++b) {
        Box &B = c->hbox[b];
        B.ctab = (int32_t)ctab.size();
        for (int d = 0; d < 3; ++d)
            for (int k = 0; k < B.nc[d]; ++k) ctab.push_back(((double)k + 0.5) * B.h[d]);
    }
    CK(dalloc(&c->ctab, ctab.size()));
    CK(cudaMemcpy(c->ctab, ctab.data(), sizeof(double) * ctab.size(), cudaMemcpyHostToDevice));
    CK(dalloc(&c->dbox, (size_t)nbox));
    CK(cudaMemcpy(c->dbox, c->hbox.data(), sizeof(Box) * nbox, cudaMemcpyHostToDevice));
    std::vector<int32_t> tb(ns / 32), cb((size_t)c->ncell_tot);
    for (int b = 0; b < nbox; ++b) {
        const Box &B = c->hbox[b];
        for (int t = 0; t < B.npad / 32; ++t) tb[B.slot_off / 32 + t] = b;
        for (int k = 0; k < B.ncell; ++k) cb[B.cell_off + k] = b;
    }
    CK(dalloc(&c->tile_box, tb.size()));
    CK(cudaMemcpy(c->tile_box, tb.data(), tb.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(dalloc(&c->cell_box, cb.size()));
    CK(cudaMemcpy(c->cell_box, cb.data(), cb.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(dalloc(&c->dpair, 1));
    CK(cudaMemcpy(c->dpair, &c->hpair, sizeof(Pair), cudaMemcpyHostToDevice));
    CK(dalloc(&c->dflags, 1));
    CK(cudaMemset(c->dflags, 0, sizeof(Flags)));
    CK(dalloc(&c->tpart, ns * TP));  // enough for T = 1 (one warp-tile per 32 slots ... ns/A tiles)
    CK(dalloc(&c->tbox, (size_t)nbox * TB));
    {
        // first-level thermo CTAs per box: ~2048 warp-tiles each, 1..64
        int64_t maxslots = 0;
        for (const Box &B : c->hbox) maxslots = std::max<int64_t>(maxslots, B.npad);
        c->fsplit = (int)std::min<int64_t>(64, std::max<int64_t>(1, maxslots / 8 / 2048));
        CK(dalloc(&c->fpart, (size_t)nbox * c->fsplit * 6));
    }
    CK(cudaMemset(c->tbox, 0, sizeof(double) * TB * nbox));
    c->tlog_cap = 4096;
    CK(dalloc(&c->tlog, (size_t)c->tlog_cap * 4));
    CK(cudaMemset(c->tlog, 0, sizeof(double) * 4 * c->tlog_cap));
    CK(cudaMallocHost(reinterpret_cast<void **>(&c->hflags), sizeof(Flags)));
    CK(cudaMallocHost(reinterpret_cast<void **>(&c->htbox), sizeof(double) * TB * nbox));
    std::memset(c->htbox, 0, sizeof(double) * TB * nbox);
    // list pad: observed rows in an LJ liquid stay within ~1.3x the mean count
    int pad = p.neigh_pad;
    if (pad <= 0) {
        const double mean = 4.18879020478639 * rs * rs * rs * max_rho * (p.half_list ? 0.5 : 1.0);
        pad = (int)(1.15 * mean) + 8;
    }
    return alloc_list(c, pad);
}

const void *dev_input(md_ctx *c, const void *p, size_t bytes, size_t stage_off, md_status *st) {
    *st = MD_OK;
    if (!p) return nullptr;
    if (is_device_ptr(p)) return p;
    char *s = static_cast<char *>(stage_buffer(c, stage_off + bytes));
    if (!s) {
        *st = fail(c, MD_ERR_NOMEM, "staging allocation failed");
        return nullptr;
    }
    cudaError_t e = cudaMemcpyAsync(s + stage_off, p, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
        *st = cuda_fail(c, e, "cudaMemcpyAsync H2D");
        return nullptr;
    }
    return s + stage_off;
}

// Host velocities (n x 3) into their place in the staging buffer on the side
// stream, ordered after the work already on the context's stream; ev_side
// marks the copy's end.
md_status copy_velocities_beside(md_ctx *c, const double *v, const double **vdev) {
    const size_t n = (size_t)c->n_total;
    char *st = static_cast<char *>(stage_buffer(c, 6 * n * sizeof(double) + n * sizeof(int32_t)));
    if (!st) return fail(c, MD_ERR_NOMEM, "staging allocation failed");
    if (!c->side) {
        CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->ev_main, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_side, cudaEventDisableTiming));
    }
    double *dst = reinterpret_cast<double *>(st) + 3 * n;
    CK(cudaEventRecord(c->ev_main, c->stream));
    CK(cudaStreamWaitEvent(c->side, c->ev_main, 0));
    CK(cudaMemcpyAsync(dst, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->side));
    CK(cudaEventRecord(c->ev_side, c->side));
    *vdev = dst;
    return MD_OK;
}

// `types` from the caller are range-checked; the context's own (md_set_state
// reloading the current types) are not.
md_status load_state(md_ctx *c, const double *x, const double *v, const int32_t *types,
                     bool check_types = true) {
    const size_t n = (size_t)c->n_total;
    md_status st;
    // stage layout: x | v | types (host inputs only); sized once so that no
    // later request reallocates under an earlier copy
    if (!stage_buffer(c, 6 * n * sizeof(double) + n * sizeof(int32_t)))
        return fail(c, MD_ERR_NOMEM, "staging allocation failed");
    const void *dx = dev_input(c, x, 3 * n * sizeof(double), 0, &st);
    if (st) return st;
    const void *dv = dev_input(c, v, 3 * n * sizeof(double), 3 * n * sizeof(double), &st);
    if (st) return st;
    const void *dt = dev_input(c, types, n * sizeof(int32_t), 6 * n * sizeof(double), &st);
    if (st) return st;
    if (types && check_types) {
        std::vector<int32_t> h(n);
        if (is_device_ptr(types)) {
            CK(cudaMemcpy(h.data(), types, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(h.data(), types, n * sizeof(int32_t));
        }
        for (int32_t t : h)
            if (t < 0 || t >= c->params.ntypes) return fail(c, MD_ERR_ARG, "atom type out of range");
    }
    CK(launch_unpack_input(c, static_cast<const double *>(dx), static_cast<const double *>(dv),
                           static_cast<const int32_t *>(dt)));
    return MD_OK;
}

md_status create_common(md_ctx *c, const double *x, const double *v, const int32_t *types) {
    md_status s = load_state(c, x, v, types);
    if (s) return s;
    c->step = 0;
    s = sort_build_forces(c, true);
    if (s) return s;
    return pull_thermo(c);
}

// Output helper: device pointers are written directly; host pointers go
// through the staging buffer.
struct OutBuf {
    void *user;
    void *dev;
    size_t bytes;
};

}  // namespace

namespace mdb {
// For solvers attached to a context (md_spme.cu): the list guarantee that
// md_compute_forces gives (build it if the context has none), failures
// reported in c->err.
md_status ensure_list(md_ctx *c) {
    if (!c->ready) return fail(c, MD_ERR_ARG, "internal: state between half-steps");
    if (c->list_valid) return MD_OK;
    return build_with_retry(c);
}
bool is_device_pointer(const void *p) { return is_device_ptr(p); }
// Re-sort the drifted state into cells and rebuild the list (pad grown on
// overflow), as md_step does at a rebuild step; c->step is the step of the state.
md_status resort_and_build(md_ctx *c) {
    md_status s = sort_build(c, false);
    if (s) return s;
    if (c->hflags->status & ST_TIMEOUT) return timeout_fail(c);
    c->list_valid = true;
    return MD_OK;
}
// Read the device flags and turn a frozen state into its status.
md_status check_run_flags(md_ctx *c) {
    md_status s = read_flags(c);
    if (s) return s;
    const uint32_t st = c->hflags->status;
    if (st & ST_TIMEOUT) return timeout_fail(c);
    if (st & ST_NONFINITE) return fail(c, MD_ERR_NONFINITE, "non-finite position");
    if (st & ST_OVERFLOW) return fail(c, MD_ERR_NEIGH_OVERFLOW, "a list row overflowed");
    return MD_OK;
}
}  // namespace mdb

md_status mdb::set_global_error(md_status s, const std::string &msg) {
    g_create_error = msg;
    return s;
}

// With profiling on, `launch` is bracketed by a pair of CUDA events tagged
// 0 (force), 1 (re-sort) or 2 (list build).
template <typename F>
static md_status record_timed(md_ctx *c, int tag, F &&launch) {
    if (!c->prof) {
        CK(launch());
        return MD_OK;
    }
    if (c->ev_used + 2 > c->ev_pool.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->ev_pool.push_back(e);
        }
    }
    cudaEvent_t e0 = c->ev_pool[c->ev_used], e1 = c->ev_pool[c->ev_used + 1];
    c->ev_tag.resize(c->ev_used / 2 + 1);
    c->ev_tag[c->ev_used / 2] = tag;
    c->ev_used += 2;
    CK(cudaEventRecord(e0, c->stream));
    CK(launch());
    CK(cudaEventRecord(e1, c->stream));
    return MD_OK;
}

static md_status record_force(md_ctx *c, int mode) {
    return record_timed(c, 0, [&] { return launch_force(c, mode); });
}

extern "C" {

void md_params_default(md_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->ntypes = 1;
    p->eps = kUnit;
    p->sigma = kUnit;
    p->mass = kUnit;
    p->rc = 2.5;
    p->skin = 0.3;
    p->dt = 0.005;
    p->rebuild_every = 20;
    p->precision = MD_MIXED;
    p->use_graphs = 1;
}

md_status md_batch_create(int32_t nbox, const int64_t *n_per_box, const md_box *boxes,
                          const double *x, const double *v, const int32_t *types,
                          const md_params *params, void *stream, md_ctx **out) {
    MD_TRACE("md_batch_create");
    if (out) *out = nullptr;
    if (!out || !x) return fail(nullptr, MD_ERR_ARG, "NULL argument");
    md_ctx *c = new (std::nothrow) md_ctx();
    if (!c) return fail(nullptr, MD_ERR_NOMEM, "host allocation failed");
    md_status s = init_ctx(c, nbox, n_per_box, boxes, params, stream);
    if (s == MD_OK) s = create_common(c, x, v, types);
    if (s != MD_OK) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        cudaGetLastError();   // a failed allocation's error is reported, not left pending
        return s;
    }
    *out = c;
    return MD_OK;
}

md_status md_create(const md_box *box, int64_t n, const double *x, const double *v,
                    const int32_t *types, const md_params *params, void *stream, md_ctx **out) {
    if (n < 1) {
        if (out) *out = nullptr;
        return fail(nullptr, MD_ERR_ARG, "n must be >= 1");
    }
    return md_batch_create(1, &n, box, x, v, types, params, stream, out);
}

md_status md_bin_sort(md_ctx *c) {
    MD_TRACE("md_bin_sort");
    if (!c) return MD_ERR_ARG;
    if (!c->ready) return fail(c, MD_ERR_ARG, "internal: state between half-steps");
    CK(launch_bin_sort(c, false));
    md_status s = read_flags(c);
    if (s) return s;
    if (c->hflags->status & ST_TIMEOUT) return timeout_fail(c);
    if (c->hflags->status & ST_NONFINITE) return fail(c, MD_ERR_NONFINITE, "non-finite position");
    c->sorted_at = c->step;
    c->built_at = -1;
    c->list_valid = false;
    c->forces_valid = false;
    invalidate_graphs(c);
    return MD_OK;
}

md_status md_build_neighbors(md_ctx *c) {
    MD_TRACE("md_build_neighbors");
    if (!c) return MD_ERR_ARG;
    if (c->sorted_at != c->step) {
        // the atoms moved since their cells were assigned: re-sort first, so
        // every neighbor lies in the 27 cells around an atom's cell
        md_status s = md_bin_sort(c);
        if (s) return s;
    }
    CK(launch_build(c));
    md_status s = read_flags(c);
    if (s) return s;
    if (c->hflags->status & ST_OVERFLOW) {
        const int need = c->hflags->maxnn;
        s = clear_status(c);
        if (s) return s;
        s = alloc_list(c, grown_pad(c, need));
        if (s) return s;
        return fail(c, MD_ERR_NEIGH_OVERFLOW,
                    "a list row needs " + std::to_string(need) + " slots; pad grown, call again");
    }
    c->list_valid = true;
    c->built_at = c->step;
    c->forces_valid = false;
    return MD_OK;
}

md_status md_compute_forces(md_ctx *c, double *energy_out) {
    MD_TRACE("md_compute_forces");
    if (!c) return MD_ERR_ARG;
    if (!c->ready) return fail(c, MD_ERR_ARG, "internal: state between half-steps");
    if (!c->list_valid) {
        md_status s = build_with_retry(c);
        if (s) return s;
    }
    CK(launch_force(c, MODE_FORCE_ONLY));
    CK(launch_finalize(c, MODE_FORCE_ONLY));
    md_status s = pull_thermo(c);
    if (s) return s;
    c->forces_valid = true;
    if (energy_out) {
        double e = 0.0;
        for (int b = 0; b < c->nbox; ++b) e += c->htbox[b * TB + 0];
        *energy_out = e;
    }
    return MD_OK;
}

static md_status flush_profile_events(md_ctx *c) {
    if (c->ev_used == 0) return MD_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev_pool[k], c->ev_pool[k + 1]));
        switch (c->ev_tag[k / 2]) {
            case 0: c->prof_ms += ms; c->prof_launches += 1; break;
            case 1: c->prof_sort_ms += ms; c->prof_rebuilds += 1; break;
            default: c->prof_build_ms += ms; break;
        }
    }
    c->ev_used = 0;
    return MD_OK;
}

static bool thermo_step(const md_ctx *c, int64_t n) {
    return c->params.thermo_every > 0 && n % c->params.thermo_every == 0;
}

// Steps n .. n + every - 1 (all FUSED), n a rebuild step, captured once per
// buffer parity and replayed.
static md_status run_period_graph(md_ctx *c) {
    const int key = c->pc * 2 + c->oc;
    const int every = c->params.rebuild_every;
    const int pc0 = c->pc, oc0 = c->oc;
    const int64_t k0 = c->kernels;
    if (!c->gexec[key]) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_bin_sort(c, false);
        if (e == cudaSuccess) e = launch_build(c);
        for (int k = 0; k < every && e == cudaSuccess; ++k) {
            e = launch_force(c, MODE_FUSED);
            if (e == cudaSuccess) e = launch_finalize(c, MODE_FUSED);
        }
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
        if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->gexec[key], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec[key] = nullptr;
            return cuda_fail(c, e, "cudaGraphInstantiate");
        }
        // capture recorded the parity changes; restore and replay below
        c->pc = pc0;
        c->oc = oc0;
        c->graph_nk[key] = c->kernels - k0;
        c->kernels = k0;
    }
    CK(cudaGraphLaunch(c->gexec[key], c->stream));
    c->kernels += c->graph_nk[key];
    c->oc ^= 1;
    if (every % 2) c->pc ^= 1;
    return MD_OK;
}

md_status md_step(md_ctx *c, int32_t nsteps, md_thermo *last_out) {
    MD_TRACE("md_step");
    if (!c) return MD_ERR_ARG;
    if (nsteps < 0) return fail(c, MD_ERR_ARG, "nsteps must be >= 0");
    md_status s;
    if (c->ready) {
        s = ensure_forces(c);
        if (s) return s;
    }
    const int every = c->params.rebuild_every;
    const int64_t target = c->step + (c->ready ? nsteps : nsteps);
    const bool graphs = c->params.use_graphs && c->stream != nullptr && !c->prof;
    for (int recover = 0; recover < 8; ++recover) {
        int64_t n;
        if (c->ready) {
            if (c->step >= target) break;
            CK(launch_kick_drift(c));
            c->ready = false;
            c->forces_valid = false;
            n = c->step + 1;
        } else {
            n = c->step;
        }
        while (n <= target) {
            if (graphs && n % every == 0 && c->built_at != n && n + every <= target &&
                c->list_valid) {
                s = run_period_graph(c);
                if (s) return s;
                c->sorted_at = n;
                c->built_at = n;
                n += every;
                continue;
            }
            if (n % every == 0 && c->built_at != n) {
                s = record_timed(c, 1, [&] { return launch_bin_sort(c, false); });
                if (s) return s;
                s = record_timed(c, 2, [&] { return launch_build(c); });
                if (s) return s;
                c->sorted_at = n;
                c->built_at = n;
                c->list_valid = true;
            }
            const int mode = n == target ? MODE_FINAL : MODE_FUSED;
            s = record_force(c, mode);
            if (s) return s;
            if (mode == MODE_FINAL || thermo_step(c, n)) CK(launch_finalize(c, mode));
            if (mode == MODE_FINAL) break;
            ++n;
        }
        s = read_flags(c);
        if (s) return s;
        if (c->prof) {
            s = flush_profile_events(c);
            if (s) return s;
        }
        const uint32_t st = c->hflags->status;
        if (st & ST_TIMEOUT) return timeout_fail(c);
        if (st & ST_NONFINITE) return fail(c, MD_ERR_NONFINITE, "non-finite position during md_step");
        if (!(st & ST_OVERFLOW)) {
            c->step = target;
            c->ready = true;
            c->forces_valid = true;
            break;
        }
        // A list overflowed at step clock: the state is sorted and drifted to
        // that step; grow the pad, rebuild the list there and resume.
        const int64_t nf = c->hflags->clock;
        s = clear_status(c);
        if (s) return s;
        s = alloc_list(c, grown_pad(c, c->hflags->maxnn));
        if (s) return s;
        s = build_with_retry(c);
        if (s) return s;
        c->built_at = nf;
        c->step = nf;
        c->ready = false;
        if (recover == 7) return fail(c, MD_ERR_NEIGH_OVERFLOW, "list kept overflowing in md_step");
    }
    s = pull_thermo(c);
    if (s) return s;
    if (last_out) fill_thermo(c, 0, last_out);
    if (c->params.check_displacement && c->hflags->dangerous > 0)
        return fail(c, MD_ERR_DANGEROUS_BUILD, "an atom moved more than skin/2 between builds");
    return MD_OK;
}

md_status md_get_state(md_ctx *c, double *x, double *v, double *f, int32_t *img, int32_t *ids) {
    MD_TRACE("md_get_state");
    if (!c) return MD_ERR_ARG;
    if (f) {
        md_status s = ensure_forces(c);
        if (s) return s;
    }
    const size_t n = (size_t)c->n_total;
    const size_t b3d = 3 * n * sizeof(double), b3i = 3 * n * sizeof(int32_t), b1i = n * sizeof(int32_t);
    OutBuf o[5] = {{x, nullptr, b3d}, {v, nullptr, b3d}, {f, nullptr, b3d}, {img, nullptr, b3i},
                   {ids, nullptr, b1i}};
    size_t need = 0;
    for (auto &b : o)
        if (b.user && !is_device_ptr(b.user)) need += b.bytes;
    char *st = need ? static_cast<char *>(stage_buffer(c, need)) : nullptr;
    if (need && !st) return fail(c, MD_ERR_NOMEM, "staging allocation failed");
    size_t off = 0;
    for (auto &b : o) {
        if (!b.user) continue;
        if (is_device_ptr(b.user)) b.dev = b.user;
        else {
            b.dev = st + off;
            off += b.bytes;
        }
    }
    CK(launch_get_state(c, (double *)o[0].dev, (double *)o[1].dev, (double *)o[2].dev,
                        (int32_t *)o[3].dev, (int32_t *)o[4].dev, nullptr));
    for (auto &b : o)
        if (b.user && b.dev != b.user)
            CK(cudaMemcpyAsync(b.user, b.dev, b.bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MD_OK;
}

md_status md_get_permutation(md_ctx *c, int32_t *perm) {
    MD_TRACE("md_get_permutation");
    if (!c || !perm) return MD_ERR_ARG;
    if (c->nbox != 1) return fail(c, MD_ERR_ARG, "md_get_permutation: single-box contexts only");
    const size_t n = (size_t)c->n_total;
    // slots of box 0 start at 0 and perm holds slot indices < n
    CK(cudaMemcpyAsync(perm, c->perm, n * sizeof(int32_t), cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MD_OK;
}

md_status md_get_neighbors(md_ctx *c, int32_t *nn, int32_t *nbr, int32_t *pad) {
    MD_TRACE("md_get_neighbors");
    if (!c) return MD_ERR_ARG;
    if (pad) *pad = c->pad;
    if (!nn && !nbr) return MD_OK;
    if (!c->list_valid) {
        md_status s = build_with_retry(c);
        if (s) return s;
    }
    const size_t n = (size_t)c->n_total;
    const size_t bnn = n * sizeof(int32_t), bnb = n * (size_t)c->pad * sizeof(int32_t);
    const bool hn = nn && !is_device_ptr(nn), hb = nbr && !is_device_ptr(nbr);
    char *st = static_cast<char *>(stage_buffer(c, (hn ? bnn : 0) + (hb ? bnb : 0) + 16));
    if (!st) return fail(c, MD_ERR_NOMEM, "staging allocation failed");
    int32_t *dnn = nn ? (hn ? reinterpret_cast<int32_t *>(st) : nn) : nullptr;
    int32_t *dnb = nbr ? (hb ? reinterpret_cast<int32_t *>(st + (hn ? bnn : 0)) : nbr) : nullptr;
    CK(launch_get_neighbors(c, dnn, dnb, c->pad));
    if (hn) CK(cudaMemcpyAsync(nn, dnn, bnn, cudaMemcpyDeviceToHost, c->stream));
    if (hb) CK(cudaMemcpyAsync(nbr, dnb, bnb, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MD_OK;
}

md_status md_get_thermo(md_ctx *c, md_thermo *out) {
    if (!c || !out) return MD_ERR_ARG;
    md_status s = ensure_forces(c);
    if (s) return s;
    s = pull_thermo(c);
    if (s) return s;
    fill_thermo(c, 0, out);
    return MD_OK;
}

md_status md_batch_thermo(md_ctx *c, md_thermo *out) {
    if (!c || !out) return MD_ERR_ARG;
    md_status s = ensure_forces(c);
    if (s) return s;
    s = pull_thermo(c);
    if (s) return s;
    for (int b = 0; b < c->nbox; ++b) fill_thermo(c, b, out + b);
    return MD_OK;
}

md_status md_get_thermo_log(md_ctx *c, double *rows, int32_t *count) {
    if (!c || !count) return MD_ERR_ARG;
    const int64_t avail = c->params.thermo_every > 0 ? c->step / c->params.thermo_every + 1 : 0;
    int32_t m = (int32_t)std::min<int64_t>(std::min<int64_t>(avail, c->tlog_cap), *count);
    if (rows && m > 0) {
        CK(cudaMemcpyAsync(rows, c->tlog, sizeof(double) * 4 * m, cudaMemcpyDefault, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    *count = m;
    return MD_OK;
}

md_status md_force_backward(md_ctx *c, const double *dL_dF, double dL_dE, double *dL_dx,
                            double *dL_deps, double *dL_dsigma) {
    MD_TRACE("md_force_backward");
    if (!c || !dL_dF) return MD_ERR_ARG;
    if (c->hpair.nt > 4) return fail(c, MD_ERR_ARG, "md_force_backward supports ntypes <= 4");
    if (c->params.half_list) return fail(c, MD_ERR_ARG, "md_force_backward needs full lists");
    if (!c->ready) return fail(c, MD_ERR_ARG, "internal: state between half-steps");
    // The list is recomputed from the current positions, never reused.
    CK(launch_bin_sort(c, false));
    c->sorted_at = c->step;
    c->list_valid = false;
    c->forces_valid = false;
    invalidate_graphs(c);
    md_status s = build_with_retry(c);
    if (s) return s;
    c->built_at = c->step;
    const size_t n = (size_t)c->n_total;
    const int NP = 2 * c->hpair.nt * c->hpair.nt;
    const size_t need = adjoint_scratch_doubles(c) + 3 * n + 3 * n;
    if (need * sizeof(double) > c->dscratch_bytes) {
        if (c->dscratch) cudaFree(c->dscratch);
        c->dscratch = nullptr;
        c->dscratch_bytes = 0;
        CK(dalloc(&c->dscratch, need));
        c->dscratch_bytes = need * sizeof(double);
    }
    double *G = c->dscratch;                 // 3n (device copy of dL_dF if host)
    double *dx = G + 3 * n;                  // 3n
    double *rest = dx + 3 * n;
    const double *Gd = dL_dF;
    if (!is_device_ptr(dL_dF)) {
        CK(cudaMemcpyAsync(G, dL_dF, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        Gd = G;
    }
    double *dxd = (dL_dx && is_device_ptr(dL_dx)) ? dL_dx : dx;
    double *totals = rest + (adjoint_scratch_doubles(c) - NP);
    CK(launch_adjoint(c, Gd, dL_dE, dxd, totals, rest));
    if (dL_dx && dxd != dL_dx)
        CK(cudaMemcpyAsync(dL_dx, dxd, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    std::vector<double> tot(NP);
    CK(cudaMemcpyAsync(tot.data(), totals, NP * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int nt = c->hpair.nt;
    std::vector<double> de(nt * nt), ds(nt * nt);
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nt; ++b) {
            const int ab = a * nt + b, ba = b * nt + a;
            de[ab] = a == b ? tot[2 * ab] : tot[2 * ab] + tot[2 * ba];
            ds[ab] = a == b ? tot[2 * ab + 1] : tot[2 * ab + 1] + tot[2 * ba + 1];
        }
    if (dL_deps) CK(cudaMemcpy(dL_deps, de.data(), nt * nt * sizeof(double), cudaMemcpyDefault));
    if (dL_dsigma) CK(cudaMemcpy(dL_dsigma, ds.data(), nt * nt * sizeof(double), cudaMemcpyDefault));
    return MD_OK;
}

md_status md_set_state(md_ctx *c, const double *x, const double *v) {
    MD_TRACE("md_set_state");
    if (!c) return MD_ERR_ARG;
    if (!x && !v) return MD_OK;
    const size_t n = (size_t)c->n_total;
    // Current state in original order (for whatever is not replaced), kept in
    // a buffer of its own so that load_state may use the staging buffer.
    const size_t need = 6 * n * sizeof(double) + n * sizeof(int32_t);
    if (need > c->restage_bytes) {
        if (c->restage) cudaFree(c->restage);
        c->restage = nullptr;
        c->restage_bytes = 0;
        CK(cudaMalloc(&c->restage, need));
        c->restage_bytes = need;
    }
    double *xcur = static_cast<double *>(c->restage);
    double *vcur = xcur + 3 * n;
    int32_t *tcur = reinterpret_cast<int32_t *>(vcur + 3 * n);
    CK(launch_get_state(c, x ? nullptr : xcur, v ? nullptr : vcur, nullptr, nullptr, nullptr, tcur));
    // New positions with host velocities: the velocity copy runs on a side
    // stream while the positions are binned, sorted and listed; the
    // velocities go into place (by atom id) before the forces, whose thermo
    // needs them.
    const bool side_v = x && v && !is_device_ptr(v);
    const double *vdev = nullptr;
    if (side_v) {
        md_status s = copy_velocities_beside(c, v, &vdev);
        if (s) return s;
    }
    md_status s = load_state(c, x ? x : xcur, side_v ? nullptr : (v ? v : vcur), tcur, false);
    if (s) return s;
    invalidate_graphs(c);
    s = sort_build(c, true);
    if (s) return s;
    if (side_v) {
        CK(cudaStreamWaitEvent(c->stream, c->ev_side, 0));
        CK(launch_load_velocities(c, vdev));
    }
    s = forces_at_build(c);
    if (s) return s;
    return pull_thermo(c);
}

md_status md_set_positions(md_ctx *c, const double *x) {
    if (!c || !x) return MD_ERR_ARG;
    return md_set_state(c, x, nullptr);
}

md_status md_set_params(md_ctx *c, const double *eps, const double *sigma) {
    MD_TRACE("md_set_params");
    if (!c) return MD_ERR_ARG;
    const int nt = c->hpair.nt;
    std::vector<double> e(eps ? eps : c->eps.data(), (eps ? eps : c->eps.data()) + nt * nt);
    std::vector<double> s(sigma ? sigma : c->sigma.data(), (sigma ? sigma : c->sigma.data()) + nt * nt);
    if (eps && is_device_ptr(eps)) CK(cudaMemcpy(e.data(), eps, nt * nt * sizeof(double), cudaMemcpyDeviceToHost));
    if (sigma && is_device_ptr(sigma)) CK(cudaMemcpy(s.data(), sigma, nt * nt * sizeof(double), cudaMemcpyDeviceToHost));
    md_status st = setup_pair(c, e.data(), s.data());
    if (st) return st;
    CK(cudaMemcpyAsync(c->dpair, &c->hpair, sizeof(Pair), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->forces_valid = false;
    return MD_OK;
}

md_status md_profile(md_ctx *c, int32_t on) {
    if (!c) return MD_ERR_ARG;
    c->prof = on != 0;
    c->prof_launches = 0;
    c->prof_ms = 0.0;
    c->prof_rebuilds = 0;
    c->prof_sort_ms = c->prof_build_ms = 0.0;
    c->ev_used = 0;
    return MD_OK;
}

md_status md_profile_rebuild(md_ctx *c, int64_t *rebuilds, double *sort_ms, double *build_ms) {
    if (!c) return MD_ERR_ARG;
    md_status s = flush_profile_events(c);
    if (s) return s;
    if (rebuilds) *rebuilds = c->prof_rebuilds;
    if (sort_ms) *sort_ms = c->prof_sort_ms;
    if (build_ms) *build_ms = c->prof_build_ms;
    c->prof_rebuilds = 0;
    c->prof_sort_ms = c->prof_build_ms = 0.0;
    return MD_OK;
}

md_status md_profile_read(md_ctx *c, int64_t *launches, double *ms, double *alg_bytes) {
    if (!c) return MD_ERR_ARG;
    md_status s = flush_profile_events(c);
    if (s) return s;
    s = read_flags(c);
    if (s) return s;
    if (launches) *launches = c->prof_launches;
    if (ms) *ms = c->prof_ms;
    if (alg_bytes) {
        // per FUSED launch: list entries (4 B each) + own shadow (16) + each
        // neighbor shadow once (16) + nn (4) + r, v read and written (4 x 24)
        // + new shadow (16); FP64 path reads FP64 neighbor positions (24).
        const double n = (double)c->n_total;
        const double entries = (double)c->hflags->sumnn;
        const double pos = c->params.precision == MD_MIXED ? 16.0 : 24.0;
        *alg_bytes = 4.0 * entries + n * (pos + pos + 4.0 + 96.0 + 16.0);
    }
    c->prof_launches = 0;
    c->prof_ms = 0.0;
    return MD_OK;
}

md_status md_launch_count(md_ctx *c, int64_t *kernels) {
    if (!c || !kernels) return MD_ERR_ARG;
    *kernels = c->kernels;
    return MD_OK;
}

md_status md_debug_expire_waits(md_ctx *c, int32_t on) {
    if (!c) return MD_ERR_ARG;
    c->debug_tx_extra = on ? 16u : 0u;
    invalidate_graphs(c);  // captured launches carry the old value
    return MD_OK;
}

md_status md_info(md_ctx *c, int32_t *nbox, int64_t *n_total) {
    if (!c) return MD_ERR_ARG;
    if (nbox) *nbox = c->nbox;
    if (n_total) *n_total = c->n_total;
    return MD_OK;
}

const char *md_last_error(const md_ctx *c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

void md_destroy(md_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

}  // extern "C"

// md_common.cuh -- internal definitions shared by the CUDA sources of libmd_b300.
//
// Data layout in HBM (all per-atom arrays are indexed by "slot"):
//  * Boxes are concatenated; box b owns slots [slot_off, slot_off + npad), npad a
//    multiple of 32 so that no 32-slot tile straddles two boxes.  Slots past the
//    box's n atoms are inert padding (no cell, empty list, zero state).
//  * Positions are stored cell-relative in FP64: x = O_c + r with O_c the centre
//    of the cell the atom was binned into at the last re-sort, r in SoA
//    (r[0*ns + i], r[1*ns + i], r[2*ns + i]).  Velocities, forces: SoA FP64.
//  * The FP32 "shadow" sh[i] = (float(r_x), float(r_y), float(r_z), type bits)
//    is what the mixed-precision kernels read; cell-local coordinates keep its
//    rounding error at 2^-24 of the cell size instead of the box size.
//  * Neighbor list entries are uint32: bits 0..26 the neighbor slot j,
//    bits 27..31 the stencil offset code (ox+1) + 3 (oy+1) + 9 (oz+1) of j's
//    cell relative to i's cell, so that x_j - x_i = (r_j - r_i) + delta * h.
//    The list is padded to `pad` entries per atom and transposed per warp: with
//    T lanes per atom (A = 32/T atoms per warp), entry k of atom i lives at
//      ((i / A) * R + k / T) * 32 + (i % A) * T + k % T,     R = pad / T,
//    so one warp-wide load of 32 consecutive words serves all lanes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "md.h"

#define MD_MAXT 8
#define MD_IDX_BITS 27
#define MD_IDX_MASK 0x07FFFFFFu

// Compile-time tuning of the mixed force kernel: list entries each lane takes
// per batch, and the resident CTAs per SM its register budget is sized for.
#ifndef MD_FORCE_BATCH
#define MD_FORCE_BATCH 4
#endif
#ifndef MD_FORCE_MINB
#define MD_FORCE_MINB 6   // measured best on B300 at 4M atoms (5: 1.03 ms, 6: 0.94 ms)
#endif
// List terms combined by an FMA chain before each Kahan add (divides MD_FORCE_BATCH).
#ifndef MD_FORCE_GROUP
#define MD_FORCE_GROUP 4
#endif

namespace mdb {

enum : uint32_t { ST_OVERFLOW = 1u, ST_NONFINITE = 2u, ST_TIMEOUT = 4u };
constexpr uint32_t ST_FREEZE = ST_OVERFLOW | ST_NONFINITE | ST_TIMEOUT;

// Force-kernel modes.
enum { MODE_FORCE_ONLY = 0, MODE_FINAL = 1, MODE_FUSED = 2 };

// Per-warp-tile thermo partial: PE, KE, Px, Py, Pz, max |r - r_build|^2, 0, 0.
constexpr int TP = 8;
// Per-box thermo record: PE, KE, Px, Py, Pz, max displacement, step, spare.
constexpr int TB = 8;

struct Box {
    double L[3];
    double h[3];      // cell edge L / nc
    double inv[3];    // nc / L (FP64, computed once)
    float hf[3];      // float(h)
    int32_t nc[3];
    int32_t cell_off; // first global cell id of this box
    int32_t ncell;
    int32_t slot_off; // first slot
    int32_t n;        // atoms
    int32_t npad;     // slots (multiple of 32)
    int32_t ctab;     // offset of this box's cell centres in md_ctx::ctab
    int64_t atom_base;  // sum of n over earlier boxes
};

struct Pair {
    int32_t nt;
    int32_t shift;
    double rc2, rs2, dt, half_skin;
    float rc2f, rs2f, bandf, pad_;
    double eps[64], sig[64];
    double e24[64], s2[64], e4[64], ush[64];  // 24 eps, sigma^2, 4 eps, U(rc) (0 if unshifted)
    float fs2[64], fe4[64], fush[64];  // sigma^2, 4 eps, U(rc) in FP32
    float fc1[64];                      // 24 eps / sigma^2 in FP32
    double mass[MD_MAXT], dtm[MD_MAXT], hdtm[MD_MAXT];
};

// Device counters / flags of one context.
struct Flags {
    uint32_t status;
    int32_t maxnn;
    int64_t clock;          // step whose forces are computed next / of the READY state
    unsigned long long sumnn;  // sum of row lengths at the last build
    int64_t builds;
    int64_t dangerous;
    uint32_t maxdisp_bits;  // float bits of max displacement seen by the current re-sort
    uint32_t thermo;        // 1 if the last force launch wrote thermo partials
    uint32_t done;          // CTA completion counter of the force kernel (last-CTA pattern)
    uint32_t check_site;    // checked build: first failing index check (CheckSite), else 0
    int64_t check_index;    // checked build: the index that failed it
};

// Checked build (nvcc -DMD_CHECKED): the hot path's gathers and scatters test
// each index against the array it addresses.  An index out of range is
// recorded (the first failing site and its index, in the context's flags);
// a gather then reads a harmless in-range element instead and a scatter is
// skipped, and the next host call that reads the flags fails with
// MD_ERR_CUDA naming the site.  In the default build the checks compile to
// nothing.
enum CheckSite : uint32_t {
    CHK_NONE = 0,
    CHK_SORT_SCATTER,    // k_scatter: destination slot inside the atom's box
    CHK_SORT_PERMUTE,    // k_permute: source slot inside the atom's box
    CHK_BUILD_HOME,      // k_build: home atom slot < ns
    CHK_BUILD_CAND,      // k_build: candidate slot < ns
    CHK_FORCE_GATHER,    // mixed force kernels: neighbor shadow slot <= ns
    CHK_FORCE64_GATHER,  // FP64 force kernel: neighbor slot (< ns for positions)
    CHK_ADJ_GATHER,      // adjoint kernel: neighbor slot < ns
    CHK_SPME_GATHER,     // SPME real-space pass: neighbor slot (<= ns shadows, < ns positions)
    CHK_SITES
};

// Index i for an access to an array of n elements: i itself when in range,
// else (checked build) `safe` after recording the failure.
__device__ __forceinline__ int64_t chk_index(int64_t i, int64_t n, uint32_t site, Flags *fl,
                                             int64_t safe) {
#ifdef MD_CHECKED
    if (i >= 0 && i < n) return i;
    if (atomicCAS(&fl->check_site, 0u, site) == 0u) fl->check_index = i;
    return safe;
#else
    (void)n; (void)site; (void)fl; (void)safe;
    return i;
#endif
}

// Whether a scatter to index i may go ahead: lo <= i < hi (always true in the
// default build).
__device__ __forceinline__ bool chk_ok(int64_t i, int64_t lo, int64_t hi, uint32_t site,
                                       Flags *fl) {
#ifdef MD_CHECKED
    if (i >= lo && i < hi) return true;
    if (atomicCAS(&fl->check_site, 0u, site) == 0u) fl->check_index = i;
    return false;
#else
    (void)i; (void)lo; (void)hi; (void)site; (void)fl;
    return true;
#endif
}

// Stencil code of a zero offset (ox = oy = oz = 0).
constexpr uint32_t kCodeZero = 13;

// The centre of cell (cx, cy, cz) along axis d, computed identically wherever
// an FP64 position is reconstructed as O + r.
// Centre of cell c along axis d of box B: (c + 1/2) h_d, each rounded once,
// tabulated on the host (md_ctx::ctab: per box the nc_x, nc_y, nc_z centres).
__device__ __forceinline__ double cell_centre(const double *__restrict__ ctab, const Box &B, int d,
                                              int c) {
    return __ldg(ctab + B.ctab + (d == 0 ? 0 : (d == 1 ? B.nc[0] : B.nc[0] + B.nc[1])) + c);
}

__device__ __forceinline__ void unpack_cell(int32_t p, int &cx, int &cy, int &cz) {
    cx = p & 1023;
    cy = (p >> 10) & 1023;
    cz = (p >> 20) & 1023;
}
__device__ __forceinline__ int32_t pack_cell(int cx, int cy, int cz) {
    return cx | (cy << 10) | (cz << 20);
}

}  // namespace mdb

// The context.  Plain struct so that every .cu file can launch on it.
struct md_ctx {
    // configuration
    int32_t nbox = 0;
    int64_t n_total = 0;     // atoms
    int64_t ns = 0;          // slots (padded)
    int32_t ncell_tot = 0;
    std::vector<mdb::Box> hbox;
    md_params params{};
    std::vector<double> eps, sigma, mass;
    mdb::Pair hpair{};
    cudaStream_t stream = nullptr;
    int nsm = 148;
    int T = 4;               // lanes per atom (list layout + force kernel)
    int block = 128;         // force kernel CTA size
    int pad = 128;           // list slots per atom
    int R = 32;              // rows per warp tile = pad / T

    // device buffers
    double *r[2] = {nullptr, nullptr};
    double *v[2] = {nullptr, nullptr};
    double *f = nullptr, *rbuild = nullptr, *xw = nullptr, *xws = nullptr, *xraw = nullptr;
    float4 *sh[2] = {nullptr, nullptr};
    int32_t *type[2] = {nullptr, nullptr}, *id[2] = {nullptr, nullptr};
    int32_t *img[2] = {nullptr, nullptr}, *cellc[2] = {nullptr, nullptr};
    int32_t *cell = nullptr, *rank = nullptr, *perm = nullptr, *ptmp = nullptr;
    int32_t *count = nullptr, *cstart = nullptr, *nn = nullptr;
    int32_t *scan_part = nullptr;  // per-block sums of the cell-count scan
    double *ctab = nullptr;        // cell centres of every box and axis (Box::ctab)
    uint32_t *nbr = nullptr;
    size_t nbr_words = 0;
    mdb::Box *dbox = nullptr;
    int32_t *tile_box = nullptr;   // per 32-slot tile
    int32_t *cell_box = nullptr;   // per global cell
    mdb::Pair *dpair = nullptr;
    mdb::Flags *dflags = nullptr;
    double *tpart = nullptr;       // ns/ (32/T) warp tiles * TP  (allocated for T = 1: ns * TP)
    double *tbox = nullptr;        // nbox * TB
    double *fpart = nullptr;       // nbox * fsplit * 6: first-level thermo sums
    int fsplit = 1;                // CTAs per box in the first thermo level
    double *tlog = nullptr;        // log rows * 4
    int32_t tlog_cap = 0;
    float4 *facc = nullptr;        // half lists: per-slot force + energy accumulators (ns + 1)
    double *facc64 = nullptr;      // half lists, FP64 context: the same, 4 doubles per slot
    float *shv = nullptr;          // shadow_vl > 0: AoSoA copy of the shadows (slots 0..ns)
    double *dscratch = nullptr;    // adjoint partials etc.
    size_t dscratch_bytes = 0;
    // pinned host mirrors
    mdb::Flags *hflags = nullptr;
    double *htbox = nullptr;

    // dynamic state
    int pc = 0, oc = 0;            // current position / order buffers
    int64_t step = 0;
    bool ready = true;             // READY: v = v_n and f = F(x_n); else DRIFTED
    bool list_valid = false;
    int64_t sorted_at = -1;        // step of the state at the last cell sort
    int64_t host_builds = 0;
    int32_t cur_tlog_rows = 0;

    // graphs: one executable per (pc, oc) parity at the start of a period
    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t graph_nk[4] = {0, 0, 0, 0};   // kernels in each captured graph
    int64_t built_at = -1;         // step at which the current list was built
    bool forces_valid = false;
    // host-pointer staging
    void *stage = nullptr;
    size_t stage_bytes = 0;
    void *restage = nullptr;       // current state in original order (md_set_state)
    cudaStream_t side = nullptr;   // md_set_state: host velocities copied beside the sort
    cudaEvent_t ev_main = nullptr, ev_side = nullptr;
    size_t restage_bytes = 0;

    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_tag;       // per used event pair: 0 force, 1 re-sort, 2 list build
    size_t ev_used = 0;
    int64_t prof_launches = 0;
    int64_t prof_rebuilds = 0;
    double prof_sort_ms = 0.0, prof_build_ms = 0.0;
    int64_t kernels = 0;           // library kernels enqueued (see md_launch_count)
    uint32_t debug_tx_extra = 0;   // md_debug_expire_waits
    double prof_ms = 0.0;
    double prof_bytes = 0.0;

    std::string err;
};

// ---- launchers implemented across the .cu files (host side) -------------
namespace mdb {
// md_sort.cu
cudaError_t launch_bin_sort(md_ctx *c, bool raw_input);
cudaError_t launch_load_velocities(md_ctx *c, const double *v_aos);
cudaError_t launch_unpack_input(md_ctx *c, const double *x_aos, const double *v_aos,
                                const int32_t *types);
// md_neigh.cu
cudaError_t launch_build(md_ctx *c);
size_t build_smem_bytes(int pad);
// md_force.cu
cudaError_t launch_force(md_ctx *c, int mode);
cudaError_t launch_kick_drift(md_ctx *c);
cudaError_t launch_finalize(md_ctx *c, int mode);
cudaError_t launch_get_state(md_ctx *c, double *x_aos, double *v_aos, double *f_aos,
                             int32_t *img_aos, int32_t *ids, int32_t *types);
cudaError_t launch_get_neighbors(md_ctx *c, int32_t *nn_out, int32_t *nbr_out, int pad_out);
// md_adjoint.cu
cudaError_t launch_adjoint(md_ctx *c, const double *G_aos, double gE, double *dx_aos,
                           double *totals_out, double *scratch);
size_t adjoint_scratch_doubles(md_ctx *c);
// The list entry that pads rows past their count (up to the warp-tile's
// longest row after each build; the rows of padding slots hold it from the
// list's allocation on): the dummy shadow slot ns (kept far from every atom)
// with a zero offset; a pair evaluated against it is masked by rc.
// 1/x in FP64 for the FP64 pair kernels (x a normal positive number): the
// hardware's approximate FP64 reciprocal (relative error ~1e-6) refined by two
// Newton-Raphson steps for f(y) = 1/y - x, y' = y + y (1 - x y), each of which
// squares the relative error.  Measured on B300 over 1.7e7 arguments in
// [0.25, 64): equal to the IEEE quotient on every one, in fewer FP64
// instructions than the division.  (The same scheme for 1/sqrt(x) came within
// 2 ulp but cost more than rsqrt().)
__device__ __forceinline__ double rcp_newton64(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double e = fma(-x, y, 1.0);
        y = fma(y, e, y);
    }
    return y;
}

__host__ __device__ inline uint32_t sentinel_entry(int64_t ns) {
    return (uint32_t)ns | (kCodeZero << MD_IDX_BITS);
}
inline uint32_t sentinel_entry(const md_ctx *c) { return sentinel_entry(c->ns); }
cudaError_t fill_list_sentinel(md_ctx *c);
// md_api.cu: record a message for md_last_error(NULL) and return s
md_status set_global_error(md_status s, const std::string &msg);
}  // namespace mdb

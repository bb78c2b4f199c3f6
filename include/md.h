/*
 * md.h -- C ABI of the B300 (sm_103a) short-range Lennard-Jones MD library.
 *
 * The calls follow the paper's anatomy of an MD timestep (arXiv 2109.09056,
 * Introduction and Fig. 1: "from a description of the neighborhood (neighbor
 * list), each particle's forces are calculated to propagate the particles to
 * new positions; the particles are then resorted to begin the next timestep"),
 * and the Cabana operations it lists for that step: particle sorting by
 * geometric binning (Section "Particle Sorting"), Verlet neighbor lists built
 * by binning (Section "Neighbor List Creation"), and the Lennard-Jones
 * short-range force kernel of CabanaMD (Section "CabanaMD").
 *
 * Conventions shared by every call
 *  - Every function returns md_status and never aborts or throws across the
 *    ABI.  On failure md_last_error(ctx) returns a message (per context; for a
 *    failed md_create / md_batch_create, md_last_error(NULL) holds it).
 *  - Array arguments are plain pointers.  Each one may be host or device
 *    memory: it is treated as device memory iff cudaPointerGetAttributes says
 *    so.  Input arrays are copied into library-owned device buffers; output
 *    arrays are caller-owned and written in full.
 *  - Positions, velocities, forces and gradients are n x 3 row-major (AoS)
 *    float64, in ORIGINAL atom order (the order of md_create's input).  The
 *    library re-sorts atoms into cell order internally; only md_get_state's
 *    ids, md_get_permutation and md_get_neighbors expose that internal order.
 *  - All device work is enqueued on the CUDA stream given at creation
 *    (NULL = legacy default stream); md_set_state alone copies host
 *    velocities on a library-owned side stream, ordered after that stream and
 *    before the work that needs them by events.  Calls that return values to
 *    the host (getters, md_step, md_compute_forces) synchronise that stream.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Units are reduced LJ units (k_B = 1).  The box is orthorhombic with its
 *    origin at 0 and periodic on all axes.
 */
#ifndef MD_B300_H
#define MD_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = 1,              /* bad argument (NULL, n < 1, type out of range, ...) */
    MD_ERR_BOX_TOO_SMALL = 2,    /* some box edge L <= 2 (rc + skin) */
    MD_ERR_NEIGH_OVERFLOW = 3,   /* md_build_neighbors: a row needs more than the list pad
                                    (md_step grows the pad and rebuilds by itself) */
    MD_ERR_DANGEROUS_BUILD = 4,  /* only with md_params.check_displacement: some atom moved
                                    more than skin/2 between two builds; the run completed */
    MD_ERR_NONFINITE = 5,        /* a position or velocity is NaN/Inf; the run froze there */
    MD_ERR_TIMEOUT = 6,          /* a bounded device wait (~1 s; the mixed force kernel's wait
                                    for a list copy) ran out; the step was abandoned, the
                                    state is undefined: destroy the context */
    MD_ERR_CUDA = 7,             /* a CUDA runtime call failed (message has the CUDA error) */
    MD_ERR_NOMEM = 8             /* device or host allocation failed */
} md_status;

enum { MD_FP64 = 0, MD_MIXED = 1 };

typedef struct {
    double L[3];                 /* box edges; all three must exceed 2 (rc + skin) */
} md_box;

typedef struct {
    int32_t ntypes;              /* 1 .. 8 */
    const double *eps;           /* ntypes*ntypes, symmetric, row-major (host memory) */
    const double *sigma;         /* ntypes*ntypes, symmetric, row-major (host memory) */
    const double *mass;          /* ntypes (host memory) */
    double rc;                   /* pair cutoff (absolute, not scaled by sigma); strict r < rc */
    double skin;                 /* list radius is rc + skin; strict r < rc + skin */
    double dt;
    int32_t rebuild_every;       /* re-sort + list rebuild when step % rebuild_every == 0 */
    int32_t precision;           /* MD_FP64 or MD_MIXED */
    int32_t shift_energy;        /* 0: plain truncation at rc; 1: U(r) - U(rc) per pair */
    int32_t check_displacement;  /* 1: md_step returns MD_ERR_DANGEROUS_BUILD (see above) */
    int32_t thermo_every;        /* >0: log PE/KE/T/momentum every k steps (md_get_thermo_log) */
    int32_t neigh_pad;           /* list slots per atom; 0 = automatic (grown on overflow) */
    int32_t lanes_per_atom;      /* 1, 2, 4 or 8 lanes per atom in the force kernel; 0 = auto
                                    (4; 1 for MD_FP64 contexts of >= 8192 atoms per SM) */
    int32_t block_threads;       /* mixed force-kernel CTA size (64..768, multiple of 32; an
                                    upper bound when its list buffers would not fit in shared
                                    memory; the FP64 kernel uses at most 256); 0 = automatic
                                    (768 when the system has enough warp-tiles and it fits) */
    int32_t use_graphs;          /* 1: md_step replays one rebuild period as a CUDA graph */
    int32_t half_list;           /* 1: half Verlet lists (Newton's third law: each pair once,
                                    its reaction added to the partner by atomics, FP32 in a
                                    mixed context, FP64 in an FP64 one); 4 lanes per atom
                                    only (else MD_ERR_ARG); forces are then reproducible to
                                    rounding, not bitwise; md_force_backward refuses such a
                                    context (the SPME solver's real-space pass takes half
                                    lists too).  0: full lists (default). */
    int32_t shadow_vl;           /* layout the mixed force kernel gathers neighbor positions
                                    from: 0 = one float4 (x, y, z, type) per atom (default);
                                    8 or 32 = blocks of that many atoms holding x[], y[],
                                    z[], type[] in turn (AoSoA), refreshed from the float4
                                    shadows before each force evaluation; mixed precision
                                    with 4 lanes per atom and full lists only (else
                                    MD_ERR_ARG).  Same forces bit for bit. */
} md_params;

/* Fills p with the classic LJ-melt settings: 1 type, eps = sigma = m = 1,
 * rc = 2.5, skin = 0.3, dt = 0.005, rebuild every 20, MD_MIXED, graphs on.
 * The eps/sigma/mass pointers are set to library-owned static unit values. */
void md_params_default(md_params *p);

typedef struct {
    int64_t step;                /* step counter of the state the numbers describe */
    double pe;                   /* potential energy, FP64 total */
    double ke;                   /* kinetic energy, sum 1/2 m v^2 */
    double etot;                 /* pe + ke */
    double temperature;          /* 2 ke / (3n - 3) */
    double momentum[3];          /* sum m v */
    double max_displacement;     /* max |x - x_at_last_build| over atoms */
    int32_t nn_max;              /* largest list row at the last build */
    int32_t pad;                 /* current list slots per atom */
    int64_t builds;              /* list builds so far */
    int64_t dangerous_builds;    /* builds that found max_displacement > skin/2 */
} md_thermo;

typedef struct md_ctx md_ctx;

/* ---- one periodic box ------------------------------------------------- */

/* Creates a context for n atoms in one box: copies x, v (n x 3) and types (n,
 * values in [0, ntypes)), then wraps, bins, re-sorts into cell order, builds
 * the neighbor list and computes the forces of step 0.  `stream` is a
 * cudaStream_t (NULL = default stream).  *out receives the context; on
 * failure *out is NULL (when out is not NULL).
 * Errors: MD_ERR_ARG, MD_ERR_BOX_TOO_SMALL, MD_ERR_NONFINITE, MD_ERR_NOMEM,
 * MD_ERR_CUDA. */
md_status md_create(const md_box *box, int64_t n, const double *x, const double *v,
                    const int32_t *types, const md_params *params, void *stream,
                    md_ctx **out);

/* The resort step (Section "Particle Sorting": sort by geometric binning):
 * wraps positions into [0, L), computes each atom's cell
 *   c = (cz * nc_y + cy) * nc_x + cx,  c_d = min(floor(x_d * nc_d / L_d), nc_d - 1),
 *   nc_d = floor(L_d / (rc + skin)),
 * and re-orders all per-atom state stably by (cell, current index) with an
 * atomic histogram, a prefix scan and a per-cell ordering by prior index.
 * md_get_permutation then returns perm[new] = old for this sort.  The
 * neighbor list and forces are invalid until md_build_neighbors /
 * md_compute_forces run. */
md_status md_bin_sort(md_ctx *ctx);

/* Builds the full Verlet list (Section "Neighbor List Creation"): for every
 * atom i, every j != i whose nearest-image distance satisfies
 *   r^2 = (dx*dx + dy*dy) + dz*dz < (rc + skin)^2,  d = x_j - x_i folded once by +-L,
 * evaluated in FP64 with each operation rounded separately, searched over the
 * 27 cells around i's cell.  If the atoms moved since the last cell sort, it
 * first re-sorts them (as md_bin_sort).  The list is stored padded and
 * transposed (warp-coalesced).  Returns MD_ERR_NEIGH_OVERFLOW if a row needs
 * more than the current pad (the pad is then grown, call again). */
md_status md_build_neighbors(md_ctx *ctx);

/* Lennard-Jones 12-6 forces and energy over the current list (Section
 * "CabanaMD": the LJ short-range benchmark kernel):
 *   F_i = sum_j 24 eps_ab / r^2 [2 (sigma_ab/r)^12 - (sigma_ab/r)^6] (x_i - x_j),  r < rc,
 *   PE  = sum_{i<j} 4 eps_ab [(sigma_ab/r)^12 - (sigma_ab/r)^6]  (- U(rc) if shifted).
 * MD_FP64: all FP64.  MD_MIXED: FP32 pair arithmetic on cell-local FP32
 * coordinates, per-atom Kahan-compensated FP32 sums, FP64 force output and
 * FP64 energy total.  *energy_out (host pointer, may be NULL) receives PE. */
md_status md_compute_forces(md_ctx *ctx, double *energy_out);

/* Advances nsteps velocity-Verlet steps ("forces are calculated to propagate
 * the particles to new positions; the particles are then resorted"):
 *   v += dt/2 F/m;  x += dt v;  [re-sort + rebuild when step % rebuild_every == 0];
 *   F = F(x);  v += dt/2 F/m.
 * The two half-kicks between consecutive force evaluations are applied as one
 * kick v += dt F/m except on thermo-log steps.  If the list overflows the pad
 * during the run, the run freezes at that step, the pad is grown, and the
 * run resumes from there.  *last_out (host, may be NULL) receives thermo of the
 * final state. */
md_status md_step(md_ctx *ctx, int32_t nsteps, md_thermo *last_out);

/* Force-matching adjoint (the backward of md_compute_forces).  Given
 * dL_dF (n x 3, original order) and dL_dE, writes
 *   dL_dx (n x 3):   sum_{j in nbr(k)} M_kj (G_k - G_j) - dL_dE * F_k,
 *                    M_kj = phi I + 2 dphi/du d d^T,  phi = (24 eps/u)(2 s12 - s6),
 *   dL_deps, dL_dsigma (ntypes x ntypes, symmetric): derivative w.r.t. the one
 *                    parameter of each unordered type pair (mirrored),
 * all in FP64.  The list is recomputed from the current positions (re-sort and
 * rebuild), never taken from a stored forward pass.  Any output pointer may be
 * NULL to skip it. */
md_status md_force_backward(md_ctx *ctx, const double *dL_dF, double dL_dE, double *dL_dx,
                            double *dL_deps, double *dL_dsigma);

/* Replaces positions (n x 3, original order) and optionally the pair tables
 * (ntypes*ntypes host arrays; NULL keeps the current ones); velocities kept.
 * Follows with the same wrap/sort/build/forces as md_create. */
md_status md_set_positions(md_ctx *ctx, const double *x);
/* Replaces positions and velocities (n x 3 each, original order; NULL keeps
 * the current array) and re-sorts / rebuilds / recomputes forces. */
md_status md_set_state(md_ctx *ctx, const double *x, const double *v);
md_status md_set_params(md_ctx *ctx, const double *eps, const double *sigma);

/* Copies the state out in ORIGINAL order: x (n x 3, positions as stored: wrapped
 * at the last re-sort, then drifted), v, f (forces of the current state),
 * img (n x 3 int32 periodic image counts: unwrapped = x + img * L), and ids
 * (n, int32): ids[k] = original index of internal slot k.  Any pointer may be
 * NULL. */
md_status md_get_state(md_ctx *ctx, double *x, double *v, double *f, int32_t *img,
                       int32_t *ids);

/* perm (n, int32): perm[new] = old internal index for the most recent sort. */
md_status md_get_permutation(md_ctx *ctx, int32_t *perm);

/* Current list in INTERNAL order: nn (n), and, if nbr != NULL, rows
 * nbr[i * (*pad) + k] (k < nn[i]) holding internal neighbor indices.  Call
 * with nbr == NULL first to read *pad. */
md_status md_get_neighbors(md_ctx *ctx, int32_t *nn, int32_t *nbr, int32_t *pad);

/* Thermo of the current state (synchronises). */
md_status md_get_thermo(md_ctx *ctx, md_thermo *out);

/* Thermo log written every params.thermo_every steps since creation:
 * rows of 4 doubles (step, PE, KE, Etot); *count (in: capacity in rows,
 * out: rows written). */
md_status md_get_thermo_log(md_ctx *ctx, double *rows, int32_t *count);

/* Kernel timing: when on, the force kernel launches are bracketed by CUDA
 * events on the context's stream (graphs are bypassed).  md_profile_read
 * returns the number of force-kernel launches and their summed device time
 * (ms) since the last reset, plus the bytes each launch touches by the
 * algorithmic count (list entries + positions + state), and resets. */
md_status md_profile(md_ctx *ctx, int32_t on);
md_status md_profile_read(md_ctx *ctx, int64_t *launches, double *ms, double *alg_bytes);
/* The same for the rebuilds md_step performs while profiling is on: their
 * number and the summed device time (ms) of the re-sort (binning, scan,
 * permutation, state gather) and of the list build since the last call. */
md_status md_profile_rebuild(md_ctx *ctx, int64_t *rebuilds, double *sort_ms, double *build_ms);

/* Number of library kernels enqueued on this context since creation (graph
 * replays count every kernel node of the replayed graph). */
md_status md_launch_count(md_ctx *ctx, int64_t *kernels);

/* Test hook for the timeout path, off by default: with on != 0 the mixed force
 * kernel arms each list-copy barrier for 16 bytes more than it copies, so its
 * bounded waits run out and the call returns MD_ERR_TIMEOUT (no device fault,
 * no unbounded wait).  Not for production use. */
md_status md_debug_expire_waits(md_ctx *ctx, int32_t on);

const char *md_last_error(const md_ctx *ctx);
void md_destroy(md_ctx *ctx);

/* ---- batched ensemble: many independent boxes in one context ----------- */
/* Pattern: hundreds of independent small boxes (the parallel-replica use the
 * paper mentions for EXAALT) advanced together: every kernel runs over all
 * boxes in one launch, and each step is one persistent force launch. */

/* nbox boxes; n_per_box[b] atoms in box b; x, v (sum n x 3) and types
 * concatenated in box order.  Same params for all boxes. */
md_status md_batch_create(int32_t nbox, const int64_t *n_per_box, const md_box *boxes,
                          const double *x, const double *v, const int32_t *types,
                          const md_params *params, void *stream, md_ctx **out);

/* Per-box thermo of the current state: out has nbox entries. */
md_status md_batch_thermo(md_ctx *ctx, md_thermo *out);

/* Number of boxes (1 for md_create contexts) and total atoms. */
md_status md_info(md_ctx *ctx, int32_t *nbox, int64_t *n_total);

/* ---- binning + stable cell-order permutation without any allocation ----
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory: code running under an allocator that owns the
 * device's memory, or a loop that must not pay the device-wide
 * synchronisation cudaMalloc/cudaFree can trigger.  It computes what
 * md_bin_sort does for a fresh box (wrap, cell per atom, stable sort by
 * (cell, input index)) and writes perm[new] = old for the n positions x.
 *   box, rs      : box edges (each > 2 rs) and the cell-size floor rs = rc + skin;
 *   x            : n x 3 positions, DEVICE memory, read only;
 *   perm         : n int32, DEVICE memory, written;
 *   stream       : cudaStream_t the work is enqueued on (returns without waiting).
 * It allocates nothing: its intermediates live in one fixed array inside the
 * library (about 4 MiB, held on every GPU that loads the library until the
 * process exits).  Limits: n <= 262144 and nc_x*nc_y*nc_z <= 131072, else
 * MD_ERR_ARG.  Cost: the per-cell ordering is O(m^2) for a cell of m atoms
 * (one warp ranks each atom against the whole cell), so a cell holding
 * thousands of atoms is slow; liquid densities put ~20 in a cell.  Host pointers are rejected (MD_ERR_ARG).  Errors are reported
 * through md_last_error(NULL).  The first call on a device looks up the
 * array's device address (a host-side query), so make that first call before
 * any stream capture.  All calls share the array: calls whose work may
 * overlap on the GPU (unordered streams) race and must be serialised by the
 * caller.  Positions must be finite: a non-finite coordinate is clamped to
 * an edge cell (no access leaves the arrays) but its place in the order is
 * meaningless. */
md_status md_bin_sort_noalloc(const md_box *box, int64_t n, const double *x, double rs,
                              int32_t *perm, void *stream);

/* Asynchronous state download, for trajectory output while the context keeps
 * stepping.  md_state_stream_push takes a snapshot of x and v (n x 3 FP64,
 * original atom order) on the context's stream, in stream order, into one of
 * two library-owned device slots, and queues its copy into x and v (either
 * may be NULL; host buffers should be pinned for the copy to overlap the
 * context's work) on the object's own stream; it returns without waiting.
 * The buffers hold the snapshot once md_state_stream_wait has returned; a slot
 * is reused only after its previous copy finished.  Errors: MD_ERR_ARG,
 * MD_ERR_NOMEM, MD_ERR_CUDA; messages via md_state_stream_last_error.  The
 * object must be destroyed before its context. */
typedef struct md_state_stream md_state_stream;
md_status md_state_stream_create(md_ctx *ctx, md_state_stream **out);
md_status md_state_stream_push(md_state_stream *s, double *x, double *v);
md_status md_state_stream_wait(md_state_stream *s);
const char *md_state_stream_last_error(const md_state_stream *s);
void md_state_stream_destroy(md_state_stream *s);

#ifdef __cplusplus
}
#endif
#endif /* MD_B300_H */

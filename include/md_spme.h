/*
 * md_spme.h -- C ABI of the long-range Coulomb solver of libmd_b300: smooth
 * particle mesh Ewald (SPME) attached to a single-box md_ctx.
 *
 * The paper's CabanaMD section lists the long-range solver's steps: spline
 * kernels spread each particle's charge onto a uniform grid, 3-D FFTs give the
 * reciprocal-space energy and forces, a gradient kernel gathers the grid's
 * force contributions back onto the particles, and real-space pairs are
 * evaluated with the same neighbor iteration as the short-range forces.  The
 * method it cites is Essmann et al., "A smooth particle mesh Ewald method",
 * J. Chem. Phys. 103, 8577 (1995).  With a unit Coulomb constant (pair energy
 * q_i q_j / r) the energy is split as
 *
 *   E_real  = sum_{i<j, r_ij < rc} q_i q_j erfc(alpha r_ij) / r_ij
 *             (over the context's Verlet list, nearest image);
 *   E_recip = 1/2 sum_m theta(m) |FFT(Q)(m)|^2,
 *             Q(k) = sum_i q_i prod_d M_p(u_id - k_d)  (k_d mod K_d),
 *             u_d = K_d x_d / L_d, M_p the cardinal B-spline of order p,
 *             theta(m) = B(m) exp(-pi^2 |m|^2/alpha^2) / (pi V |m|^2),
 *             theta(0) = 0, B the product of the Euler-spline moduli;
 *   E_self  = -alpha/sqrt(pi) sum_i q_i^2;
 *   E_bg    = -pi (sum_i q_i)^2 / (2 V alpha^2)  (neutralising background).
 *
 * Forces are -dE/dx: the real-space pair forces plus, per atom, the spline
 * gradient of Q contracted with dE/dQ = inverse FFT of theta FFT(Q).
 *
 * Conventions are those of md.h (status returns, host-or-device pointers,
 * original atom order, the context's stream; the real-space pass runs on a
 * solver-owned side stream, ordered after the context's stream and before the
 * work that needs it by events, unless profiling is on).  Arithmetic follows the
 * context's precision.  MD_FP64: everything in FP64 (double-complex FFTs).
 * MD_MIXED: reciprocal part with FP32 spline weights, an FP32 grid,
 * single-precision FFTs and an FP32 gather; real-space pairs in FP32 on the
 * context's cell-relative shadow with Kahan-compensated per-atom sums; energy
 * totals accumulated in FP64 and forces returned in FP64.  The 3-D FFTs are
 * cuFFT (real-to-complex and back, out of place).
 */
#ifndef MD_B300_SPME_H
#define MD_B300_SPME_H

#include <stdint.h>

#include "md.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_spme md_spme;

typedef struct {
    double alpha;     /* Ewald splitting parameter (1/length), > 0 */
    double rc;        /* real-space cutoff, 0 < rc <= the context's md_params.rc, so
                         that the context's list (rc + skin) holds every real-space pair
                         under the same displacement condition as the LJ forces */
    int32_t K[3];     /* reciprocal grid points along x, y, z: order <= K_d <= 4096, each a
                         product of 2s, 3s, 5s and 7s (the FFTs' radices), else MD_ERR_ARG */
    int32_t order;    /* B-spline order p: 4, 6 or 8 (even: the Euler-spline
                         moduli of an odd order vanish at m = K/2 for even K) */
} md_spme_params;

/* Attaches an SPME solver to ctx, which must hold one box and outlive the
 * solver.  q: n charges (the context's n) in original atom order, host or
 * device, copied.  Allocates the grid (K_x K_y K_z reals), its half spectrum
 * (K_z K_y (K_x/2+1) complex), the influence table theta (K_z K_y (K_x/2+1)
 * reals, built once on the device), reals FP64 or FP32 by the context's
 * precision, and two cuFFT plans on the context's stream.
 * Errors: MD_ERR_ARG (NULL pointer, batched context, parameter out of range),
 * MD_ERR_NONFINITE (a charge is NaN/Inf), MD_ERR_NOMEM, MD_ERR_CUDA (also for a
 * cuFFT failure).  On failure *out is NULL and md_spme_last_error(NULL) holds
 * the message. */
md_status md_spme_create(md_ctx *ctx, const double *q, const md_spme_params *p, md_spme **out);

/* Replaces the charges (n values, original atom order, host or device). */
md_status md_spme_set_charges(md_spme *s, const double *q);

/* Coulomb forces and energies at the context's current positions (its current
 * step; the context must not be between the halves of a step, which it never
 * is between calls).  Builds the context's list first if it has none.
 * f: n x 3 forces (original atom order, host or device, may be NULL);
 * energy: host array of 4 (may be NULL): E_real, E_recip, E_self + E_bg,
 * total.  Synchronises the context's stream.  Errors: MD_ERR_ARG, and those of
 * md_build_neighbors / CUDA / cuFFT. */
md_status md_spme_compute(md_spme *s, double *f, double *energy);

/* nsteps of velocity Verlet (paper, Introduction and Fig. 1: forces ->
 * propagate -> resort) with the total force LJ + Coulomb: per step the
 * context's kick and drift, its re-sort and list rebuild every rebuild_every
 * steps, its LJ forces, the SPME forces added to them, and the closing
 * half-kick.  The total forces of the starting state are those this solver's
 * previous md_spme_step left, if nothing has changed the context since (no
 * other call launched work on it and its pair parameters are the same), and
 * are recomputed otherwise.  Library kernels of the solver count in
 * md_launch_count.  energy:
 * host array of 4 (may be NULL) for the final state: LJ PE, Coulomb energy
 * (real + reciprocal + self + background), kinetic energy, total.  The
 * context's own thermo records keep describing LJ only; after this call
 * md_get_state's forces and md_step recompute LJ-only forces.  Synchronises the
 * context's stream once per rebuild and at the end.  Errors: MD_ERR_ARG, and
 * those of the context's sort, list build and forces (MD_ERR_NONFINITE,
 * MD_ERR_NEIGH_OVERFLOW, MD_ERR_TIMEOUT, MD_ERR_CUDA). */
md_status md_spme_step(md_spme *s, int32_t nsteps, double *energy);

/* Per-kernel device times of the last md_spme_compute, in ms, measured with
 * CUDA events on the context's stream when `on` was set by md_spme_profile:
 * ms[0] charge spread, [1] forward FFT, [2] influence (energy + multiply),
 * [3] inverse FFT, [4] gather (+ force output), [5] real-space pairs.
 * Profiling adds event records between the launches; off by default. */
md_status md_spme_profile(md_spme *s, int32_t on);
md_status md_spme_profile_read(md_spme *s, double *ms /* 6 */);

/* Message of the last failed call on s (NULL: of the last failed create). */
const char *md_spme_last_error(const md_spme *s);

/* Frees the solver (NULL is a no-op).  It may run after md_destroy of its
 * context: it uses only its own buffers and the stream handles. */
void md_spme_destroy(md_spme *s);

#ifdef __cplusplus
}
#endif

#endif

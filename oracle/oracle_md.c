/*
 * oracle_md.c -- plain, slow, FP64 CPU oracle for the short-range
 * Lennard-Jones molecular-dynamics timestep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it is used by tests/, by the smoke check and by the benchmark's CPU-baseline
 * leg.  It shares no code, header or table with the CUDA library.
 *
 * What it follows.  The paper (arXiv 2109.09056) describes the MD timestep as
 * "neighbor list -> forces -> propagate -> resort" (Introduction, anatomy of a
 * timestep, Fig. 1), neighbor lists built by traditional binning (Verlet lists,
 * Section "Neighbor List Creation"), particle sorting by geometric binning
 * (Section "Particle Sorting"), and names the Lennard-Jones short-range kernel
 * as CabanaMD's benchmark (Section "CabanaMD").  It prints no formula for any
 * of these, so each function below is the textbook definition, with every
 * choice the paper leaves open fixed as stated in its comment.
 *
 * Parity status: no value here comes from the paper (it prints none for this
 * path).  Every function is pinned by closed forms, invariants, brute force or
 * finite differences in tests/test_oracle_*.py.
 *
 * Arrays: positions/velocities/forces are n x 3, row-major (AoS), float64.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so every product and sum is a separately rounded IEEE operation).
 * OpenMP only splits independent per-atom loops; every total is summed
 * serially in atom order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_BOX 1       /* some L[d] <= 2 * (rc + skin) */
#define ORACLE_ERR_ALLOC 2
#define ORACLE_ERR_ARG 3
/* a negative return -k from a list builder means "capacity too small, need k" */

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------
 * Cell grid.  nc[d] = floor(L[d] / rs) cells per axis, so every cell edge is
 * at least rs = rc + skin and the 27-cell stencil holds every pair closer than
 * rs.  A box with L <= 2 rs is rejected: the nearest periodic image of a pair
 * within rs would not be unique.
 * ------------------------------------------------------------------------ */
int oracle_cell_grid(const double L[3], double rs, int32_t nc[3]) {
    for (int d = 0; d < 3; ++d) {
        if (!(L[d] > 2.0 * rs)) return ORACLE_ERR_BOX;
        nc[d] = (int32_t)floor(L[d] / rs);
    }
    return ORACLE_OK;
}

/* Wrap one coordinate into [0, L): w = x - L*floor(x/L) (each op rounded);
 * a result below 0 gets +L, a result at or above L gets -L.  *shift receives
 * the number of box lengths removed, so x ~= w + shift*L. */
static double wrap1(double x, double L, int32_t *shift) {
    double q = floor(x / L);
    double p = L * q;
    double w = x - p;
    int32_t k = (int32_t)q;
    if (w < 0.0) { w = w + L; k -= 1; }
    if (w >= L) { w = w - L; k += 1; }
    *shift = k;
    return w;
}

/* Wrap all positions in place; img (n x 3, may be NULL) accumulates the
 * number of box lengths each coordinate was shifted by. */
void oracle_wrap(int64_t n, double *x, int32_t *img, const double L[3]) {
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            int32_t k;
            x[3 * i + d] = wrap1(x[3 * i + d], L[d], &k);
            if (img) img[3 * i + d] += k;
        }
}

/* Cell of each (wrapped) atom: c_d = (int)(x_d * (nc_d / L_d)) clamped to
 * [0, nc_d - 1], with nc_d / L_d computed once in FP64; the linear cell id is
 * c = (c_z * nc_y + c_y) * nc_x + c_x. */
void oracle_cell_index(int64_t n, const double *x, const double L[3],
                       const int32_t nc[3], int32_t *cell) {
    double inv[3];
    for (int d = 0; d < 3; ++d) inv[d] = (double)nc[d] / L[d];
    for (int64_t i = 0; i < n; ++i) {
        int32_t c[3];
        for (int d = 0; d < 3; ++d) {
            double t = x[3 * i + d] * inv[d];
            int32_t k = (int32_t)t;
            if (k < 0) k = 0;
            if (k > nc[d] - 1) k = nc[d] - 1;
            c[d] = k;
        }
        cell[i] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    }
}

/* Stable sort of atom indices by cell id (counting sort: histogram,
 * exclusive prefix sum, then placement in increasing prior index).
 * perm[new] = old. */
int oracle_stable_sort_by_cell(int64_t n, const int32_t *cell, int64_t ncell,
                               int32_t *perm) {
    int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!start) return ORACLE_ERR_ALLOC;
    for (int64_t i = 0; i < n; ++i) start[cell[i] + 1] += 1;
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    for (int64_t i = 0; i < n; ++i) perm[start[cell[i]]++] = (int32_t)i;
    free(start);
    return ORACLE_OK;
}

/* The canonical pair distance: d = x_j - x_i per axis, folded once to the
 * nearest image (d > L/2 -> d - L, d < -L/2 -> d + L), then
 * r^2 = (dx*dx + dy*dy) + dz*dz, every operation separately rounded. */
static double canonical_r2(const double *xi, const double *xj, const double L[3]) {
    double d[3];
    for (int a = 0; a < 3; ++a) {
        double t = xj[a] - xi[a];
        double h = 0.5 * L[a];
        if (t > h) t = t - L[a];
        else if (t < -h) t = t + L[a];
        d[a] = t;
    }
    double sx = d[0] * d[0];
    double sy = d[1] * d[1];
    double sz = d[2] * d[2];
    return (sx + sy) + sz;
}

/* Nearest-image separation x_i - x_j (the vector the force on i points along). */
static void min_image(const double *xi, const double *xj, const double L[3], double d[3]) {
    for (int a = 0; a < 3; ++a) {
        double t = xi[a] - xj[a];
        double h = 0.5 * L[a];
        if (t > h) t = t - L[a];
        else if (t < -h) t = t + L[a];
        d[a] = t;
    }
}

/* Full Verlet list by binning: for each atom i, every j != i with canonical
 * r^2 < rs^2 (strict), searched over the 27 cells around i's cell; when an
 * axis has fewer than 3 cells the stencil offsets are deduplicated modulo nc
 * so each cell is visited once.  Row i of nbr (capacity maxnb) lists the
 * neighbors in visiting order; nn[i] is the count.  Returns -max_count if
 * some row needs more than maxnb entries (rows are then truncated). */
int oracle_neighbors_cells(int64_t n, const double *x, const double L[3],
                           const int32_t nc[3], double rs, int32_t maxnb,
                           int32_t *nn, int32_t *nbr) {
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!cell || !order || !start) { free(cell); free(order); free(start); return ORACLE_ERR_ALLOC; }
    oracle_cell_index(n, x, L, nc, cell);
    for (int64_t i = 0; i < n; ++i) start[cell[i] + 1] += 1;
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
        if (!fill) { free(cell); free(order); free(start); return ORACLE_ERR_ALLOC; }
        memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
        for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = (int32_t)i;
        free(fill);
    }
    const double rs2 = rs * rs;
    int32_t worst = 0;
#pragma omp parallel for schedule(static) reduction(max : worst)
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = cell[i];
        int32_t cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / (nc[0] * nc[1]);
        int32_t visited[27];
        int nvisited = 0;
        int32_t cnt = 0;
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    int32_t jx = (cx + ox + nc[0]) % nc[0];
                    int32_t jy = (cy + oy + nc[1]) % nc[1];
                    int32_t jz = (cz + oz + nc[2]) % nc[2];
                    int32_t jc = (jz * nc[1] + jy) * nc[0] + jx;
                    int seen = 0;
                    for (int v = 0; v < nvisited; ++v) seen |= (visited[v] == jc);
                    if (seen) continue;
                    visited[nvisited++] = jc;
                    for (int64_t s = start[jc]; s < start[jc + 1]; ++s) {
                        int32_t j = order[s];
                        if (j == i) continue;
                        if (canonical_r2(&x[3 * i], &x[3 * j], L) < rs2) {
                            if (cnt < maxnb) nbr[i * maxnb + cnt] = j;
                            cnt += 1;
                        }
                    }
                }
        nn[i] = cnt;
        if (cnt > worst) worst = cnt;
    }
    free(cell); free(order); free(start);
    return worst > maxnb ? -worst : ORACLE_OK;
}

/* The same list by brute force over all j != i (O(n^2)); rows in increasing j. */
int oracle_neighbors_brute(int64_t n, const double *x, const double L[3], double rs,
                           int32_t maxnb, int32_t *nn, int32_t *nbr) {
    const double rs2 = rs * rs;
    int32_t worst = 0;
#pragma omp parallel for schedule(static) reduction(max : worst)
    for (int64_t i = 0; i < n; ++i) {
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (canonical_r2(&x[3 * i], &x[3 * j], L) < rs2) {
                if (cnt < maxnb) nbr[i * maxnb + cnt] = (int32_t)j;
                cnt += 1;
            }
        }
        nn[i] = cnt;
        if (cnt > worst) worst = cnt;
    }
    return worst > maxnb ? -worst : ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Lennard-Jones 12-6 pair term for types (a, b), r^2 = u:
 *   U(r)   = 4 eps [ (sigma/r)^12 - (sigma/r)^6 ]
 *   F_i   += 24 eps / r^2 [ 2 (sigma/r)^12 - (sigma/r)^6 ] (x_i - x_j)
 * evaluated through r2inv = 1/u and s6 = (sigma^2 r2inv)^3.  Pairs interact
 * iff u < rc^2 (strict); the cutoff is absolute (not scaled by sigma).  With
 * shift != 0 the energy of each interacting pair is U(r) - U(rc); forces are
 * the same either way.
 * ------------------------------------------------------------------------ */
static void lj_pair(double u, double eps, double sig, double rc, int shift,
                    double *phi, double *U) {
    double r2inv = 1.0 / u;
    double s2 = (sig * sig) * r2inv;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    *phi = 24.0 * eps * r2inv * (2.0 * s12 - s6);
    double e = 4.0 * eps * (s12 - s6);
    if (shift) {
        double c2 = (sig * sig) / (rc * rc);
        double c6 = c2 * c2 * c2;
        e -= 4.0 * eps * (c6 * c6 - c6);
    }
    *U = e;
}

/* Forces and energies over a full neighbor list (rows of capacity maxnb).
 * f (n x 3) is overwritten; e_atom (n, may be NULL) gets e_i = 1/2 sum_j U_ij;
 * *pe gets PE = sum_i e_i summed in atom order (= sum over pairs i<j of U). */
void oracle_lj_forces(int64_t n, const double *x, const int32_t *type, const double L[3],
                      int32_t ntypes, const double *eps, const double *sigma, double rc,
                      int shift, const int32_t *nn, const int32_t *nbr, int32_t maxnb,
                      double *f, double *e_atom, double *pe) {
    const double rc2 = rc * rc;
    double *ea = e_atom ? e_atom : (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        double ei = 0.0;
        for (int32_t k = 0; k < nn[i]; ++k) {
            int32_t j = nbr[i * maxnb + k];
            double d[3];
            min_image(&x[3 * i], &x[3 * j], L, d);
            double u = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(u < rc2)) continue;
            int32_t ab = type[i] * ntypes + type[j];
            double phi, U;
            lj_pair(u, eps[ab], sigma[ab], rc, shift, &phi, &U);
            for (int a = 0; a < 3; ++a) fi[a] += phi * d[a];
            ei += 0.5 * U;
        }
        for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
        ea[i] = ei;
    }
    double tot = 0.0;
    for (int64_t i = 0; i < n; ++i) tot += ea[i];
    if (pe) *pe = tot;
    if (!e_atom) free(ea);
}

/* Forces and energies by brute force over all pairs j != i (no list). */
void oracle_lj_forces_brute(int64_t n, const double *x, const int32_t *type,
                            const double L[3], int32_t ntypes, const double *eps,
                            const double *sigma, double rc, int shift, double *f,
                            double *e_atom, double *pe) {
    const double rc2 = rc * rc;
    double *ea = e_atom ? e_atom : (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        double ei = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], L, d);
            double u = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(u < rc2)) continue;
            int32_t ab = type[i] * ntypes + type[j];
            double phi, U;
            lj_pair(u, eps[ab], sigma[ab], rc, shift, &phi, &U);
            for (int a = 0; a < 3; ++a) fi[a] += phi * d[a];
            ei += 0.5 * U;
        }
        for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
        ea[i] = ei;
    }
    double tot = 0.0;
    for (int64_t i = 0; i < n; ++i) tot += ea[i];
    if (pe) *pe = tot;
    if (!e_atom) free(ea);
}

/* Thermodynamics: KE = sum 1/2 m v^2, momentum P = sum m v (out[2..4]),
 * T = 2 KE / (3n - 3) (k_B = 1, centre-of-mass motion removed). */
void oracle_thermo(int64_t n, const double *v, const int32_t *type, const double *mass,
                   double out[5]) {
    double ke = 0.0, p[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        double m = mass[type[i]];
        double v2 = (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1]) + v[3 * i + 2] * v[3 * i + 2];
        ke += 0.5 * m * v2;
        for (int a = 0; a < 3; ++a) p[a] += m * v[3 * i + a];
    }
    out[0] = ke;
    out[1] = n > 1 ? 2.0 * ke / (3.0 * (double)n - 3.0) : 0.0;
    out[2] = p[0]; out[3] = p[1]; out[4] = p[2];
}

/* Wrap, bin and stably re-sort the whole state into cell order (the
 * "resort" step of the timestep); perm_out (n, may be NULL) gets perm[new]=old. */
static int resort(int64_t n, double *x, double *v, int32_t *type, int32_t *id, int32_t *img,
                  const double L[3], const int32_t nc[3], int32_t *perm_out) {
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * nn);
    double *tmp = (double *)malloc(sizeof(double) * 3 * nn);
    int32_t *itmp = (int32_t *)malloc(sizeof(int32_t) * 3 * nn);
    if (!cell || !perm || !tmp || !itmp) { free(cell); free(perm); free(tmp); free(itmp); return ORACLE_ERR_ALLOC; }
    oracle_wrap(n, x, img, L);
    oracle_cell_index(n, x, L, nc, cell);
    int rc = oracle_stable_sort_by_cell(n, cell, ncell, perm);
    if (rc == ORACLE_OK) {
        for (int64_t k = 0; k < n; ++k) memcpy(&tmp[3 * k], &x[3 * perm[k]], 3 * sizeof(double));
        memcpy(x, tmp, 3 * (size_t)n * sizeof(double));
        for (int64_t k = 0; k < n; ++k) memcpy(&tmp[3 * k], &v[3 * perm[k]], 3 * sizeof(double));
        memcpy(v, tmp, 3 * (size_t)n * sizeof(double));
        for (int64_t k = 0; k < n; ++k) itmp[k] = type[perm[k]];
        memcpy(type, itmp, (size_t)n * sizeof(int32_t));
        for (int64_t k = 0; k < n; ++k) itmp[k] = id[perm[k]];
        memcpy(id, itmp, (size_t)n * sizeof(int32_t));
        if (img) {
            for (int64_t k = 0; k < n; ++k) memcpy(&itmp[3 * k], &img[3 * perm[k]], 3 * sizeof(int32_t));
            memcpy(img, itmp, 3 * (size_t)n * sizeof(int32_t));
        }
        if (perm_out) memcpy(perm_out, perm, (size_t)n * sizeof(int32_t));
    }
    free(cell); free(perm); free(tmp); free(itmp);
    return rc;
}

/* Velocity-Verlet NVE run ("forces are calculated to propagate the particles
 * to new positions; the particles are then resorted", Introduction).
 *
 * Entry: (x, v) at step counter step0.  If step0 % rebuild_every == 0 the
 * state is first wrapped, re-sorted into cell order and a list built;
 * otherwise a list is built on the current order.  Forces at entry are then
 * computed.  Each of the nsteps steps is
 *     v += (dt/2) F/m;  x += dt v;
 *     if (step % rebuild_every == 0) wrap + stable cell re-sort + new list;
 *     F = F(x);  v += (dt/2) F/m
 * with `step` the counter after the step.  The list holds pairs closer than
 * rc + skin; forces use only pairs closer than rc.
 *
 * All arrays are in the oracle's internal (cell) order on return; id[] maps
 * each row to its original atom.  thermo_out (may be NULL) receives, for
 * entry and each step, 4 numbers: PE, KE, Etot, max |x - x_at_last_build|.
 * Returns 0, ORACLE_ERR_*, or -k when a list row needed k > maxnb slots. */
int oracle_md_run(int64_t n, double *x, double *v, double *f, int32_t *type, int32_t *id,
                  int32_t *img, const double L[3], int32_t ntypes, const double *eps,
                  const double *sigma, const double *mass, double rc, double skin, double dt,
                  int32_t rebuild_every, int shift, int64_t step0, int32_t nsteps,
                  int32_t maxnb, double *thermo_out) {
    int32_t nc[3];
    if (n < 1 || rebuild_every < 1 || maxnb < 1) return ORACLE_ERR_ARG;
    int rc_ = oracle_cell_grid(L, rc + skin, nc);
    if (rc_) return rc_;
    size_t nn_ = (size_t)n;
    int32_t *nn = (int32_t *)malloc(sizeof(int32_t) * nn_);
    int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * nn_ * (size_t)maxnb);
    double *xb = (double *)malloc(sizeof(double) * 3 * nn_);
    if (!nn || !nbr || !xb) { free(nn); free(nbr); free(xb); return ORACLE_ERR_ALLOC; }
    int status = ORACLE_OK;
    double pe = 0.0;
    if (step0 % rebuild_every == 0) {
        status = resort(n, x, v, type, id, img, L, nc, NULL);
        if (status) goto done;
    }
    status = oracle_neighbors_cells(n, x, L, nc, rc + skin, maxnb, nn, nbr);
    if (status) goto done;
    memcpy(xb, x, 3 * nn_ * sizeof(double));
    oracle_lj_forces(n, x, type, L, ntypes, eps, sigma, rc, shift, nn, nbr, maxnb, f, NULL, &pe);
    for (int32_t s = 0; s <= nsteps; ++s) {
        if (s > 0) {
            int64_t step = step0 + s;
            for (int64_t i = 0; i < n; ++i) {
                double hm = 0.5 * dt / mass[type[i]];
                for (int a = 0; a < 3; ++a) {
                    v[3 * i + a] = v[3 * i + a] + hm * f[3 * i + a];
                    x[3 * i + a] = x[3 * i + a] + dt * v[3 * i + a];
                }
            }
            if (step % rebuild_every == 0) {
                status = resort(n, x, v, type, id, img, L, nc, NULL);
                if (status) goto done;
                status = oracle_neighbors_cells(n, x, L, nc, rc + skin, maxnb, nn, nbr);
                if (status) goto done;
                memcpy(xb, x, 3 * nn_ * sizeof(double));
            }
            oracle_lj_forces(n, x, type, L, ntypes, eps, sigma, rc, shift, nn, nbr, maxnb, f, NULL, &pe);
            for (int64_t i = 0; i < n; ++i) {
                double hm = 0.5 * dt / mass[type[i]];
                for (int a = 0; a < 3; ++a) v[3 * i + a] = v[3 * i + a] + hm * f[3 * i + a];
            }
        }
        if (thermo_out) {
            double th[5];
            oracle_thermo(n, v, type, mass, th);
            double dmax = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double t = x[3 * i + a] - xb[3 * i + a];
                    d2 += t * t;
                }
                if (d2 > dmax) dmax = d2;
            }
            thermo_out[4 * s + 0] = pe;
            thermo_out[4 * s + 1] = th[0];
            thermo_out[4 * s + 2] = pe + th[0];
            thermo_out[4 * s + 3] = sqrt(dmax);
        }
    }
done:
    free(nn); free(nbr); free(xb);
    return status;
}

/* ------------------------------------------------------------------------
 * Force-matching adjoint.  Given G = dL/dF (n x 3) and gE = dL/dE, returns
 * dL/dx (n x 3) and dL/d eps, dL/d sigma (ntypes x ntypes, symmetric: the
 * entry (a,b) = (b,a) is the derivative with respect to the one parameter that
 * the symmetric table holds for the unordered type pair {a,b}).
 *
 * With d = x_i - x_j (nearest image), u = |d|^2, s6 = sigma^6/u^3, s12 = s6^2:
 *   phi(u)   = (24 eps / u)(2 s12 - s6),           F_i = sum_j phi_ij d_ij
 *   dphi/du  = (24 eps / u^2)(4 s6 - 14 s12),      psi = 2 dphi/du
 *   M_ij     = phi I + psi d d^T  (= dF_i/dx_i contribution; dF_i/dx_j = -M_ij)
 *   dL/dx_k  = sum_{j in nbr(k)} M_kj (G_k - G_j) - gE F_k
 *   dphi/deps = phi/eps,   dphi/dsigma = (24 eps/u)(24 s12 - 6 s6)/sigma
 *   dU/deps   = U/eps,     dU/dsigma   = 4 eps (12 s12 - 6 s6)/sigma
 *   dL/dtheta = sum_{ordered (i,j)} (G_i . d_ij) dphi/dtheta
 *             + gE sum_{i<j} dU/dtheta    (minus dU(rc)/dtheta when shifted)
 * The list used is the full list of pairs closer than rc (brute-force search
 * over all j when nbr == NULL, else the given rs-list filtered to rc).
 * ------------------------------------------------------------------------ */
void oracle_lj_adjoint(int64_t n, const double *x, const int32_t *type, const double L[3],
                       int32_t ntypes, const double *eps, const double *sigma, double rc,
                       int shift, const int32_t *nn, const int32_t *nbr, int32_t maxnb,
                       const double *G, double gE, double *dLdx, double *dLdeps,
                       double *dLdsig) {
    const double rc2 = rc * rc;
    const int32_t nt2 = ntypes * ntypes;
    /* per-atom, per-ordered-type-pair partials, summed serially afterwards */
    double *pe_ = (double *)calloc((size_t)(n > 0 ? n : 1) * (size_t)nt2 * 2, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double gx[3] = {0.0, 0.0, 0.0};
        double fi[3] = {0.0, 0.0, 0.0};
        int64_t cnt = nbr ? nn[i] : n;
        for (int64_t k = 0; k < cnt; ++k) {
            int64_t j = nbr ? nbr[i * maxnb + k] : k;
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], L, d);
            double u = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(u < rc2)) continue;
            int32_t ab = type[i] * ntypes + type[j];
            double e = eps[ab], s = sigma[ab];
            double s2 = (s * s) / u;
            double s6 = s2 * s2 * s2, s12 = s6 * s6;
            double phi = (24.0 * e / u) * (2.0 * s12 - s6);
            double dphidu = (24.0 * e / (u * u)) * (4.0 * s6 - 14.0 * s12);
            double psi = 2.0 * dphidu;
            double Gd[3], dG = 0.0, dGi = 0.0;
            for (int a = 0; a < 3; ++a) {
                Gd[a] = G[3 * i + a] - G[3 * j + a];
                dG += d[a] * Gd[a];
                dGi += d[a] * G[3 * i + a];
            }
            for (int a = 0; a < 3; ++a) {
                gx[a] += phi * Gd[a] + psi * d[a] * dG;
                fi[a] += phi * d[a];
            }
            double U = 4.0 * e * (s12 - s6);
            double dphide = phi / e;
            double dphids = (24.0 * e / u) * (24.0 * s12 - 6.0 * s6) / s;
            double dUde = U / e;
            double dUds = 4.0 * e * (12.0 * s12 - 6.0 * s6) / s;
            if (shift) {
                double c2 = (s * s) / rc2, c6 = c2 * c2 * c2, c12 = c6 * c6;
                dUde -= 4.0 * (c12 - c6);
                dUds -= 4.0 * e * (12.0 * c12 - 6.0 * c6) / s;
            }
            double *row = &pe_[((size_t)i * nt2 + ab) * 2];
            row[0] += dGi * dphide + 0.5 * gE * dUde;
            row[1] += dGi * dphids + 0.5 * gE * dUds;
        }
        for (int a = 0; a < 3; ++a) dLdx[3 * i + a] = gx[a] - gE * fi[a];
    }
    double *acc = (double *)calloc((size_t)nt2 * 2, sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int32_t ab = 0; ab < nt2; ++ab) {
            acc[2 * ab] += pe_[((size_t)i * nt2 + ab) * 2];
            acc[2 * ab + 1] += pe_[((size_t)i * nt2 + ab) * 2 + 1];
        }
    for (int32_t a = 0; a < ntypes; ++a)
        for (int32_t b = 0; b < ntypes; ++b) {
            int32_t ab = a * ntypes + b, ba = b * ntypes + a;
            if (a == b) {
                dLdeps[ab] = acc[2 * ab];
                dLdsig[ab] = acc[2 * ab + 1];
            } else {
                dLdeps[ab] = acc[2 * ab] + acc[2 * ba];
                dLdsig[ab] = acc[2 * ab + 1] + acc[2 * ba + 1];
            }
        }
    free(acc);
    free(pe_);
}

/* ------------------------------------------------------------------------
 * Sampled outputs for systems too large to list in full: for each of the m
 * atoms idx[s], its force (by brute force over all j, pairs closer than rc)
 * and its neighbor row (all j with canonical r^2 < rs^2, increasing j).
 * Same definitions as oracle_lj_forces_brute / oracle_neighbors_brute.
 * ------------------------------------------------------------------------ */
void oracle_lj_forces_sample(int64_t n, const double *x, const int32_t *type, const double L[3],
                             int32_t ntypes, const double *eps, const double *sigma, double rc,
                             int shift, int64_t m, const int64_t *idx, double *f, double *e_atom) {
    const double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic)
    for (int64_t s = 0; s < m; ++s) {
        const int64_t i = idx[s];
        double fi[3] = {0.0, 0.0, 0.0};
        double ei = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], L, d);
            double u = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(u < rc2)) continue;
            int32_t ab = type[i] * ntypes + type[j];
            double phi, U;
            lj_pair(u, eps[ab], sigma[ab], rc, shift, &phi, &U);
            for (int a = 0; a < 3; ++a) fi[a] += phi * d[a];
            ei += 0.5 * U;
        }
        for (int a = 0; a < 3; ++a) f[3 * s + a] = fi[a];
        if (e_atom) e_atom[s] = ei;
    }
}

int oracle_neighbors_sample(int64_t n, const double *x, const double L[3], double rs, int64_t m,
                            const int64_t *idx, int32_t maxnb, int32_t *nn, int32_t *nbr) {
    const double rs2 = rs * rs;
    int32_t worst = 0;
#pragma omp parallel for schedule(dynamic) reduction(max : worst)
    for (int64_t s = 0; s < m; ++s) {
        const int64_t i = idx[s];
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (canonical_r2(&x[3 * i], &x[3 * j], L) < rs2) {
                if (cnt < maxnb) nbr[s * maxnb + cnt] = (int32_t)j;
                cnt += 1;
            }
        }
        nn[s] = cnt;
        if (cnt > worst) worst = cnt;
    }
    return worst > maxnb ? -worst : ORACLE_OK;
}

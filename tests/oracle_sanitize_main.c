/* Memory-safety and undefined-behaviour run of the C oracle (test
 * infrastructure).  tests/test_oracle_sanitize.py compiles this driver
 * together with oracle/oracle_md.c under AddressSanitizer and
 * UndefinedBehaviorSanitizer (no recovery: the first finding aborts) and runs
 * it.  The driver calls every exported oracle function on small seeded
 * systems, including the edge cases of the definitions: boxes with 2 and 3
 * cells per axis (deduplicated stencils), atoms outside the box before the
 * wrap, a neighbor capacity too small for the rows (truncated rows, reported
 * overflow), two atom types, one atom, and empty cells.  Alongside the
 * sanitizers it checks the oracle's own consistency (cell list == brute
 * force, list forces == brute-force forces, sampled rows == full rows), so a
 * silent out-of-bounds read that changes a result also fails.  Prints "ok"
 * and exits 0 on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_cell_grid(const double L[3], double rs, int32_t nc[3]);
void oracle_wrap(int64_t n, double *x, int32_t *img, const double L[3]);
void oracle_cell_index(int64_t n, const double *x, const double L[3], const int32_t nc[3],
                       int32_t *cell);
int oracle_stable_sort_by_cell(int64_t n, const int32_t *cell, int64_t ncell, int32_t *perm);
int oracle_neighbors_cells(int64_t n, const double *x, const double L[3], const int32_t nc[3],
                           double rs, int32_t maxnb, int32_t *nn, int32_t *nbr);
int oracle_neighbors_brute(int64_t n, const double *x, const double L[3], double rs,
                           int32_t maxnb, int32_t *nn, int32_t *nbr);
void oracle_lj_forces(int64_t n, const double *x, const int32_t *type, const double L[3],
                      int32_t ntypes, const double *eps, const double *sigma, double rc,
                      int shift, const int32_t *nn, const int32_t *nbr, int32_t maxnb,
                      double *f, double *e_atom, double *pe);
void oracle_lj_forces_brute(int64_t n, const double *x, const int32_t *type, const double L[3],
                            int32_t ntypes, const double *eps, const double *sigma, double rc,
                            int shift, double *f, double *e_atom, double *pe);
void oracle_thermo(int64_t n, const double *v, const int32_t *type, const double *mass,
                   double out[5]);
int oracle_md_run(int64_t n, double *x, double *v, double *f, int32_t *type, int32_t *id,
                  int32_t *img, const double L[3], int32_t ntypes, const double *eps,
                  const double *sigma, const double *mass, double rc, double skin, double dt,
                  int32_t rebuild_every, int shift, int64_t step0, int32_t nsteps,
                  int32_t maxnb, double *thermo_out);
void oracle_lj_adjoint(int64_t n, const double *x, const int32_t *type, const double L[3],
                       int32_t ntypes, const double *eps, const double *sigma, double rc,
                       int shift, const int32_t *nn, const int32_t *nbr, int32_t maxnb,
                       const double *G, double gE, double *dLdx, double *dLdeps, double *dLdsig);
void oracle_lj_forces_sample(int64_t n, const double *x, const int32_t *type, const double L[3],
                             int32_t ntypes, const double *eps, const double *sigma, double rc,
                             int shift, int64_t m, const int64_t *idx, double *f,
                             double *e_atom);
int oracle_neighbors_sample(int64_t n, const double *x, const double L[3], double rs, int64_t m,
                            const int64_t *idx, int32_t maxnb, int32_t *nn, int32_t *nbr);

static int failures = 0;
#define CHECK(cond, ...)                                   \
    do {                                                   \
        if (!(cond)) {                                     \
            fprintf(stderr, "check failed: " __VA_ARGS__); \
            fprintf(stderr, "\n");                         \
            ++failures;                                    \
        }                                                  \
    } while (0)

/* splitmix64 for the inputs (the inputs only; no oracle arithmetic) */
static uint64_t rng_state = 0x2109090560ull;
static double uniform(void) {
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

static double *xmalloc_d(size_t k) { return (double *)calloc(k ? k : 1, sizeof(double)); }
static int32_t *xmalloc_i(size_t k) { return (int32_t *)calloc(k ? k : 1, sizeof(int32_t)); }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* FCC lattice of m^3 cells at density rho with a uniform jitter; a few atoms
 * pushed outside the box so that the wrap has work to do. */
static double fcc(int m, double rho, double jitter, double *x) {
    const int64_t n = 4LL * m * m * m;
    const double L = cbrt((double)n / rho), a = L / m;
    static const double basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    int64_t k = 0;
    for (int iz = 0; iz < m; ++iz)
        for (int iy = 0; iy < m; ++iy)
            for (int ix = 0; ix < m; ++ix)
                for (int b = 0; b < 4; ++b, ++k) {
                    const int c[3] = {ix, iy, iz};
                    for (int d = 0; d < 3; ++d)
                        x[3 * k + d] = (c[d] + basis[b][d]) * a + jitter * (2.0 * uniform() - 1.0);
                }
    for (int64_t i = 0; i < n; i += 17) x[3 * i] += (i % 2 ? 1.0 : -1.0) * L;
    return L;
}

/* One system through every oracle function. */
static void run_system(const char *name, int64_t n, double *x, const double L3[3], int ntypes) {
    const double rc = 2.5, skin = 0.3, rs = rc + skin;
    int32_t nc[3];
    if (oracle_cell_grid(L3, rs, nc)) {
        CHECK(0, "%s: box too small", name);
        return;
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *img = xmalloc_i(3 * (size_t)n), *cell = xmalloc_i((size_t)n),
            *perm = xmalloc_i((size_t)n), *type = xmalloc_i((size_t)n);
    oracle_wrap(n, x, img, L3);
    for (int64_t i = 0; i < 3 * n; ++i) CHECK(x[i] >= 0.0 && x[i] < L3[i % 3], "%s: wrap", name);
    oracle_cell_index(n, x, L3, nc, cell);
    CHECK(oracle_stable_sort_by_cell(n, cell, ncell, perm) == 0, "%s: sort", name);
    for (int64_t k = 1; k < n; ++k)
        CHECK(cell[perm[k - 1]] < cell[perm[k]] ||
                  (cell[perm[k - 1]] == cell[perm[k]] && perm[k - 1] < perm[k]),
              "%s: stable order", name);
    for (int64_t i = 0; i < n; ++i) type[i] = ntypes > 1 ? (int32_t)(i % ntypes) : 0;

    /* lists: cell search vs brute force (as sets), then a capacity too small */
    const int32_t maxnb = 160;
    int32_t *nn = xmalloc_i((size_t)n), *nbr = xmalloc_i((size_t)n * maxnb);
    int32_t *nn2 = xmalloc_i((size_t)n), *nbr2 = xmalloc_i((size_t)n * maxnb);
    CHECK(oracle_neighbors_cells(n, x, L3, nc, rs, maxnb, nn, nbr) == 0, "%s: cells", name);
    CHECK(oracle_neighbors_brute(n, x, L3, rs, maxnb, nn2, nbr2) == 0, "%s: brute", name);
    int32_t worst = 0;
    for (int64_t i = 0; i < n; ++i) {
        CHECK(nn[i] == nn2[i], "%s: count of atom %lld", name, (long long)i);
        if (nn[i] != nn2[i]) continue;
        if (nn[i] > worst) worst = nn[i];
        qsort(nbr + i * maxnb, (size_t)nn[i], sizeof(int32_t), cmp_i32);
        CHECK(memcmp(nbr + i * maxnb, nbr2 + i * maxnb, sizeof(int32_t) * (size_t)nn[i]) == 0,
              "%s: row of atom %lld", name, (long long)i);
    }
    if (worst > 4) {
        const int32_t small = worst / 2;
        int32_t *nbs = xmalloc_i((size_t)n * small), *nns = xmalloc_i((size_t)n);
        CHECK(oracle_neighbors_cells(n, x, L3, nc, rs, small, nns, nbs) == -worst,
              "%s: overflow report (cells)", name);
        CHECK(oracle_neighbors_brute(n, x, L3, rs, small, nns, nbs) == -worst,
              "%s: overflow report (brute)", name);
        free(nbs);
        free(nns);
    }

    /* forces: list vs brute force; sampled forces and rows vs the full ones */
    double eps[4] = {1.0, 0.9, 0.9, 1.1}, sig[4] = {1.0, 1.05, 1.05, 0.95}, mass[2] = {1.0, 2.0};
    double *f = xmalloc_d(3 * (size_t)n), *f2 = xmalloc_d(3 * (size_t)n);
    double *ea = xmalloc_d((size_t)n), pe = 0.0, pe2 = 0.0;
    for (int shift = 0; shift < 2; ++shift) {
        oracle_lj_forces(n, x, type, L3, ntypes, eps, sig, rc, shift, nn2, nbr2, maxnb, f, ea, &pe);
        oracle_lj_forces(n, x, type, L3, ntypes, eps, sig, rc, shift, nn2, nbr2, maxnb, f, NULL,
                         &pe2);
        CHECK(pe == pe2, "%s: pe with and without e_atom", name);
        oracle_lj_forces_brute(n, x, type, L3, ntypes, eps, sig, rc, shift, f2, NULL, &pe2);
        CHECK(fabs(pe - pe2) <= 1e-12 * fabs(pe) + 1e-12, "%s: pe list vs brute", name);
        for (int64_t k = 0; k < 3 * n; ++k)
            CHECK(fabs(f[k] - f2[k]) <= 1e-10 * (1.0 + fabs(f2[k])), "%s: force", name);
    }
    const int64_t m = n < 7 ? n : 7;
    int64_t idx[7];
    for (int64_t s = 0; s < m; ++s) idx[s] = (s * 37) % n;
    double fs[21], es[7];
    oracle_lj_forces_sample(n, x, type, L3, ntypes, eps, sig, rc, 1, m, idx, fs, es);
    for (int64_t s = 0; s < m; ++s)
        for (int d = 0; d < 3; ++d)
            CHECK(fs[3 * s + d] == f2[3 * idx[s] + d], "%s: sampled force", name);
    int32_t nns[7], *nbs = xmalloc_i(7 * (size_t)maxnb);
    CHECK(oracle_neighbors_sample(n, x, L3, rs, m, idx, maxnb, nns, nbs) == 0, "%s: sample rows",
          name);
    for (int64_t s = 0; s < m; ++s) {
        CHECK(nns[s] == nn2[idx[s]], "%s: sampled count", name);
        CHECK(memcmp(nbs + s * maxnb, nbr2 + idx[s] * maxnb, sizeof(int32_t) * (size_t)nns[s]) == 0,
              "%s: sampled row", name);
    }

    /* adjoint over the list and by brute force (nbr == NULL) */
    double *G = xmalloc_d(3 * (size_t)n), *g1 = xmalloc_d(3 * (size_t)n),
           *g2 = xmalloc_d(3 * (size_t)n);
    double de1[4], ds1[4], de2[4], ds2[4];
    for (int64_t k = 0; k < 3 * n; ++k) G[k] = 2.0 * uniform() - 1.0;
    oracle_lj_adjoint(n, x, type, L3, ntypes, eps, sig, rc, 1, nn2, nbr2, maxnb, G, 0.5, g1, de1,
                      ds1);
    oracle_lj_adjoint(n, x, type, L3, ntypes, eps, sig, rc, 1, NULL, NULL, 0, G, 0.5, g2, de2, ds2);
    for (int64_t k = 0; k < 3 * n; ++k)
        CHECK(fabs(g1[k] - g2[k]) <= 1e-9 * (1.0 + fabs(g2[k])), "%s: adjoint dL/dx", name);
    for (int q = 0; q < ntypes * ntypes; ++q)
        CHECK(fabs(de1[q] - de2[q]) <= 1e-9 * (1.0 + fabs(de2[q])) &&
                  fabs(ds1[q] - ds2[q]) <= 1e-9 * (1.0 + fabs(ds2[q])),
              "%s: adjoint parameters", name);

    /* a short run with re-sorts and rebuilds, then thermo */
    double *v = xmalloc_d(3 * (size_t)n), th[5];
    for (int64_t k = 0; k < 3 * n; ++k) v[k] = 0.5 * (2.0 * uniform() - 1.0);
    int32_t *id = xmalloc_i((size_t)n);
    for (int64_t i = 0; i < n; ++i) id[i] = (int32_t)i;
    const int32_t nsteps = 9;
    double *thermo = xmalloc_d(4 * (size_t)(nsteps + 1));
    CHECK(oracle_md_run(n, x, v, f, type, id, img, L3, ntypes, eps, sig, mass, rc, skin, 0.002, 4,
                        1, 0, nsteps, maxnb, thermo) == 0,
          "%s: md run", name);
    for (int k = 0; k <= nsteps; ++k)
        CHECK(isfinite(thermo[4 * k + 2]), "%s: thermo row %d", name, k);
    oracle_thermo(n, v, type, mass, th);
    CHECK(isfinite(th[0]) && th[0] >= 0.0, "%s: kinetic energy", name);
    /* a capacity too small for the run (half the longest row of the state it
     * starts from): reported, nothing written past it */
    CHECK(oracle_neighbors_brute(n, x, L3, rs, maxnb, nn2, nbr2) == 0, "%s: brute", name);
    worst = 0;
    for (int64_t i = 0; i < n; ++i) worst = nn2[i] > worst ? nn2[i] : worst;
    if (worst > 4)
        CHECK(oracle_md_run(n, x, v, f, type, id, img, L3, ntypes, eps, sig, mass, rc, skin, 0.002,
                            4, 0, 0, 2, worst / 2, NULL) == -worst,
              "%s: md run overflow", name);

    free(img); free(cell); free(perm); free(type); free(nn); free(nbr); free(nn2); free(nbr2);
    free(f); free(f2); free(ea); free(nbs); free(G); free(g1); free(g2); free(v); free(id);
    free(thermo);
}

int main(void) {
    {   /* 4^3 FCC at rho 0.7: L = 7.15, 2 cells per axis (deduplicated stencil) */
        double *x = xmalloc_d(3 * 256);
        const double L = fcc(4, 0.7, 0.05, x);
        const double L3[3] = {L, L, L};
        run_system("fcc4", 256, x, L3, 1);
        free(x);
    }
    {   /* 6^3 FCC at rho 0.8442: 3 cells per axis, two types */
        double *x = xmalloc_d(3 * 864);
        const double L = fcc(6, 0.8442, 0.1, x);
        const double L3[3] = {L, L, L};
        run_system("fcc6", 864, x, L3, 2);
        free(x);
    }
    {   /* 151 random atoms, no two closer than 0.85, in the lower half (y) of an
         * orthorhombic box, so that the upper cells are empty */
        const int64_t n = 151;
        double *x = xmalloc_d(3 * (size_t)n);
        const double L3[3] = {9.0, 11.5, 6.0};
        for (int64_t i = 0; i < n;) {
            for (int d = 0; d < 3; ++d) x[3 * i + d] = (d == 1 ? 0.5 : 1.0) * L3[d] * uniform();
            int clash = 0;
            for (int64_t j = 0; j < i && !clash; ++j) {
                double r2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double t = x[3 * i + d] - x[3 * j + d];
                    t -= L3[d] * round(t / L3[d]);
                    r2 += t * t;
                }
                clash = r2 < 0.85 * 0.85;
            }
            if (!clash) ++i;
        }
        run_system("random", n, x, L3, 2);
        free(x);
    }
    {   /* one atom: no neighbors, zero force */
        double x[3] = {1.0, 2.0, 3.0};
        const double L3[3] = {6.0, 6.0, 6.0};
        run_system("single", 1, x, L3, 1);
    }
    {   /* a box too small is reported, not run */
        int32_t nc[3];
        const double L3[3] = {5.0, 9.0, 9.0};
        CHECK(oracle_cell_grid(L3, 2.8, nc) != 0, "small box");
    }
    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("ok\n");
    return 0;
}

/* Host-side AddressSanitizer / UndefinedBehaviorSanitizer run of the C ABI's
 * argument checking and error paths (test infrastructure).
 * tests/test_abi_sanitize.py links this driver against a variant of
 * libmd_b300 whose host code is compiled with the sanitizers, and runs it on
 * a machine without a GPU.  Every call below is rejected before any device
 * work: NULL handles and pointers, out-of-range parameters, boxes too small,
 * too many cells, host pointers where device memory is required.  With the
 * argument "create" the driver also makes one valid md_create call, which on
 * a machine without a GPU fails in the CUDA runtime and must clean up its
 * partly built context (MD_ERR_CUDA).  Each rejection must return the
 * documented status and leave a message in the matching last-error call.
 * Prints "ok" and exits 0 on success. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "md.h"
#include "md_spme.h"

static int failures = 0;
#define EXPECT(call, want)                                                                  \
    do {                                                                                    \
        md_status got_ = (call);                                                            \
        if (got_ != (want)) {                                                               \
            fprintf(stderr, "line %d: %s returned %d, expected %d\n", __LINE__, #call,     \
                    (int)got_, (int)(want));                                                \
            ++failures;                                                                     \
        }                                                                                   \
    } while (0)
#define MSG(s)                                                                \
    do {                                                                      \
        const char *m_ = (s);                                                 \
        if (!m_ || !m_[0]) {                                                  \
            fprintf(stderr, "line %d: empty error message\n", __LINE__);     \
            ++failures;                                                       \
        }                                                                     \
    } while (0)

int main(int argc, char **argv) {
    const int try_create = argc > 1 && strcmp(argv[1], "create") == 0;
    md_params p;
    md_params_default(&p);
    if (p.ntypes != 1 || p.rc != 2.5 || p.skin != 0.3 || p.rebuild_every != 20 || !p.eps ||
        p.eps[0] != 1.0 || p.sigma[0] != 1.0 || p.mass[0] != 1.0) {
        fprintf(stderr, "md_params_default\n");
        ++failures;
    }
    const md_box box = {{10.0, 10.0, 10.0}};
    double x[6] = {1, 1, 1, 3, 3, 3}, v[6] = {0};
    int32_t ty[2] = {0, 0};
    md_ctx *c = (md_ctx *)0x1;

    /* md_create / md_batch_create: arguments checked before any device work */
    EXPECT(md_create(&box, 0, x, v, ty, &p, NULL, &c), MD_ERR_ARG);
    MSG(md_last_error(NULL));
    if (c != NULL) { fprintf(stderr, "out not cleared on n = 0\n"); ++failures; }
    EXPECT(md_create(&box, 2, x, v, ty, &p, NULL, NULL), MD_ERR_ARG);
    c = (md_ctx *)0x1;
    EXPECT(md_create(&box, 2, NULL, v, ty, &p, NULL, &c), MD_ERR_ARG);
    if (c != NULL) { fprintf(stderr, "out not cleared on failure\n"); ++failures; }
    EXPECT(md_create(NULL, 2, x, v, ty, &p, NULL, &c), MD_ERR_ARG);
    EXPECT(md_create(&box, 2, x, v, ty, NULL, NULL, &c), MD_ERR_ARG);
    {
        md_params q = p;
        q.ntypes = 0;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q.ntypes = 9;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.eps = NULL;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.mass = NULL;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.rc = 0.0;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.rc = NAN;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.skin = -0.1;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.dt = INFINITY;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.rebuild_every = 0;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.precision = 7;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.lanes_per_atom = 3;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.block_threads = 100;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        q = p; q.block_threads = 800;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        const double bad_mass[1] = {-1.0};
        q = p; q.mass = bad_mass;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        const double neg_eps[1] = {-1.0};
        q = p; q.eps = neg_eps;
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        const double eps2[4] = {1.0, 0.5, 0.7, 1.0}, sig2[4] = {1, 1, 1, 1}, m2[2] = {1, 1};
        q = p; q.ntypes = 2; q.eps = eps2; q.sigma = sig2; q.mass = m2;   /* not symmetric */
        EXPECT(md_create(&box, 2, x, v, ty, &q, NULL, &c), MD_ERR_ARG);
        MSG(md_last_error(NULL));
    }
    {
        const md_box small = {{5.0, 10.0, 10.0}}, nan_box = {{NAN, 10.0, 10.0}},
                     huge = {{3000.0, 10.0, 10.0}};
        EXPECT(md_create(&small, 2, x, v, ty, &p, NULL, &c), MD_ERR_BOX_TOO_SMALL);
        EXPECT(md_create(&nan_box, 2, x, v, ty, &p, NULL, &c), MD_ERR_BOX_TOO_SMALL);
        EXPECT(md_create(&huge, 2, x, v, ty, &p, NULL, &c), MD_ERR_ARG);
        MSG(md_last_error(NULL));
        const int64_t counts[2] = {2, 0};
        const md_box boxes[2] = {box, box};
        EXPECT(md_batch_create(0, counts, boxes, x, v, ty, &p, NULL, &c), MD_ERR_ARG);
        EXPECT(md_batch_create(2, NULL, boxes, x, v, ty, &p, NULL, &c), MD_ERR_ARG);
        EXPECT(md_batch_create(2, counts, boxes, x, v, ty, &p, NULL, &c), MD_ERR_ARG);
    }

    /* every context call with a NULL context */
    md_thermo th;
    double e[4];
    int32_t i32 = 0;
    int64_t i64 = 0;
    EXPECT(md_bin_sort(NULL), MD_ERR_ARG);
    EXPECT(md_build_neighbors(NULL), MD_ERR_ARG);
    EXPECT(md_compute_forces(NULL, e), MD_ERR_ARG);
    EXPECT(md_step(NULL, 1, &th), MD_ERR_ARG);
    EXPECT(md_force_backward(NULL, x, 0.0, x, e, e), MD_ERR_ARG);
    EXPECT(md_set_positions(NULL, x), MD_ERR_ARG);
    EXPECT(md_set_state(NULL, x, v), MD_ERR_ARG);
    EXPECT(md_set_params(NULL, p.eps, p.sigma), MD_ERR_ARG);
    EXPECT(md_get_state(NULL, x, v, NULL, NULL, NULL), MD_ERR_ARG);
    EXPECT(md_get_permutation(NULL, ty), MD_ERR_ARG);
    EXPECT(md_get_neighbors(NULL, ty, ty, &i32), MD_ERR_ARG);
    EXPECT(md_get_thermo(NULL, &th), MD_ERR_ARG);
    EXPECT(md_get_thermo_log(NULL, e, &i32), MD_ERR_ARG);
    EXPECT(md_profile(NULL, 1), MD_ERR_ARG);
    EXPECT(md_profile_read(NULL, &i64, e, e), MD_ERR_ARG);
    EXPECT(md_profile_rebuild(NULL, &i64, e, e), MD_ERR_ARG);
    EXPECT(md_launch_count(NULL, &i64), MD_ERR_ARG);
    EXPECT(md_debug_expire_waits(NULL, 1), MD_ERR_ARG);
    EXPECT(md_batch_thermo(NULL, &th), MD_ERR_ARG);
    EXPECT(md_info(NULL, &i32, &i64), MD_ERR_ARG);
    md_destroy(NULL);

    /* the no-allocation sort: arguments and host pointers rejected */
    int32_t perm[2];
    EXPECT(md_bin_sort_noalloc(NULL, 2, x, 2.8, perm, NULL), MD_ERR_ARG);
    EXPECT(md_bin_sort_noalloc(&box, 0, x, 2.8, perm, NULL), MD_ERR_ARG);
    EXPECT(md_bin_sort_noalloc(&box, 262145, x, 2.8, perm, NULL), MD_ERR_ARG);
    EXPECT(md_bin_sort_noalloc(&box, 2, x, 0.0, perm, NULL), MD_ERR_ARG);
    EXPECT(md_bin_sort_noalloc(&box, 2, x, 6.0, perm, NULL), MD_ERR_BOX_TOO_SMALL);
    EXPECT(md_bin_sort_noalloc(&box, 2, x, 2.8, perm, NULL), MD_ERR_ARG);   /* host memory */
    MSG(md_last_error(NULL));

    /* SPME and state-stream handles */
    md_spme *sp = NULL;
    const md_spme_params sprm = {1.25, 2.5, {16, 16, 16}, 4};
    const double q[2] = {1.0, -1.0};
    EXPECT(md_spme_create(NULL, q, &sprm, &sp), MD_ERR_ARG);
    MSG(md_spme_last_error(NULL));
    EXPECT(md_spme_set_charges(NULL, q), MD_ERR_ARG);
    EXPECT(md_spme_compute(NULL, x, e), MD_ERR_ARG);
    EXPECT(md_spme_step(NULL, 1, e), MD_ERR_ARG);
    EXPECT(md_spme_profile(NULL, 1), MD_ERR_ARG);
    EXPECT(md_spme_profile_read(NULL, e), MD_ERR_ARG);
    md_spme_destroy(NULL);
    md_state_stream *ss = NULL;
    EXPECT(md_state_stream_create(NULL, &ss), MD_ERR_ARG);
    EXPECT(md_state_stream_push(NULL, x, v), MD_ERR_ARG);
    EXPECT(md_state_stream_wait(NULL), MD_ERR_ARG);
    md_state_stream_destroy(NULL);
    (void)md_state_stream_last_error(NULL);

    /* a valid create on a machine without a GPU: the CUDA runtime refuses,
     * the partly built context is freed */
    if (try_create) {
        c = (md_ctx *)0x1;
        EXPECT(md_create(&box, 2, x, v, ty, &p, NULL, &c), MD_ERR_CUDA);
        MSG(md_last_error(NULL));
        if (c != NULL) { fprintf(stderr, "out not cleared after MD_ERR_CUDA\n"); ++failures; }
    }

    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("ok\n");
    return 0;
}

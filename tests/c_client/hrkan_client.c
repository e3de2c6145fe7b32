/*
 * A plain C99 client of libhrkan.so: it includes only include/hrkan.h and the
 * C library, and calls the entry points that run on the host (shape queries,
 * argument validation, the checkpoint file).  Exit status 0 when every check
 * holds; one line per failed check on stderr otherwise.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hrkan.h"

static int failures = 0;

static void check(int ok, const char* what) {
    if (!ok) {
        fprintf(stderr, "FAILED: %s (last error: %s)\n", what, hrkan_last_error());
        ++failures;
    }
}

static hrkan_cfg make_cfg(int n_widths, const int* widths, int G, int m) {
    hrkan_cfg c;
    memset(&c, 0, sizeof c);
    c.n_widths = n_widths;
    for (int i = 0; i < n_widths; ++i) c.widths[i] = widths[i];
    c.G = G;
    c.k = 3;
    c.m = m;
    c.prec = HRKAN_FP32;
    c.grid_lo = -1.0;
    c.grid_hi = 1.0;
    c.n_instances = 1;
    return c;
}

int main(int argc, char** argv) {
    const char* path = argc > 1 ? argv[1] : "hrkan_client.ck";

    /* P = sum over layers of I * O * (G + k) */
    const int w1[] = {2, 10, 10, 1}, w2[] = {3, 16, 1}, w3[] = {2, 5, 2};
    hrkan_cfg c1 = make_cfg(4, w1, 10, 4), c2 = make_cfg(3, w2, 6, 6), c3 = make_cfg(3, w3, 5, 4);
    check(hrkan_param_count(&c1) == (2 * 10 + 10 * 10 + 10 * 1) * 13, "param count [2,10,10,1] G=10");
    check(hrkan_param_count(&c2) == (3 * 16 + 16 * 1) * 9, "param count [3,16,1] G=6");
    check(hrkan_param_count(&c3) == 0, "two outputs are not a network");

    /* configurations refused before any device work */
    hrkan_t h = (hrkan_t)&failures;   /* overwritten with NULL on failure */
    hrkan_cfg bad = make_cfg(4, w1, 10, 7);
    check(hrkan_init(&h, &bad) == HRKAN_EUNSUPPORTED && h == NULL, "m = 7 is refused");
    check(strlen(hrkan_last_error()) > 0, "a refusal leaves a message");
    bad = make_cfg(4, w1, 0, 4);
    check(hrkan_init(&h, &bad) == HRKAN_EINVAL, "G = 0 is refused");
    check(hrkan_init(NULL, &c1) == HRKAN_EINVAL, "NULL output handle is refused");

    /* a NULL handle is refused by the calls that take one */
    check(hrkan_forward_jets(NULL, NULL, NULL, 0, 0x1Fu, NULL, NULL, NULL) == HRKAN_EINVAL, "forward, NULL handle");
    check(hrkan_backward(NULL, NULL, NULL, 0, 0x1Fu, NULL, NULL, NULL, 0, NULL) == HRKAN_EINVAL, "backward, NULL handle");
    check(adam_step(NULL, NULL, NULL, 1e-3, 0.9, 0.999, 1e-8, 1, NULL) == HRKAN_EINVAL, "adam, NULL handle");
    check(hrkan_tape_floats(NULL, 100, 0x1Fu) == 0, "tape floats, NULL handle");
    hrkan_destroy(NULL);

    /* the checkpoint file round-trips the training state */
    const int64_t P = hrkan_param_count(&c1);
    const int inst = 2;
    const size_t n = (size_t)P * inst;
    float* W = malloc(n * sizeof *W);
    double* m = malloc(n * sizeof *m);
    double* v = malloc(n * sizeof *v);
    float* W2 = malloc(n * sizeof *W2);
    double* m2 = malloc(n * sizeof *m2);
    double* v2 = malloc(n * sizeof *v2);
    if (!W || !m || !v || !W2 || !m2 || !v2) return 2;
    for (size_t i = 0; i < n; ++i) {
        W[i] = (float)sin(0.1 * (double)i);
        m[i] = cos(0.2 * (double)i);
        v[i] = 1e-3 * (double)i;
    }
    check(hrkan_checkpoint_write(path, P, inst, 1234, 77, W, m, v) == HRKAN_OK, "checkpoint write");
    int64_t t = 0, td = 0;
    check(hrkan_checkpoint_read(path, P, inst, &t, &td, W2, m2, v2) == HRKAN_OK, "checkpoint read");
    check(t == 1234 && td == 77, "checkpoint step counts");
    check(memcmp(W, W2, n * sizeof *W) == 0 && memcmp(m, m2, n * sizeof *m) == 0 &&
              memcmp(v, v2, n * sizeof *v) == 0, "checkpoint contents");
    check(hrkan_checkpoint_read(path, P + 1, inst, &t, &td, W2, m2, v2) == HRKAN_EINVAL, "checkpoint shape mismatch");
    remove(path);
    check(hrkan_checkpoint_read(path, P, inst, &t, &td, W2, m2, v2) == HRKAN_EIO, "missing checkpoint");
    free(W); free(m); free(v); free(W2); free(m2); free(v2);

    if (failures == 0) printf("hrkan C client: all checks passed\n");
    return failures == 0 ? 0 : 1;
}

/* A plain C program against the C ABI (compiled and linked by
 * tests/test_native_checks.py on the host; it runs only where a GPU is present).
 * It applies a three-step wiring diagram -- the Figure 2 circuit of the
 * paper: NOT a(2); a(2) controls a(1); NOT a(2) -- to the Sec. 2b input
 * (1, -1, 1, -1)/2 and checks the state and probabilities, then checks an
 * invalid step is rejected and leaves the state alone. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "qsim.h"

static int expect(int rc, const char *what)
{
    if (rc != QSIM_OK) {
        fprintf(stderr, "%s failed: %d (%s)\n", what, rc, qsim_last_error());
        return 1;
    }
    return 0;
}

int main(void)
{
    qsim_ctx *ctx = NULL;
    if (expect(qsim_create(2, QSIM_C128, &ctx), "qsim_create")) return 1;
    const double h = 0.5;
    double k1[8] = {h, 0, -h, 0, h, 0, -h, 0}; /* interleaved (re, im) */
    /* bit 0 is a(1), bit 1 is a(2) */
    const qsim_step steps[3] = {
        {1, 0, 0, 0},         /* NOT a(2) */
        {0, 0, 2, 2},         /* a(2) on |1> controls a(1) */
        {1, 0, 0, 0},         /* NOT a(2) */
    };
    double k2[8], p[4], norm = 0;
    int bad = expect(qsim_load_state(ctx, k1, 4), "qsim_load_state") ||
              expect(qsim_apply_circuit(ctx, steps, 3), "qsim_apply_circuit") ||
              expect(qsim_read_state(ctx, k2, 4), "qsim_read_state") ||
              expect(qsim_probabilities(ctx, p, 4, &norm), "qsim_probabilities");
    /* net effect: a(1) flips where a(2) = 0, so rows 0 and 1 swap */
    const double want[8] = {-h, 0, h, 0, h, 0, -h, 0};
    if (!bad && memcmp(k2, want, sizeof want) != 0) {
        fprintf(stderr, "state differs from the Figure 2 result\n");
        bad = 1;
    }
    for (int i = 0; !bad && i < 4; ++i)
        if (p[i] != 0.25) bad = 1;
    if (!bad && fabs(norm - 1.0) > 1e-15) bad = 1;
    const qsim_step wrong = {0, 0, 1, 1}; /* target among its own controls */
    if (!bad && qsim_apply_circuit(ctx, &wrong, 1) != QSIM_EINVAL) bad = 1;
    if (!bad && (qsim_read_state(ctx, k2, 4) != QSIM_OK || memcmp(k2, want, sizeof want) != 0)) bad = 1;
    qsim_destroy(ctx);
    printf(bad ? "failed\n" : "ok\n");
    return bad;
}

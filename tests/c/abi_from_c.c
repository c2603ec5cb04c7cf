/* The boundary used from plain C (C99): the header compiles as C, the library links and its
 * host-only entry points run without a GPU.
 *  - plsqr_workspace_bytes: a valid 1024 x 1024 single-precision configuration has a positive
 *    size; sizes that 2^(levels-1) does not divide are rejected with -1.
 *  - plsqr_projected_solve with k = 1: the projected problem (3.6) is
 *        min_y || [alpha_1; beta_2] y - [beta_1; 0] ||^2 + tau y^2,
 *    so y = alpha_1 beta_1 / (alpha_1^2 + beta_2^2 + tau) and ||rbar_1|| is the square root of
 *    the minimised value; invalid arguments return PLSQR_E_INVALID.
 * Prints "ok" and exits 0 when every check holds. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "plsqr.h"

static int fails = 0;

static void check(int cond, const char* what) {
    if (!cond) {
        printf("FAILED: %s\n", what);
        ++fails;
    }
}

int main(void) {
    plsqr_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.ndim = 2;
    cfg.precision = PLSQR_FP32;
    cfg.n[0] = 1024;
    cfg.n[1] = 1024;
    cfg.n[2] = 1;
    cfg.mg_levels = 6;
    cfg.mg_sweeps = 2;
    cfg.mg_cycles = 1;
    cfg.max_batch = 1;
    cfg.kappa_floor = 1e-4;
    plsqr_operator op;
    memset(&op, 0, sizeof op);
    op.kind = PLSQR_OP_BLUR;
    op.sigma[0] = op.sigma[1] = 4.0;
    op.radius[0] = op.radius[1] = 12;
    const int64_t bytes = plsqr_workspace_bytes(&cfg, &op);
    check(bytes > (int64_t)6 * 1024 * 1024 * 4, "workspace of the 1024 x 1024 configuration");
    cfg.n[0] = cfg.n[1] = 100;
    cfg.mg_levels = 4;
    check(plsqr_workspace_bytes(&cfg, &op) == -1, "100 x 100 with 4 levels is rejected");

    const double alpha[2] = {0.8, 0.3}, beta[2] = {2.0, 0.6};
    const double taus[3] = {0.0, 0.05, 1.0};
    for (int t = 0; t < 3; ++t) {
        const double tau = taus[t];
        double y = 0.0, rbar = 0.0;
        check(plsqr_projected_solve(1, alpha, beta, tau, &y, &rbar) == PLSQR_OK, "projected solve k = 1");
        const double y_ref = alpha[0] * beta[0] / (alpha[0] * alpha[0] + beta[1] * beta[1] + tau);
        const double r0 = beta[0] - alpha[0] * y_ref, r1 = beta[1] * y_ref;
        const double rbar_ref = sqrt(r0 * r0 + r1 * r1 + tau * y_ref * y_ref);
        check(fabs(y - y_ref) <= 1e-14 * fabs(y_ref), "y of k = 1");
        check(fabs(rbar - rbar_ref) <= 1e-14 * rbar_ref, "rbar of k = 1");
    }
    double y = 0.0;
    check(plsqr_projected_solve(0, alpha, beta, 0.0, &y, NULL) == PLSQR_E_INVALID, "k = 0 rejected");
    check(plsqr_projected_solve(1, NULL, beta, 0.0, &y, NULL) == PLSQR_E_INVALID, "NULL alpha rejected");
    check(plsqr_projected_solve(1, alpha, beta, -1.0, &y, NULL) == PLSQR_E_INVALID, "tau < 0 rejected");
    if (fails) return 1;
    printf("ok\n");
    return 0;
}

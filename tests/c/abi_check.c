/* A plain C99 client of include/lb.h: checks, without any GPU work, that the
 * header compiles as C and that the library's host-side paths behave as the
 * header states (status strings, argument validation, NULL handling). */
#include <stdio.h>
#include <string.h>

#include "lb.h"

static int failures = 0;

static void expect(int cond, const char* what)
{
    if (!cond) {
        printf("FAIL: %s\n", what);
        ++failures;
    }
}

int main(void)
{
    double rho[25];
    lb_params p;
    lb_state* s = (lb_state*)&p;   /* must be overwritten with NULL on failure */
    lb_batch* b = (lb_batch*)&p;
    double out[4];
    int i, c = -1;

    for (i = 0; i < 25; ++i) rho[i] = 0.7;
    memset(&p, 0, sizeof p);
    p.nx = 5;
    p.ny = 5;
    p.omega = 1.0;
    p.G1 = -5.0;
    p.G2 = 0.6;
    p.rho0 = 1.0;
    p.psi_form = LB_PSI_SC_EXP;
    p.prec = LB_FP32;
    p.trace_every = 10;

    expect(strcmp(lb_status_str(LB_OK), lb_status_str(LB_ERR_ARG)) != 0, "distinct status strings");
    expect(lb_status_str((lb_status)17) != NULL, "unknown status has a string");

    p.nx = 4;   /* below the 5 x 5 minimum */
    expect(lb_init(&s, &p, rho, NULL) == LB_ERR_ARG && s == NULL, "nx = 4 rejected, out cleared");
    p.nx = 5;
    p.omega = 2.0;
    expect(lb_init(&s, &p, rho, NULL) == LB_ERR_ARG, "omega = 2 rejected");
    p.omega = 1.0;
    p.rho0 = 0.0;
    expect(lb_init(&s, &p, rho, NULL) == LB_ERR_ARG, "rho0 = 0 rejected");
    p.rho0 = 1.0;
    p.prec = (lb_precision)7;
    expect(lb_init(&s, &p, rho, NULL) == LB_ERR_ARG, "unknown precision rejected");
    p.prec = LB_FP32;
    expect(lb_init(&s, &p, NULL, NULL) == LB_ERR_ARG, "NULL rho_init rejected");
    expect(lb_init(NULL, &p, rho, NULL) == LB_ERR_ARG, "NULL out rejected");
    expect(lb_init(&s, NULL, rho, NULL) == LB_ERR_ARG, "NULL params rejected");

    expect(lb_step(NULL, 1) == LB_ERR_ARG, "lb_step(NULL)");
    expect(lb_energy(NULL, out) == LB_ERR_ARG, "lb_energy(NULL)");
    expect(lb_fields(NULL, rho, NULL, NULL) == LB_ERR_ARG, "lb_fields(NULL)");
    expect(lb_trace(NULL, out, 0, &c) == LB_ERR_ARG, "lb_trace(NULL)");
    expect(lb_time(NULL) < 0, "lb_time(NULL) negative");
    lb_destroy(NULL);   /* a no-op */

    expect(lb_batch_init(&b, 0, &p, NULL, NULL) == LB_ERR_ARG && b == NULL, "empty batch rejected");
    expect(lb_batch_count(NULL) <= 0, "lb_batch_count(NULL)");
    lb_batch_destroy(NULL);

    expect(lb_energy_noalloc(NULL, NULL, 5, 5, -5.0, 0.6, out, NULL) == LB_ERR_ARG,
           "lb_energy_noalloc(NULL) rejected");

    printf(failures ? "abi_check: %d failure(s)\n" : "abi_check: ok\n", failures);
    return failures ? 1 : 0;
}

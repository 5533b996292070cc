/* A plain C99 client that runs a lattice through include/lb.h on the GPU:
 * lb_init from host memory, 200 steps, trace, energy, fields, save/resume,
 * destroy. Checks what holds for any correct implementation: mass is
 * conserved, the trace has one row per 10 steps, fields average to the mass,
 * and a resumed run repeats the original bit for bit. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lb.h"

#define NX 96
#define NY 80

static int failures = 0;

static void expect(int cond, const char* what)
{
    if (!cond) {
        printf("FAIL: %s\n", what);
        ++failures;
    }
}

static int check(lb_status st, const char* what)
{
    if (st != LB_OK) {
        printf("FAIL: %s: %s\n", what, lb_status_str(st));
        ++failures;
        return 0;
    }
    return 1;
}

int main(void)
{
    static double rho0[NX * NY], rho[NX * NY], rho2[NX * NY], trace[64 * 5];
    double e[4], mass0 = 0.0, sum = 0.0;
    lb_params p;
    lb_state* s = NULL;
    lb_state* r = NULL;
    int i, count = 0;
    unsigned long long x = 12345u;
    size_t bytes;
    unsigned char* saved;

    for (i = 0; i < NX * NY; ++i) {   /* 0.7 (1 +- 1%), a fixed 64-bit LCG */
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        rho0[i] = 0.7 * (1.0 + 0.01 * (2.0 * (double)(x >> 11) / 9007199254740992.0 - 1.0));
        mass0 += rho0[i];
    }
    memset(&p, 0, sizeof p);
    p.nx = NX;
    p.ny = NY;
    p.omega = 1.0;
    p.G1 = -5.0;
    p.G2 = 0.6;
    p.rho0 = 1.0;
    p.psi_form = LB_PSI_SC_EXP;
    p.prec = LB_FP32;
    p.trace_every = 10;
    if (!check(lb_init(&s, &p, rho0, NULL), "lb_init")) return 1;
    check(lb_step(s, 100), "lb_step 100");
    bytes = lb_state_bytes(s);
    saved = (unsigned char*)malloc(bytes);
    check(lb_save_state(s, saved, bytes), "lb_save_state");
    check(lb_step(s, 100), "lb_step 100 more");
    expect(lb_time(s) == 200, "time 200");
    check(lb_energy(s, e), "lb_energy");
    expect(isfinite(e[0]) && isfinite(e[1]) && isfinite(e[2]), "finite energies");
    expect(fabs(e[3] - mass0) <= 1e-6 * mass0, "mass conserved");
    check(lb_trace(s, trace, 64, &count), "lb_trace");
    expect(count == 20, "20 trace rows (t = 0, 10, ..., 190)");
    expect(count > 0 && trace[0] == 0.0 && trace[5 * (count - 1)] == 190.0, "trace times");
    check(lb_fields(s, rho, NULL, NULL), "lb_fields");
    for (i = 0; i < NX * NY; ++i) sum += rho[i];
    expect(fabs(sum - mass0) <= 1e-6 * mass0, "fields sum to the mass");

    /* resume from the state saved at t = 100 */
    if (check(lb_init(&r, &p, rho0, NULL), "lb_init (resume)")) {
        check(lb_load_state(r, saved, bytes), "lb_load_state");
        expect(lb_time(r) == 100, "resumed at t = 100");
        check(lb_step(r, 100), "resumed steps");
        check(lb_fields(r, rho2, NULL, NULL), "lb_fields (resumed)");
        expect(memcmp(rho, rho2, sizeof rho) == 0, "resumed run bit-identical");
        lb_destroy(r);
    }
    free(saved);
    lb_destroy(s);
    printf(failures ? "abi_run: %d failure(s)\n" : "abi_run: ok\n", failures);
    return failures ? 1 : 0;
}

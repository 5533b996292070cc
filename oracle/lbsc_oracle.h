/*
 * lbsc_oracle.h — interface of the FP64 CPU oracle for the two-belt
 * Shan–Chen D2Q9 lattice Boltzmann method (Chibbaro, Falcucci, Chen, Shan,
 * Chiatti, Succi, "Lattice Boltzmann models for non-ideal fluids with
 * arrested phase-separation", arXiv:1008.2865).
 *
 * TEST INFRASTRUCTURE ONLY. This header belongs to the oracle and to nothing
 * else: the CUDA library neither includes nor links it, and the oracle never
 * includes the library's headers. Only the tests, the package smoke check and
 * the benchmark's CPU-baseline leg may load the oracle.
 *
 * Conventions (all arrays are caller-owned, FP64, row-major [y][x]):
 *   populations  f[i][y][x], i = 0..8 in the D2Q9 order
 *                (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *   every lattice is periodic in x and y; nx, ny >= 5 so that the two-site
 *   force stencil never sees its own periodic image twice.
 */
#ifndef LBSC_ORACLE_H
#define LBSC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;      /* lattice size */
    double omega;    /* BGK relaxation frequency 1/tau (Eq. 1) */
    double G1;       /* first-belt coupling, D2Q9 weights w_i (Eq. FORCE) */
    double G2;       /* coupling on the E(8) weights p of both belts (Eq. FORCE) */
    double rho0;     /* pseudopotential density scale (psi form, Sec. 2) */
} orc_params;

/* Number of OpenMP threads the oracle uses. */
int orc_threads(void);

/* The 25-entry link table (rest link first, then belt 1 in Table 1 order,
 * then belt 2): speeds (cx, cy), D2Q9 weight w (0 on belt 2) and E(8)
 * weight p (the rest entry's p follows from the normalisation Eq. weights_1). */
void orc_link_table(int* cx, int* cy, double* w, double* p);

/* psi(rho) = sqrt(rho0) (1 - exp(-rho/rho0)), elementwise over n values. */
void orc_psi(long n, const double* rho, double rho0, double* psi);

/* Two-belt pseudopotential force of Eq. FORCE (with the attractive sign of
 * Eq. forza) from a psi field: F = -(F_s + F_m). */
void orc_force(const orc_params* P, const double* psi, double* Fx, double* Fy);

/* Pseudo-energies of Sec. 5 from a psi field: out = {E_s, E_m, E_bulk}. */
void orc_energy(const orc_params* P, const double* psi, double out[3]);

/* f_i = w_i rho (the u = 0 equilibrium) — the initial state. */
void orc_init(const orc_params* P, const double* rho, double* f);

/* rho = sum f_i, (ux, uy) = sum c_i f_i / rho; any output may be NULL. */
void orc_moments(const orc_params* P, const double* f, double* rho, double* ux, double* uy);

/* One full step of Eq. 1: moments, psi, force, BGK collision towards the
 * velocity-shifted equilibrium, streaming. f_in and f_out must not alias. */
void orc_step(const orc_params* P, const double* f_in, double* f_out);

/* Run `steps` steps from f_i = w_i rho_init. Every state t < steps with
 * t % trace_every == 0 appends a row (t, mass, E_s, E_m, E_bulk) to trace
 * while fewer than trace_cap rows are stored (trace_every <= 0: no trace).
 * On return rho/ux/uy (any may be NULL) hold the moments of state `steps`.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int orc_run(const orc_params* P, const double* rho_init, long steps, int trace_every,
            double* rho, double* ux, double* uy,
            double* trace, int trace_cap, int* trace_count);

/* J = E_s(T) + E_m(T) + sum_x (rho(x, T) - rho_target(x))^2 after `steps`
 * steps from f = w rho_init (the energy is also returned in *E if non-NULL).
 * Returns NaN on bad arguments. */
double orc_objective(const orc_params* P, const double* rho_init, long steps,
                     const double* rho_target, double* E);

/* J and its gradient with respect to rho_init (N values) and (G1, G2), by a
 * hand-written reverse sweep over all stored states. Returns 0 or -1. */
int orc_gradient(const orc_params* P, const double* rho_init, long steps,
                 const double* rho_target, double* J, double* grad_rho, double* grad_G);

/* The transpose of one step's Jacobian at populations f applied to lam_next
 * (both [9][ny][nx]); gG receives the step's explicit d/dG1, d/dG2 terms. */
void orc_adjoint_step(const orc_params* P, const double* f, const double* lam_next, double* lam,
                      double* gG);

#ifdef __cplusplus
}
#endif
#endif

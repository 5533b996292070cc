/*
 * lbsc_oracle.c — plain FP64 CPU oracle for the two-belt Shan–Chen D2Q9
 * lattice Boltzmann method of Chibbaro et al., arXiv:1008.2865.
 *
 * TEST INFRASTRUCTURE ONLY: the CUDA library never links, includes or calls
 * this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg load it. It is deliberately slow and literal: one site
 * at a time, every formula written in the paper's order and notation, FP64,
 * compiled without floating-point contraction (-ffp-contract=off) so that the
 * arithmetic is exactly what the source text says. OpenMP splits rows among
 * threads; every output element is written by exactly one thread and every
 * reduction is summed in a fixed order, so results do not depend on the
 * thread count.
 *
 * Readings of passages the paper leaves open (each is also listed in the
 * design notes):
 *   - Force sign: Eq. FORCE is printed without the minus sign that Eq. forza
 *     and Eq. ftot carry; with G < 0 meaning attraction (Sec. 3) and the
 *     critical coupling G_cr = -4 (Sec. 2) the force is F = -(F_s + F_m).
 *   - G2 multiplies the E(8) weights on both belts: p_s on belt 1 inside F_s
 *     and p_m on belt 2 in F_m (Eq. FORCE); G1 multiplies the D2Q9 weights w
 *     on belt 1 only.
 *   - The forcing term F_i of Eq. 1 is the Shan–Chen velocity shift: the
 *     equilibrium of Eq. 4 is taken at u_eq = u + F/(omega rho).
 *   - The rest weight p_s0 of the energy sum E_s follows from the
 *     normalisation Eq. weights_1 (p_s0 = 1 - sum of the 24 link weights),
 *     and the belt-2 energy sum E_m runs over the 16 belt-2 links only.
 *   - Energies and mass of state t use rho(t) and psi(t) of the populations
 *     after streaming into t (before the collision of step t).
 */
#include "lbsc_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#if LDBL_MANT_DIG < 113
#include <quadmath.h>
#endif

/* ---- lattice (Sec. 2 and Sec. 3, Table 1) ------------------------------- */

/* D2Q9 speeds c_i and weights w_i of the standard model (Sec. 2); the same
 * eight non-rest speeds form belt 1 of the force (Sec. 3, Fig. 1 caption). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0,
                            1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Table 1, belt 1 (the short-range belt s): p(1) = 4/63 on the four axis
 * links i = 1..4, p(2) = 4/135 on the four diagonals i = 5..8, in the same
 * order as the D2Q9 speeds above (index 0 unused here). */
static const double PS[9] = {0.0,
                             4.0 / 63.0,  4.0 / 63.0,  4.0 / 63.0,  4.0 / 63.0,
                             4.0 / 135.0, 4.0 / 135.0, 4.0 / 135.0, 4.0 / 135.0};

/* Table 1, belt 2 (the mid-range belt m): |c|^2 = 4 on i = 1..4, |c|^2 = 5 on
 * i = 5..12, |c|^2 = 8 on i = 13..16 (Fig. 1 caption: energies 4, 5, 8). */
static const int MCX[16] = {2, 0, -2, 0,
                            2, 1, -1, -2, -2, -1, 1, 2,
                            2, -2, -2, 2};
static const int MCY[16] = {0, 2, 0, -2,
                            1, 2, 2, 1, -1, -2, -2, -1,
                            2, 2, -2, -2};
static const double PM[16] = {1.0 / 180.0, 1.0 / 180.0, 1.0 / 180.0, 1.0 / 180.0,
                              2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0,
                              2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0,
                              1.0 / 15120.0, 1.0 / 15120.0, 1.0 / 15120.0, 1.0 / 15120.0};

/* Rest weight of the E(8) set from Eq. weights_1: the weights of the rest
 * link and of all 24 links sum to one. */
static double ps_rest(void)
{
    double s = 0.0;
    for (int i = 1; i <= 8; ++i) s += PS[i];
    for (int k = 0; k < 16; ++k) s += PM[k];
    return 1.0 - s;
}

static inline long wrap(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

static inline long site(const orc_params* P, long x, long y)
{
    return wrap(y, P->ny) * (long)P->nx + wrap(x, P->nx);
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_link_table(int* cx, int* cy, double* w, double* p)
{
    cx[0] = 0; cy[0] = 0; w[0] = W[0]; p[0] = ps_rest();
    for (int i = 1; i <= 8; ++i) {
        cx[i] = CX[i]; cy[i] = CY[i]; w[i] = W[i]; p[i] = PS[i];
    }
    for (int k = 0; k < 16; ++k) {
        cx[9 + k] = MCX[k]; cy[9 + k] = MCY[k]; w[9 + k] = 0.0; p[9 + k] = PM[k];
    }
}

/* ---- pseudopotential (Sec. 2, the Shan–Chen psi; Sec. 3: rho0 = 1) ------- */

/* exp(x) correctly rounded to double: the quad-precision exponential (113-bit
 * significand, error a few quad ulps) rounded once to double. libm's double
 * exp is accurate to about half an ulp but is not correctly rounded; the
 * correctly rounded value is the one FP64 result that is fixed by the
 * mathematics alone, so it is the one an independent implementation can be
 * required to reproduce bit for bit. */
static inline double exp_cr(double x)
{
#if LDBL_MANT_DIG >= 113
    return (double)expl((long double)x);
#else
    return (double)expq((__float128)x);
#endif
}

static inline double psi_of(double rho, double rho0)
{
    return sqrt(rho0) * (1.0 - exp_cr(-rho / rho0));
}

void orc_psi(long n, const double* rho, double rho0, double* psi)
{
    for (long k = 0; k < n; ++k) psi[k] = psi_of(rho[k], rho0);
}

/* ---- force (Sec. 3, Eq. FORCE; sign of Eq. forza) ------------------------ */

/* F(x) at one site: F_s = G1 psi sum_i w_i psi(x + c_i) c_i
 *                       + G2 psi sum_i p_si psi(x + c_si) c_si  (belt 1)
 *                   F_m = G2 psi sum_i p_mi psi(x + c_mi) c_mi  (belt 2)
 *                   F   = -(F_s + F_m)                                     */
static void force_at(const orc_params* P, const double* psi, long x, long y,
                     double* Fx, double* Fy)
{
    double wx = 0.0, wy = 0.0;   /* sum_i w_i psi_i c_i, belt 1 */
    double sx = 0.0, sy = 0.0;   /* sum_i p_si psi_i c_si, belt 1 */
    double mx = 0.0, my = 0.0;   /* sum_i p_mi psi_i c_mi, belt 2 */
    for (int i = 1; i <= 8; ++i) {
        const double pn = psi[site(P, x + CX[i], y + CY[i])];
        wx += W[i] * pn * CX[i];
        wy += W[i] * pn * CY[i];
        sx += PS[i] * pn * CX[i];
        sy += PS[i] * pn * CY[i];
    }
    for (int k = 0; k < 16; ++k) {
        const double pn = psi[site(P, x + MCX[k], y + MCY[k])];
        mx += PM[k] * pn * MCX[k];
        my += PM[k] * pn * MCY[k];
    }
    const double ps = psi[site(P, x, y)];
    const double Fsx = P->G1 * ps * wx + P->G2 * ps * sx;
    const double Fsy = P->G1 * ps * wy + P->G2 * ps * sy;
    const double Fmx = P->G2 * ps * mx;
    const double Fmy = P->G2 * ps * my;
    *Fx = -(Fsx + Fmx);
    *Fy = -(Fsy + Fmy);
}

void orc_force(const orc_params* P, const double* psi, double* Fx, double* Fy)
{
#pragma omp parallel for schedule(static)
    for (long y = 0; y < P->ny; ++y)
        for (long x = 0; x < P->nx; ++x) {
            const long s = y * P->nx + x;
            force_at(P, psi, x, y, &Fx[s], &Fy[s]);
        }
}

/* ---- pseudo-energies (Sec. 5) -------------------------------------------- */

/* E_s = 1/2 sum_x psi(x) sum_{i=0..8} (G1 w_i + G2 p_si) psi(x + c_si)
 * E_m = 1/2 sum_x psi(x) sum_{i=1..16} G2 p_mi psi(x + c_mi)       (Eq. e2)
 * E_bulk = A1/2 sum_x psi(x)^2, A1 = G1 + G2                      (Eq. Ebulk)
 * Rows are summed into per-row partials, then the rows in order.          */
void orc_energy(const orc_params* P, const double* psi, double out[3])
{
    const long nx = P->nx, ny = P->ny;
    const double p0 = ps_rest();
    const double A1 = P->G1 + P->G2;
    double* rows = (double*)malloc(sizeof(double) * 3 * (size_t)ny);
    if (!rows) { out[0] = out[1] = out[2] = NAN; return; }
#pragma omp parallel for schedule(static)
    for (long y = 0; y < ny; ++y) {
        double es = 0.0, em = 0.0, eb = 0.0;
        for (long x = 0; x < nx; ++x) {
            const double ps = psi[y * nx + x];
            double ss = (P->G1 * W[0] + P->G2 * p0) * ps;
            for (int i = 1; i <= 8; ++i)
                ss += (P->G1 * W[i] + P->G2 * PS[i]) * psi[site(P, x + CX[i], y + CY[i])];
            double sm = 0.0;
            for (int k = 0; k < 16; ++k)
                sm += P->G2 * PM[k] * psi[site(P, x + MCX[k], y + MCY[k])];
            es += 0.5 * ps * ss;
            em += 0.5 * ps * sm;
            eb += 0.5 * A1 * ps * ps;
        }
        rows[3 * y + 0] = es;
        rows[3 * y + 1] = em;
        rows[3 * y + 2] = eb;
    }
    double es = 0.0, em = 0.0, eb = 0.0;
    for (long y = 0; y < ny; ++y) {
        es += rows[3 * y + 0];
        em += rows[3 * y + 1];
        eb += rows[3 * y + 2];
    }
    free(rows);
    out[0] = es; out[1] = em; out[2] = eb;
}

/* ---- kinetic update (Sec. 2, Eqs. 1-4) ----------------------------------- */

/* Initial state: the u = 0 equilibrium of Eq. 4, f_i = w_i rho. */
void orc_init(const orc_params* P, const double* rho, double* f)
{
    const long N = (long)P->nx * P->ny;
    for (int i = 0; i < 9; ++i)
        for (long s = 0; s < N; ++s) f[i * N + s] = W[i] * rho[s];
}

/* rho = sum_i f_i and rho u = sum_i c_i f_i (Eqs. 2-3), summed i = 0..8. */
static inline void moments_at(const double* f, long N, long s,
                              double* rho, double* jx, double* jy)
{
    double r = 0.0, ax = 0.0, ay = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double fi = f[i * N + s];
        r += fi;
        ax += CX[i] * fi;
        ay += CY[i] * fi;
    }
    *rho = r; *jx = ax; *jy = ay;
}

void orc_moments(const orc_params* P, const double* f, double* rho, double* ux, double* uy)
{
    const long N = (long)P->nx * P->ny;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < N; ++s) {
        double r, ax, ay;
        moments_at(f, N, s, &r, &ax, &ay);
        if (rho) rho[s] = r;
        if (ux) ux[s] = ax / r;
        if (uy) uy[s] = ay / r;
    }
}

/* One step of Eq. 1 given psi(t) of every site:
 *   f_i^eq = w_i rho (1 + c_i.u/cs2 + (c_i.u)^2/(2 cs2^2) - u^2/(2 cs2))  (Eq. 4)
 *   with cs2 = 1/3, so the three coefficients are exactly 3, 9/2 and 3/2,
 *   evaluated at u_eq = u + F/(omega rho) (velocity shift),
 *   f*_i = f_i - omega (f_i - f_i^eq), then f_i(x + c_i, t+1) = f*_i(x).   */
static void collide_stream(const orc_params* P, const double* f_in, const double* psi,
                           double* f_out)
{
    const long nx = P->nx, ny = P->ny, N = nx * ny;
    const double om = P->omega;
#pragma omp parallel for schedule(static)
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            const long s = y * nx + x;
            double rho, jx, jy, Fx, Fy;
            moments_at(f_in, N, s, &rho, &jx, &jy);
            force_at(P, psi, x, y, &Fx, &Fy);
            const double ux = jx / rho;
            const double uy = jy / rho;
            const double orho = om * rho;
            const double vx = ux + Fx / orho;   /* u_eq */
            const double vy = uy + Fy / orho;
            const double usq = vx * vx + vy * vy;
            for (int i = 0; i < 9; ++i) {
                const double cu = CX[i] * vx + CY[i] * vy;
                const double feq = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                const double fi = f_in[i * N + s];
                const double fs = fi - om * (fi - feq);
                f_out[i * N + site(P, x + CX[i], y + CY[i])] = fs;
            }
        }
}

static void psi_field(const orc_params* P, const double* f, double* rho, double* psi)
{
    const long N = (long)P->nx * P->ny;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < N; ++s) {
        double r, ax, ay;
        moments_at(f, N, s, &r, &ax, &ay);
        rho[s] = r;
        psi[s] = psi_of(r, P->rho0);
    }
}

static int params_ok(const orc_params* P)
{
    return P && P->nx >= 5 && P->ny >= 5 && P->omega > 0.0 && P->omega < 2.0 &&
           P->rho0 > 0.0 && isfinite(P->G1) && isfinite(P->G2);
}

void orc_step(const orc_params* P, const double* f_in, double* f_out)
{
    const long N = (long)P->nx * P->ny;
    double* rho = (double*)malloc(sizeof(double) * (size_t)N);
    double* psi = (double*)malloc(sizeof(double) * (size_t)N);
    if (rho && psi) {
        psi_field(P, f_in, rho, psi);
        collide_stream(P, f_in, psi, f_out);
    }
    free(rho);
    free(psi);
}

int orc_run(const orc_params* P, const double* rho_init, long steps, int trace_every,
            double* rho_out, double* ux_out, double* uy_out,
            double* trace, int trace_cap, int* trace_count)
{
    if (!params_ok(P) || !rho_init || steps < 0) return -1;
    const long N = (long)P->nx * P->ny;
    double* fa = (double*)malloc(sizeof(double) * 9 * (size_t)N);
    double* fb = (double*)malloc(sizeof(double) * 9 * (size_t)N);
    double* rho = (double*)malloc(sizeof(double) * (size_t)N);
    double* psi = (double*)malloc(sizeof(double) * (size_t)N);
    if (!fa || !fb || !rho || !psi) {
        free(fa); free(fb); free(rho); free(psi);
        return -1;
    }
    int count = 0;
    orc_init(P, rho_init, fa);
    for (long t = 0; t < steps; ++t) {
        psi_field(P, fa, rho, psi);
        if (trace && trace_every > 0 && t % trace_every == 0 && count < trace_cap) {
            double e[3], mass = 0.0;
            orc_energy(P, psi, e);
            for (long s = 0; s < N; ++s) mass += rho[s];
            double* row = trace + 5 * (long)count;
            row[0] = (double)t; row[1] = mass; row[2] = e[0]; row[3] = e[1]; row[4] = e[2];
            ++count;
        }
        collide_stream(P, fa, psi, fb);
        double* tmp = fa; fa = fb; fb = tmp;
    }
    orc_moments(P, fa, rho_out, ux_out, uy_out);
    if (trace_count) *trace_count = count;
    free(fa); free(fb); free(rho); free(psi);
    return 0;
}

/* ---- objective and its gradient (reverse mode) --------------------------- */
/*
 * J = E_s(T) + E_m(T) + sum_x (rho(x, T) - rho_target(x))^2: the pseudo-energy
 * of Sec. 5 at the final state plus a squared misfit of the final density to
 * a target field. The gradient with respect to the initial density, G1 and G2
 * is the plain reverse sweep of the step above, written out by hand:
 *   streaming   f_i(x + c_i, t+1) = f*_i(x)      ->  l*_i(x) = l_i(x + c_i, t+1)
 *   collision   f*_i = (1 - om) f_i + om feq_i(rho, v),  v = (j + F/om) / rho
 *               feq_i = w_i rho (1 + 3 c_i.v + 9/2 (c_i.v)^2 - 3/2 v.v)
 *   force       F(x) = -psi(x) S(x),  S(x) = sum_c K_c c psi(x + c)
 *   psi         psi(rho),  psi' = exp(-rho/rho0) / sqrt(rho0)
 *   moments     rho = sum_i f_i, j = sum_i c_i f_i
 *   start       f_i(x, 0) = w_i rho_init(x)
 * The force's transpose gathers Q = psi F-bar over the same 24-link stencil
 * (K_c = K_{-c}). All T+1 states are kept in memory (no checkpointing).
 */

/* sum_c K_c c psi(x + c) split into the D2Q9 (w) and E(8) (p) parts:
 * S = G1 Sw + G2 Sp. */
static void stencil_sums(const orc_params* P, const double* psi, long x, long y,
                         double* Swx, double* Swy, double* Spx, double* Spy)
{
    double wx = 0.0, wy = 0.0, px = 0.0, py = 0.0;
    for (int i = 1; i <= 8; ++i) {
        const double pn = psi[site(P, x + CX[i], y + CY[i])];
        wx += W[i] * pn * CX[i];
        wy += W[i] * pn * CY[i];
        px += PS[i] * pn * CX[i];
        py += PS[i] * pn * CY[i];
    }
    for (int k = 0; k < 16; ++k) {
        const double pn = psi[site(P, x + MCX[k], y + MCY[k])];
        px += PM[k] * pn * MCX[k];
        py += PM[k] * pn * MCY[k];
    }
    *Swx = wx; *Swy = wy; *Spx = px; *Spy = py;
}

/* Pseudo-energy of Sec. 5 at psi and its partial derivatives:
 * dE/dpsi(y) = sum_{c incl. rest} K_c psi(y + c); dE/dG1, dE/dG2. */
static double energy_and_derivatives(const orc_params* P, const double* psi, double* dEdpsi,
                                     double* dEdG1, double* dEdG2)
{
    const long nx = P->nx, ny = P->ny;
    const double p0 = ps_rest();
    double E = 0.0, g1 = 0.0, g2 = 0.0;
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            const double ps = psi[y * nx + x];
            double sw = W[0] * ps, sp = p0 * ps;           /* rest link */
            for (int i = 1; i <= 8; ++i) {
                const double pn = psi[site(P, x + CX[i], y + CY[i])];
                sw += W[i] * pn;
                sp += PS[i] * pn;
            }
            for (int k = 0; k < 16; ++k) sp += PM[k] * psi[site(P, x + MCX[k], y + MCY[k])];
            const double sk = P->G1 * sw + P->G2 * sp;      /* sum_c K_c psi(x + c) */
            E += 0.5 * ps * sk;
            g1 += 0.5 * ps * sw;
            g2 += 0.5 * ps * sp;
            dEdpsi[y * nx + x] = sk;
        }
    *dEdG1 = g1;
    *dEdG2 = g2;
    return E;
}

/* One reverse step: lam_t = (d f(t+1) / d f(t))^T lam_next at the state f_t;
 * adds the explicit dependence of step t on G1, G2 to gG[0], gG[1]. */
static void adjoint_step(const orc_params* P, const double* f, const double* lam_next,
                         double* lam, double* gG)
{
    const long nx = P->nx, ny = P->ny, N = nx * ny;
    const double om = P->omega;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* Qx = (double*)malloc(sizeof(double) * N);
    double* Qy = (double*)malloc(sizeof(double) * N);
    double* rbar = (double*)malloc(sizeof(double) * N);
    double* jbx = (double*)malloc(sizeof(double) * N);
    double* jby = (double*)malloc(sizeof(double) * N);
    psi_field(P, f, rho, psi);
    double g1 = 0.0, g2 = 0.0;
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            const long s = y * nx + x;
            double r, jx, jy, ls[9];
            moments_at(f, N, s, &r, &jx, &jy);
            for (int i = 0; i < 9; ++i) ls[i] = lam_next[i * N + site(P, x + CX[i], y + CY[i])];
            double Swx, Swy, Spx, Spy;
            stencil_sums(P, psi, x, y, &Swx, &Swy, &Spx, &Spy);
            const double Sx = P->G1 * Swx + P->G2 * Spx, Sy = P->G1 * Swy + P->G2 * Spy;
            const double ps = psi[s];
            const double Fx = -ps * Sx, Fy = -ps * Sy;
            const double vx = (jx + Fx / om) / r, vy = (jy + Fy / om) / r;
            const double usq = vx * vx + vy * vy;
            double rb = 0.0, vbx = 0.0, vby = 0.0;
            for (int i = 0; i < 9; ++i) {
                const double cu = CX[i] * vx + CY[i] * vy;
                const double feq = W[i] * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                rb += om * ls[i] * feq / r;                           /* d feq / d rho */
                vbx += om * ls[i] * W[i] * r * (3.0 * CX[i] + 9.0 * cu * CX[i] - 3.0 * vx);
                vby += om * ls[i] * W[i] * r * (3.0 * CY[i] + 9.0 * cu * CY[i] - 3.0 * vy);
            }
            /* v = (j + F/om) / rho */
            jbx[s] = vbx / r;
            jby[s] = vby / r;
            const double Fbx = vbx / (om * r), Fby = vby / (om * r);
            rb -= (vbx * vx + vby * vy) / r;
            /* F = -psi S: the leading psi(x) and the couplings */
            const double dpsi = exp_cr(-r / P->rho0) / sqrt(P->rho0);
            rbar[s] = rb + dpsi * (-(Fbx * Sx + Fby * Sy));
            Qx[s] = ps * Fbx;
            Qy[s] = ps * Fby;
            g1 += -ps * (Fbx * Swx + Fby * Swy);
            g2 += -ps * (Fbx * Spx + Fby * Spy);
        }
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            const long s = y * nx + x;
            /* psi(y) inside the neighbours' forces: sum_c K_c c . Q(y + c) */
            double pb = 0.0;
            for (int i = 1; i <= 8; ++i) {
                const long n = site(P, x + CX[i], y + CY[i]);
                const double K = P->G1 * W[i] + P->G2 * PS[i];
                pb += K * (CX[i] * Qx[n] + CY[i] * Qy[n]);
            }
            for (int k = 0; k < 16; ++k) {
                const long n = site(P, x + MCX[k], y + MCY[k]);
                pb += P->G2 * PM[k] * (MCX[k] * Qx[n] + MCY[k] * Qy[n]);
            }
            const double dpsi = exp_cr(-rho[s] / P->rho0) / sqrt(P->rho0);
            const double rb = rbar[s] + dpsi * pb;
            for (int i = 0; i < 9; ++i) {
                const double li = lam_next[i * N + site(P, x + CX[i], y + CY[i])];
                lam[i * N + s] = (1.0 - om) * li + rb + CX[i] * jbx[s] + CY[i] * jby[s];
            }
        }
    gG[0] += g1;
    gG[1] += g2;
    free(rho); free(psi); free(Qx); free(Qy); free(rbar); free(jbx); free(jby);
}

double orc_objective(const orc_params* P, const double* rho_init, long steps,
                     const double* rho_target, double* E_out)
{
    if (!params_ok(P) || steps < 0) return NAN;
    const long N = (long)P->nx * P->ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* d = (double*)malloc(sizeof(double) * N);
    if (!rho || !psi || !d ||
        orc_run(P, rho_init, steps, 0, rho, NULL, NULL, NULL, 0, NULL) != 0) {
        free(rho); free(psi); free(d);
        return NAN;
    }
    orc_psi(N, rho, P->rho0, psi);
    double g1, g2;
    const double E = energy_and_derivatives(P, psi, d, &g1, &g2);
    double mis = 0.0;
    for (long s = 0; s < N; ++s) mis += (rho[s] - rho_target[s]) * (rho[s] - rho_target[s]);
    if (E_out) *E_out = E;
    free(rho); free(psi); free(d);
    return E + mis;
}

int orc_gradient(const orc_params* P, const double* rho_init, long steps,
                 const double* rho_target, double* J, double* grad_rho, double* grad_G)
{
    if (!params_ok(P) || steps < 0) return -1;
    const long N = (long)P->nx * P->ny;
    double* f = (double*)malloc(sizeof(double) * 9 * N * (size_t)(steps + 1));
    double* la = (double*)malloc(sizeof(double) * 9 * N);
    double* lb = (double*)malloc(sizeof(double) * 9 * N);
    double* rho = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* dEdpsi = (double*)malloc(sizeof(double) * N);
    if (!f || !la || !lb || !rho || !psi || !dEdpsi) {
        free(f); free(la); free(lb); free(rho); free(psi); free(dEdpsi);
        return -1;
    }
    orc_init(P, rho_init, f);
    for (long t = 0; t < steps; ++t) orc_step(P, f + 9 * N * t, f + 9 * N * (t + 1));
    const double* fT = f + 9 * N * steps;
    psi_field(P, fT, rho, psi);
    double gE1, gE2;
    const double E = energy_and_derivatives(P, psi, dEdpsi, &gE1, &gE2);
    double mis = 0.0;
    for (long s = 0; s < N; ++s) mis += (rho[s] - rho_target[s]) * (rho[s] - rho_target[s]);
    *J = E + mis;
    /* terminal adjoint: dJ/df_i(y, T) = psi'(rho) dE/dpsi + 2 (rho - rho_target) */
    for (long s = 0; s < N; ++s) {
        const double v = exp_cr(-rho[s] / P->rho0) / sqrt(P->rho0) * dEdpsi[s] +
                         2.0 * (rho[s] - rho_target[s]);
        for (int i = 0; i < 9; ++i) la[i * N + s] = v;
    }
    grad_G[0] = gE1;
    grad_G[1] = gE2;
    for (long t = steps - 1; t >= 0; --t) {
        adjoint_step(P, f + 9 * N * t, la, lb, grad_G);
        double* tmp = la; la = lb; lb = tmp;
    }
    /* f_i(x, 0) = w_i rho_init(x) */
    for (long s = 0; s < N; ++s) {
        double g = 0.0;
        for (int i = 0; i < 9; ++i) g += W[i] * la[i * N + s];
        grad_rho[s] = g;
    }
    free(f); free(la); free(lb); free(rho); free(psi); free(dEdpsi);
    return 0;
}

/* One reverse step on its own (for the dot-product identity): lam = J_step^T lam_next
 * at state f; gG (2 doubles) receives the explicit G1, G2 terms. */
void orc_adjoint_step(const orc_params* P, const double* f, const double* lam_next, double* lam,
                      double* gG)
{
    gG[0] = 0.0;
    gG[1] = 0.0;
    adjoint_step(P, f, lam_next, lam, gG);
}

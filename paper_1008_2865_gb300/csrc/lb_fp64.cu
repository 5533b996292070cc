// lb_fp64.cu — FP64 parity path of the two-belt Shan–Chen D2Q9 step
// (Chibbaro et al., arXiv:1008.2865). Built with --fmad=false: every
// product and sum below is a separately rounded IEEE operation.
//
// The operation order is the plain per-site reading of the paper:
//   rho, rho u summed over i = 0..8 in the D2Q9 order (Eqs. 2-3);
//   psi = sqrt(rho0) (1 - exp(-rho/rho0)) (Sec. 2) with exp correctly rounded;
//   Eq. FORCE as three link sums — w_i on belt 1, p_si on belt 1, p_mi on
//   belt 2, each term (weight * psi) * c — combined as
//   F = -((G1 psi) S_w + (G2 psi) S_s + (G2 psi) S_m) (the minus sign of
//   Eq. forza);
//   u = j/rho, u_eq = u + F/(omega rho), Eq. 4 with coefficients 3, 9/2, 3/2
//   (cs2 = 1/3), f* = f - omega (f - feq), then push-streaming.
// With identical order and correctly rounded exp, the result of each step is
// fixed bit for bit by these definitions, so any other evaluation that
// follows them reproduces it exactly. The state is f(t) after streaming.
// This path is for verification; it is not tuned.
#include "lb_internal.h"

namespace lbsc {
namespace {

__device__ __forceinline__ int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// ---------------------------------------------------------------- exp
// Correctly rounded exp(x) for the finite x the lattice produces
// (|x| < 700): double-double arithmetic after Dekker (1971) and Knuth's
// TwoSum, argument reduction x = k ln2 + r with a double-double ln 2,
// r/1024 fed to the Taylor series of e^r - 1, ten squarings through
// (e^{2a} - 1) = m (m + 2) to avoid cancellation, and one final rounding of
// the double-double 1 + m, then scaling by 2^k (exact). The double-double
// result carries ~100 significant bits, so its rounding to double equals the
// correctly rounded exp except when e^x lies within ~2^-100 relative of a
// rounding boundary.
struct dd {
    double hi, lo;
};

__host__ __device__ __forceinline__ dd two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    const double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__host__ __device__ __forceinline__ dd quick_two_sum(double a, double b)
{
    const double s = a + b;
    return {s, b - (s - a)};
}

__host__ __device__ __forceinline__ dd two_prod(double a, double b)
{
    const double p = a * b;
    return {p, fma(a, b, -p)};
}

__host__ __device__ __forceinline__ dd dd_add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    const dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ dd dd_add_d(dd a, double b)
{
    dd s = two_sum(a.hi, b);
    s.lo += a.lo;
    return quick_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ dd dd_mul(dd a, dd b)
{
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}

__host__ __device__ __forceinline__ dd dd_div_d(dd a, double b)
{
    const double q1 = a.hi / b;
    const dd p = two_prod(q1, b);
    const dd s = two_sum(a.hi, -p.hi);
    const double e = (s.lo - p.lo) + a.lo;
    const double q2 = (s.hi + e) / b;
    return quick_two_sum(q1, q2);
}

__host__ __device__ double exp_cr(double x)
{
    // ln 2 = LN2_HI + LN2_LO to ~2^-107 (the two leading double parts of ln 2)
    const double LN2_HI = 6.93147180559945286227e-01;
    const double LN2_LO = 2.31904681384629955842e-17;
    const double LOG2E = 1.44269504088896338700e+00;
    if (x == 0.0) return 1.0;
    if (!(x > -700.0 && x < 700.0)) return exp(x);   // outside the lattice's range
    const double k = rint(x * LOG2E);
    // r = x - k ln2 in double-double
    const dd p1 = two_prod(k, LN2_HI);
    const dd p2 = two_prod(k, LN2_LO);
    dd r = dd_add({x, 0.0}, {-p1.hi, -p1.lo});
    r = dd_add(r, {-p2.hi, -p2.lo});
    // r' = r / 2^10 (exact)
    const dd rs = {r.hi * 0.0009765625, r.lo * 0.0009765625};
    // e^r' - 1 = r'(1 + r'/2 (1 + r'/3 (1 + ... (1 + r'/11))))
    dd q = dd_add_d(dd_div_d(rs, 11.0), 1.0);
    for (int n = 10; n >= 2; --n) q = dd_add_d(dd_div_d(dd_mul(rs, q), (double)n), 1.0);
    dd m = dd_mul(rs, q);
    for (int i = 0; i < 10; ++i) m = dd_mul(m, dd_add_d(m, 2.0));
    const dd e = dd_add_d(m, 1.0);
    const double v = e.hi + e.lo;     // the one rounding to double
    return ldexp(v, (int)k);
}

// ---------------------------------------------------------------- lattice
// D2Q9 (Sec. 2) in the order (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
__constant__ int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
// Table 1, belt 1 weights on the same eight speeds
__constant__ double PS[9] = {0.0, 4.0 / 63.0, 4.0 / 63.0, 4.0 / 63.0, 4.0 / 63.0,
                             4.0 / 135.0, 4.0 / 135.0, 4.0 / 135.0, 4.0 / 135.0};
// Table 1, belt 2: |c|^2 = 4 (i = 1..4), 5 (i = 5..12), 8 (i = 13..16)
__constant__ int MX[16] = {2, 0, -2, 0, 2, 1, -1, -2, -2, -1, 1, 2, 2, -2, -2, 2};
__constant__ int MY[16] = {0, 2, 0, -2, 1, 2, 2, 1, -1, -2, -2, -1, 2, 2, -2, -2};
__constant__ double PM[16] = {1.0 / 180.0, 1.0 / 180.0, 1.0 / 180.0, 1.0 / 180.0,
                              2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0,
                              2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0,
                              1.0 / 15120.0, 1.0 / 15120.0, 1.0 / 15120.0, 1.0 / 15120.0};

__device__ __forceinline__ long long site(int x, int y, int nx, int ny)
{
    return (long long)wrapi(y, ny) * nx + wrapi(x, nx);
}

__device__ __forceinline__ void moments(const double* f, long long N, long long s, double& rho,
                                        double& jx, double& jy)
{
    double r = 0.0, ax = 0.0, ay = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double fi = f[i * N + s];
        r = r + fi;
        ax = ax + (double)CX[i] * fi;
        ay = ay + (double)CY[i] * fi;
    }
    rho = r;
    jx = ax;
    jy = ay;
}

__global__ void k64_init(double* __restrict__ f, const double* __restrict__ rho, int nx, int ny)
{
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i * N + s] = W[i] * rho[s];
    }
}

__global__ void k64_psi(const Fp64Args a)
{
    const long long N = (long long)a.nx * a.ny;
    const double sq = sqrt(a.rho0);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        double r, jx, jy;
        moments(a.f_in, N, s, r, jx, jy);
        a.rho[s] = r;
        a.psi[s] = sq * (1.0 - exp_cr(-r / a.rho0));
    }
}

__global__ void k64_collide_stream(const Fp64Args a)
{
    const int nx = a.nx, ny = a.ny;
    const long long N = (long long)nx * ny;
    const double om = a.omega;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s % nx);
        double rho, jx, jy;
        moments(a.f_in, N, s, rho, jx, jy);
        double wx = 0.0, wy = 0.0, sx = 0.0, sy = 0.0, mx = 0.0, my = 0.0;
#pragma unroll
        for (int i = 1; i <= 8; ++i) {
            const double pn = a.psi[site(x + CX[i], y + CY[i], nx, ny)];
            wx = wx + (W[i] * pn) * (double)CX[i];
            wy = wy + (W[i] * pn) * (double)CY[i];
            sx = sx + (PS[i] * pn) * (double)CX[i];
            sy = sy + (PS[i] * pn) * (double)CY[i];
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const double pn = a.psi[site(x + MX[k], y + MY[k], nx, ny)];
            mx = mx + (PM[k] * pn) * (double)MX[k];
            my = my + (PM[k] * pn) * (double)MY[k];
        }
        const double ps = a.psi[s];
        const double Fsx = (a.G1 * ps) * wx + (a.G2 * ps) * sx;
        const double Fsy = (a.G1 * ps) * wy + (a.G2 * ps) * sy;
        const double Fmx = (a.G2 * ps) * mx;
        const double Fmy = (a.G2 * ps) * my;
        const double Fx = -(Fsx + Fmx);
        const double Fy = -(Fsy + Fmy);
        const double ux = jx / rho;
        const double uy = jy / rho;
        const double orho = om * rho;
        const double vx = ux + Fx / orho;
        const double vy = uy + Fy / orho;
        const double usq = vx * vx + vy * vy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double cu = (double)CX[i] * vx + (double)CY[i] * vy;
            const double feq = (W[i] * rho) * (((1.0 + 3.0 * cu) + (4.5 * cu) * cu) - 1.5 * usq);
            const double fi = a.f_in[i * N + s];
            a.f_out[i * N + site(x + CX[i], y + CY[i], nx, ny)] = fi - om * (fi - feq);
        }
    }
}

template <int NT>
__device__ void block_sum4(double v[4])
{
    __shared__ double red[NT / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) red[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w) {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] += red[w][k];
        }
    }
    __syncthreads();
}

// Sec. 5 energies of psi(t) and the mass of rho(t); the last CTA to finish
// sums the CTA partials in a fixed order, writes out4 = {E_s, E_m, E_bulk,
// mass} and, if trace is given, appends (t, mass, E_s, E_m, E_bulk).
__global__ void __launch_bounds__(256) k64_energy(const Fp64Args a, double* partials,
                                                  unsigned int* counter, double* out4,
                                                  double* trace, int* trace_count, long long t)
{
    const int nx = a.nx, ny = a.ny;
    const long long N = (long long)nx * ny;
    // rest weight of the E(8) set from Eq. weights_1
    double p0 = 0.0;
    for (int i = 1; i <= 8; ++i) p0 = p0 + PS[i];
    for (int k = 0; k < 16; ++k) p0 = p0 + PM[k];
    p0 = 1.0 - p0;
    const double A1 = a.G1 + a.G2;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < N; s += (long long)gridDim.x * 256) {
        const int y = (int)(s / nx), x = (int)(s % nx);
        const double ps = a.psi[s];
        double ss = (a.G1 * W[0] + a.G2 * p0) * ps;
        for (int i = 1; i <= 8; ++i)
            ss = ss + (a.G1 * W[i] + a.G2 * PS[i]) * a.psi[site(x + CX[i], y + CY[i], nx, ny)];
        double sm = 0.0;
        for (int k = 0; k < 16; ++k)
            sm = sm + (a.G2 * PM[k]) * a.psi[site(x + MX[k], y + MY[k], nx, ny)];
        v[0] = v[0] + (0.5 * ps) * ss;
        v[1] = v[1] + (0.5 * ps) * sm;
        v[2] = v[2] + ((0.5 * A1) * ps) * ps;
        v[3] = v[3] + a.rho[s];
    }
    __shared__ bool s_last;
    block_sum4<256>(v);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) partials[4 * (size_t)blockIdx.x + k] = v[k];
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned int j = threadIdx.x; j < gridDim.x; j += 256) {
        for (int k = 0; k < 4; ++k) w[k] += __ldcg(partials + 4 * (size_t)j + k);
    }
    block_sum4<256>(w);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) out4[k] = w[k];
        if (trace) {
            const int c = *trace_count;
            double* row = trace + (size_t)(c % kTraceCap) * kTraceCols;
            row[0] = (double)t;
            row[1] = w[3];
            row[2] = w[0];
            row[3] = w[1];
            row[4] = w[2];
            *trace_count = c + 1;
        }
        *counter = 0u;
    }
}

__global__ void k64_fields(const double* __restrict__ f, int nx, int ny, double* rho, double* ux,
                           double* uy)
{
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        double r, jx, jy;
        moments(f, N, s, r, jx, jy);
        if (rho) rho[s] = r;
        if (ux) ux[s] = jx / r;
        if (uy) uy[s] = jy / r;
    }
}

__global__ void k64_exp(const double* __restrict__ x, double* __restrict__ y, long long n)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x)
        y[s] = exp_cr(x[s]);
}

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t fp64_init(double* f, const double* rho_init, int nx, int ny, cudaStream_t s)
{
    k64_init<<<grid_for((long long)nx * ny), 256, 0, s>>>(f, rho_init, nx, ny);
    return cudaGetLastError();
}

cudaError_t fp64_psi(const Fp64Args& a, cudaStream_t s)
{
    k64_psi<<<grid_for((long long)a.nx * a.ny), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t fp64_collide_stream(const Fp64Args& a, cudaStream_t s)
{
    k64_collide_stream<<<grid_for((long long)a.nx * a.ny), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t fp64_energy(const Fp64Args& a, double* partials, unsigned int* counter, double* out4,
                        double* trace, int* trace_count, long long t, cudaStream_t s)
{
    k64_energy<<<grid_for((long long)a.nx * a.ny), 256, 0, s>>>(a, partials, counter, out4, trace,
                                                                trace_count, t);
    return cudaGetLastError();
}

cudaError_t fp64_fields(const double* f, int nx, int ny, double* rho, double* ux, double* uy,
                        cudaStream_t s)
{
    k64_fields<<<grid_for((long long)nx * ny), 256, 0, s>>>(f, nx, ny, rho, ux, uy);
    return cudaGetLastError();
}

cudaError_t fp64_exp_cr(const double* x, double* y, long long n, cudaStream_t s)
{
    k64_exp<<<grid_for(n), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

}  // namespace lbsc

// lb_fp32.cu — fused single-pass step of the two-belt Shan–Chen D2Q9 lattice
// Boltzmann method (Chibbaro et al., arXiv:1008.2865) for sm_103a, with the
// populations stored as deviations from the rest equilibrium at rho_ref.
//
// State between steps: g*(t-1) = post-collision deviations f*_i - w_i rho_ref
// (SoA [9][ny][nx]) and dpsi(t) = psi(rho(t)) - psi(rho_ref) ([ny][nx]).
// One launch advances t -> t+1 and moves ~80 bytes per site in FP32:
// 36 B of g* read, 36 B written, 4 B of dpsi read, 4 B written.
//
// Work decomposition. A CTA of BX threads owns a strip of BX-2 output
// columns and `rows` output rows; thread k sits on column x0-1+k, so the two
// edge threads are the one-column halo whose collisions the interior needs.
// The CTA marches down its rows. For collision row r it
//   1. pulls f_i(x, r) = f*_i(x - c_i, r) from global memory (Eq. 1 streaming,
//      periodic) — the loads of row r+1 are issued before row r is computed;
//   2. forms rho, j (Eqs. 2-3) and reads psi(t) of the 25-site stencil from a
//      ring of 8 dpsi rows kept in shared memory (each dpsi row is read from
//      HBM once per CTA);
//   3. evaluates the two-belt force of Eq. FORCE in pair form, grouped by
//      |c|^2 (the constant psi_ref cancels in every antisymmetric pair);
//   4. relaxes towards the Eq. 4 equilibrium at u + F/(omega rho) and stores
//      g*(t) for its own column;
//   5. hands its three right-moving and three left-moving post-collision
//      values to the neighbouring threads through shared memory, so that
//      every thread accumulates rho(t+1) = sum_i f*_i(x - c_i) of rows r-1,
//      r, r+1 in three rolling registers; row r-1 is then complete and its
//      dpsi(t+1) is written.
// One __syncthreads per row orders the exchange and the ring updates.
// REDUCE launches also accumulate mass and the Sec. 5 pseudo-energies of
// state t (FP32 per thread for 16 rows, then FP64), reduce them per CTA in
// FP64 and let the last CTA to finish sum all CTA partials in a fixed order
// into one trace row — deterministic for a given launch shape.
#include "lb_internal.h"

#include <cmath>

namespace lbsc {
namespace {

__device__ __forceinline__ float ldg_(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st_(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_(__half* p, float v) { *p = __float2half_rn(v); }

__device__ __forceinline__ int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// Deterministic sum of 4 doubles over a CTA of NT threads (NT a multiple of
// 32, at most 1024); the result is valid in thread 0.
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

// Store this CTA's partial, and if it is the last CTA to arrive, sum all
// partials (each thread a fixed strided subset, then a fixed tree) and return
// true in thread 0 with the total in v. Resets the counter for the next use.
template <int NT>
__device__ bool last_block_total(double v[4], double* partials, unsigned int* counter,
                                 unsigned int nblocks)
{
    __shared__ bool s_last;
    const unsigned int b = blockIdx.y * gridDim.x + blockIdx.x;
    block_sum4<NT>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) partials[4 * (size_t)b + k] = v[k];
        __threadfence();
        const unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned int j = threadIdx.x; j < nblocks; j += NT) {
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] += __ldcg(partials + 4 * (size_t)j + k);
    }
    block_sum4<NT>(w);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = w[k];
        *counter = 0u;
    }
    return threadIdx.x == 0;
}

__device__ __forceinline__ void write_trace_row(double* trace, int* trace_count, long long t,
                                                double mass, double es, double em, double eb)
{
    const int c = *trace_count;
    double* row = trace + (size_t)(c % kTraceCap) * kTraceCols;
    row[0] = (double)t;
    row[1] = mass;
    row[2] = es;
    row[3] = em;
    row[4] = eb;
    *trace_count = c + 1;
}

// Pull f_i(x, r) = f*_i(x - c_i, r - c_iy) for the 9 D2Q9 speeds in the order
// (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
template <typename T>
__device__ __forceinline__ void pull(float f[9], const T* __restrict__ g, long long N,
                                     long long om, long long oc, long long op, int xm, int xc,
                                     int xp)
{
    f[0] = ldg_(g + oc + xc);
    f[1] = ldg_(g + N + oc + xm);
    f[2] = ldg_(g + 2 * N + om + xc);
    f[3] = ldg_(g + 3 * N + oc + xp);
    f[4] = ldg_(g + 4 * N + op + xc);
    f[5] = ldg_(g + 5 * N + om + xm);
    f[6] = ldg_(g + 6 * N + om + xp);
    f[7] = ldg_(g + 7 * N + op + xp);
    f[8] = ldg_(g + 8 * N + op + xm);
}

template <typename T, int BX, bool REDUCE>
__global__ void __launch_bounds__(BX) k_step(const StepArgs<T> a)
{
    constexpr int W = BX + 4;
    __shared__ float win[8][W];              // dpsi(t) rows, slot = row & 7
    __shared__ float4 exR[2][BX + 2];        // right-moving f*: (cy=-1, 0, +1)
    __shared__ float4 exL[2][BX + 2];        // left-moving f*

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const long long N = a.N;
    const int x0 = blockIdx.x * (BX - 2);
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, ny);
    const int txe = min(BX - 2, nx - x0);
    const bool out_col = tid >= 1 && tid <= txe;
    const int xc = wrapi(x0 - 1 + tid, nx);
    const int xm = xc == 0 ? nx - 1 : xc - 1;
    const int xp = xc == nx - 1 ? 0 : xc + 1;
    const int pc0 = wrapi(x0 - 3 + tid, nx);
    const int pc1 = wrapi(x0 - 3 + BX + (tid & 3), nx);

    // dpsi rows y0-3 .. y0+1 into the ring
    for (int rr = y0 - 3; rr <= y0 + 1; ++rr) {
        const float* src = a.dpsi_in + (long long)wrapi(rr, ny) * nx;
        win[rr & 7][tid] = __ldg(src + pc0);
        if (tid < 4) win[rr & 7][BX + tid] = __ldg(src + pc1);
    }

    float f[9];
    {
        const int r = y0 - 1;
        pull(f, a.g_in, N, (long long)wrapi(r - 1, ny) * nx, (long long)wrapi(r, ny) * nx,
             (long long)wrapi(r + 1, ny) * nx, xm, xc, xp);
    }
    __syncthreads();

    float acc_m = 0.f, acc_0 = 0.f;
    float es = 0.f, em = 0.f, eb = 0.f, ms = 0.f;
    double d_es = 0.0, d_em = 0.0, d_eb = 0.0, d_ms = 0.0;

    for (int r = y0 - 1; r <= y1; ++r) {
        // ---- prefetch: dpsi row r+3 and the pulled populations of row r+1
        const bool need_psi = r <= y1 - 1;
        float pn0 = 0.f, pn1 = 0.f;
        if (need_psi) {
            const float* src = a.dpsi_in + (long long)wrapi(r + 3, ny) * nx;
            pn0 = __ldg(src + pc0);
            if (tid < 4) pn1 = __ldg(src + pc1);
        }
        float fn[9];
        if (r < y1) {
            pull(fn, a.g_in, N, (long long)wrapi(r, ny) * nx, (long long)wrapi(r + 1, ny) * nx,
                 (long long)wrapi(r + 2, ny) * nx, xm, xc, xp);
        }

        // ---- force from the dpsi(t) ring (Eq. FORCE, pair form)
        const float* rM2 = &win[(r - 2) & 7][tid + 2];
        const float* rM1 = &win[(r - 1) & 7][tid + 2];
        const float* rC = &win[r & 7][tid + 2];
        const float* rP1 = &win[(r + 1) & 7][tid + 2];
        const float* rP2 = &win[(r + 2) & 7][tid + 2];
        const float pc = a.psi_ref + rC[0];
        float Sx, Sy;
        {
            const float d10 = rC[1] - rC[-1];
            const float d01 = rP1[0] - rM1[0];
            const float d11 = rP1[1] - rM1[-1];   // (1,1) - (-1,-1)
            const float d1m = rM1[1] - rP1[-1];   // (1,-1) - (-1,1)
            const float d20 = rC[2] - rC[-2];
            const float d02 = rP2[0] - rM2[0];
            const float da = rP1[2] - rM1[-2];    // (2,1) - (-2,-1)
            const float db = rP2[1] - rM2[-1];    // (1,2) - (-1,-2)
            const float dc = rP2[-1] - rM2[1];    // (-1,2) - (1,-2)
            const float dd = rP1[-2] - rM1[2];    // (-2,1) - (2,-1)
            const float e1 = rP2[2] - rM2[-2];    // (2,2) - (-2,-2)
            const float e2 = rM2[2] - rP2[-2];    // (2,-2) - (-2,2)
            Sx = a.K1 * d10 + a.K2 * (d11 + d1m) + 2.f * a.K4 * d20 +
                 a.K5 * (2.f * (da - dd) + (db - dc)) + 2.f * a.K8 * (e1 + e2);
            Sy = a.K1 * d01 + a.K2 * (d11 - d1m) + 2.f * a.K4 * d02 +
                 a.K5 * ((da + dd) + 2.f * (db + dc)) + 2.f * a.K8 * (e1 - e2);
        }
        const float Fx = -pc * Sx;
        const float Fy = -pc * Sy;

        // ---- moments and BGK collision at the shifted velocity (Eqs. 2-4)
        const float d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
        const float rho = a.rho_ref + d;
        const float inv = __frcp_rn(rho);
        const float ux = fmaf(Fx, a.inv_omega, jx) * inv;
        const float uy = fmaf(Fy, a.inv_omega, jy) * inv;
        const float usq15 = 1.5f * fmaf(ux, ux, uy * uy);
        const float orho = a.omega * rho;
        const float A0 = orho * a.w0, A1 = orho * a.w1, A2 = orho * a.w2;
        const float od = a.omega * d;
        const float D0 = od * a.w0, D1 = od * a.w1, D2 = od * a.w2;
        const float omc = a.omc;
        float gs[9];
        gs[0] = fmaf(omc, f[0], fmaf(A0, -usq15, D0));
        {
            const float s = fmaf(4.5f * ux, ux, -usq15), t3 = 3.f * ux;
            gs[1] = fmaf(omc, f[1], fmaf(A1, s + t3, D1));
            gs[3] = fmaf(omc, f[3], fmaf(A1, s - t3, D1));
        }
        {
            const float s = fmaf(4.5f * uy, uy, -usq15), t3 = 3.f * uy;
            gs[2] = fmaf(omc, f[2], fmaf(A1, s + t3, D1));
            gs[4] = fmaf(omc, f[4], fmaf(A1, s - t3, D1));
        }
        {
            const float c = ux + uy;
            const float s = fmaf(4.5f * c, c, -usq15), t3 = 3.f * c;
            gs[5] = fmaf(omc, f[5], fmaf(A2, s + t3, D2));
            gs[7] = fmaf(omc, f[7], fmaf(A2, s - t3, D2));
        }
        {
            const float c = uy - ux;
            const float s = fmaf(4.5f * c, c, -usq15), t3 = 3.f * c;
            gs[6] = fmaf(omc, f[6], fmaf(A2, s + t3, D2));
            gs[8] = fmaf(omc, f[8], fmaf(A2, s - t3, D2));
        }

        const bool out_row = r >= y0 && r < y1;
        if (out_col && out_row) {
            T* o = a.g_out + (long long)r * nx + xc;
#pragma unroll
            for (int i = 0; i < 9; ++i) st_(o + i * N, gs[i]);
            if (REDUCE) {
                // Sec. 5 pseudo-energies of state t at (x, r), psi = psi_ref + dpsi
                const float pr = a.psi_ref;
                const float S1 = (rC[1] + rC[-1]) + (rP1[0] + rM1[0]);
                const float S2 = (rP1[1] + rP1[-1]) + (rM1[1] + rM1[-1]);
                const float S4 = (rC[2] + rC[-2]) + (rP2[0] + rM2[0]);
                const float S5 = ((rP1[2] + rP1[-2]) + (rM1[2] + rM1[-2])) +
                                 ((rP2[1] + rP2[-1]) + (rM2[1] + rM2[-1]));
                const float S8 = (rP2[2] + rP2[-2]) + (rM2[2] + rM2[-2]);
                const float b1 = a.K0 * pc + a.K1 * fmaf(4.f, pr, S1) + a.K2 * fmaf(4.f, pr, S2);
                const float b2 = a.K4 * fmaf(4.f, pr, S4) + a.K5 * fmaf(8.f, pr, S5) +
                                 a.K8 * fmaf(4.f, pr, S8);
                es = fmaf(0.5f * pc, b1, es);
                em = fmaf(0.5f * pc, b2, em);
                eb = fmaf(a.half_A1 * pc, pc, eb);
                ms += d;
                if (((r - y0) & 15) == 15) {
                    d_es += es; d_em += em; d_eb += eb; d_ms += ms;
                    es = em = eb = ms = 0.f;
                }
            }
        }

        // ---- exchange post-collision values with the neighbouring columns
        exR[r & 1][tid + 1] = make_float4(gs[8], gs[1], gs[5], 0.f);
        exL[r & 1][tid + 1] = make_float4(gs[7], gs[3], gs[6], 0.f);
        if (need_psi) {
            win[(r + 3) & 7][tid] = pn0;
            if (tid < 4) win[(r + 3) & 7][BX + tid] = pn1;
        }
        __syncthreads();
        const float4 R = exR[r & 1][tid];       // from column x-1
        const float4 L = exL[r & 1][tid + 2];   // from column x+1
        acc_m += gs[4] + (R.x + L.x);
        acc_0 += gs[0] + (R.y + L.y);
        const float acc_p = gs[2] + (R.z + L.z);
        if (out_col && r - 1 >= y0) {
            // psi(t+1) - psi_ref = -sqrt(rho0) e^{-rho_ref/rho0} expm1(-(rho - rho_ref)/rho0)
            a.dpsi_out[(long long)(r - 1) * nx + xc] = a.cpsi * expm1f(-acc_m * a.inv_rho0);
        }
        acc_m = acc_0;
        acc_0 = acc_p;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fn[i];
    }

    if (REDUCE) {
        double v[4] = {d_es + es, d_em + em, d_eb + eb, d_ms + ms};
        const unsigned int nb = gridDim.x * gridDim.y;
        if (last_block_total<BX>(v, a.partials, a.counter, nb)) {
            const double mass = (double)a.N * (double)a.rho_ref + v[3];
            write_trace_row(a.trace, a.trace_count, a.t, mass, v[0], v[1], v[2]);
        }
    }
}

// ---------------------------------------------------------------- helpers

template <typename T>
__global__ void k_delta_init(T* __restrict__ g, float* __restrict__ dpsi,
                             const double* __restrict__ rho, int nx, int ny, double rho_ref,
                             double rho0)
{
    const long long N = (long long)nx * ny;
    const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                         1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double cpsi = -sqrt(rho0) * exp(-rho_ref / rho0);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s % nx);
        // f*_i(x) such that the first pull gives f_i(x, 0) = w_i rho_init(x)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const long long src = (long long)wrapi(y + cy[i], ny) * nx + wrapi(x + cx[i], nx);
            st_(g + i * N + s, (float)(w[i] * (rho[src] - rho_ref)));
        }
        dpsi[s] = (float)(cpsi * expm1(-(rho[s] - rho_ref) / rho0));
    }
}

template <typename T>
__global__ void k_delta_fields(const T* __restrict__ g, int nx, int ny, double rho_ref,
                               double* __restrict__ rho, double* __restrict__ ux,
                               double* __restrict__ uy)
{
    const long long N = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / nx), x = (int)(s % nx);
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const long long om = (long long)(y == 0 ? ny - 1 : y - 1) * nx;
        const long long oc = (long long)y * nx;
        const long long op = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
        float f[9];
        pull(f, g, N, om, oc, op, xm, x, xp);
        double d = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) d += (double)f[i];
        jx = ((double)f[1] - f[3]) + ((double)f[5] - f[6]) + ((double)f[8] - f[7]);
        jy = ((double)f[2] - f[4]) + ((double)f[5] + f[6]) - ((double)f[7] + f[8]);
        const double r = rho_ref + d;
        if (rho) rho[s] = r;
        if (ux) ux[s] = jx / r;
        if (uy) uy[s] = jy / r;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_delta_energy(const T* __restrict__ g,
                                                      const float* __restrict__ dpsi,
                                                      const StepArgs<T> a, double* out4)
{
    const int nx = a.nx, ny = a.ny;
    const long long N = a.N;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const double pr = a.psi_ref;
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < N; s += (long long)gridDim.x * 256) {
        const int y = (int)(s / nx), x = (int)(s % nx);
        auto P = [&](int dx, int dy) -> double {
            return (double)dpsi[(long long)wrapi(y + dy, ny) * nx + wrapi(x + dx, nx)];
        };
        const double pc = pr + P(0, 0);
        const double S1 = P(1, 0) + P(-1, 0) + P(0, 1) + P(0, -1);
        const double S2 = P(1, 1) + P(-1, 1) + P(1, -1) + P(-1, -1);
        const double S4 = P(2, 0) + P(-2, 0) + P(0, 2) + P(0, -2);
        const double S5 = P(2, 1) + P(-2, 1) + P(2, -1) + P(-2, -1) + P(1, 2) + P(-1, 2) +
                          P(1, -2) + P(-1, -2);
        const double S8 = P(2, 2) + P(-2, 2) + P(2, -2) + P(-2, -2);
        const double b1 = (double)a.K0 * pc + (double)a.K1 * (4 * pr + S1) + (double)a.K2 * (4 * pr + S2);
        const double b2 = (double)a.K4 * (4 * pr + S4) + (double)a.K5 * (8 * pr + S5) +
                          (double)a.K8 * (4 * pr + S8);
        v[0] += 0.5 * pc * b1;
        v[1] += 0.5 * pc * b2;
        v[2] += (double)a.half_A1 * pc * pc;
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const long long om = (long long)(y == 0 ? ny - 1 : y - 1) * nx;
        const long long op = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
        float f[9];
        pull(f, g, N, om, (long long)y * nx, op, xm, x, xp);
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) d += (double)f[i];
        v[3] += d;
    }
    if (last_block_total<256>(v, a.partials, a.counter, gridDim.x)) {
        out4[0] = v[0];
        out4[1] = v[1];
        out4[2] = v[2];
        out4[3] = (double)N * (double)a.rho_ref + v[3];
    }
}

__global__ void __launch_bounds__(256) k_rho_check_sum(const double* __restrict__ rho, long long n,
                                                       double* partials, unsigned int* counter,
                                                       double* out_sum, int* flag)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < n; s += (long long)gridDim.x * 256) {
        const double r = rho[s];
        bad |= !(r > 0.0) || !isfinite(r);
        v[0] += r;
    }
    if (bad) atomicOr(flag, 1);
    if (last_block_total<256>(v, partials, counter, gridDim.x)) *out_sum = v[0];
}

template <typename T, int BX>
cudaError_t launch_step_bx(const StepArgs<T>& a, Fp32Launch L, bool reduce, cudaStream_t s)
{
    dim3 grid((a.nx + BX - 3) / (BX - 2), (a.ny + L.rows - 1) / L.rows);
    if (reduce)
        k_step<T, BX, true><<<grid, BX, 0, s>>>(a);
    else
        k_step<T, BX, false><<<grid, BX, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(const StepArgs<T>& a, Fp32Launch L, bool reduce, cudaStream_t s)
{
    switch (L.block_x) {
    case 64: return launch_step_bx<T, 64>(a, L, reduce, s);
    case 96: return launch_step_bx<T, 96>(a, L, reduce, s);
    case 128: return launch_step_bx<T, 128>(a, L, reduce, s);
    case 192: return launch_step_bx<T, 192>(a, L, reduce, s);
    case 256: return launch_step_bx<T, 256>(a, L, reduce, s);
    default: return cudaErrorInvalidValue;
    }
}

int grid_blocks_for(int n, int per) { return (n + per - 1) / per; }

}  // namespace

int fp32_grid_blocks(int nx, int ny, Fp32Launch L)
{
    return grid_blocks_for(nx, L.block_x - 2) * grid_blocks_for(ny, L.rows);
}

cudaError_t fp32_step(const StepArgs<float>& a, Fp32Launch L, bool reduce, cudaStream_t s)
{
    return launch_step<float>(a, L, reduce, s);
}

cudaError_t fp16_step(const StepArgs<__half>& a, Fp32Launch L, bool reduce, cudaStream_t s)
{
    return launch_step<__half>(a, L, reduce, s);
}

static int helper_grid(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T>
cudaError_t delta_init(T* g, float* dpsi, const double* rho_init, int nx, int ny, double rho_ref,
                       double rho0, cudaStream_t s)
{
    k_delta_init<T><<<helper_grid((long long)nx * ny), 256, 0, s>>>(g, dpsi, rho_init, nx, ny,
                                                                     rho_ref, rho0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t delta_fields(const T* g, int nx, int ny, double rho_ref, double* rho, double* ux,
                         double* uy, cudaStream_t s)
{
    k_delta_fields<T><<<helper_grid((long long)nx * ny), 256, 0, s>>>(g, nx, ny, rho_ref, rho, ux,
                                                                      uy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t delta_energy(const T* g, const float* dpsi, int nx, int ny, const StepArgs<T>& a,
                         double* out4, double* partials, unsigned int* counter, cudaStream_t s)
{
    StepArgs<T> b = a;
    b.partials = partials;
    b.counter = counter;
    k_delta_energy<T><<<helper_grid((long long)nx * ny), 256, 0, s>>>(g, dpsi, b, out4);
    return cudaGetLastError();
}

cudaError_t rho_check_sum(const double* rho, long long n, double* partials, unsigned int* counter,
                          double* out_sum, int* flag, cudaStream_t s)
{
    k_rho_check_sum<<<helper_grid(n), 256, 0, s>>>(rho, n, partials, counter, out_sum, flag);
    return cudaGetLastError();
}

template cudaError_t delta_init<float>(float*, float*, const double*, int, int, double, double,
                                       cudaStream_t);
template cudaError_t delta_init<__half>(__half*, float*, const double*, int, int, double, double,
                                        cudaStream_t);
template cudaError_t delta_fields<float>(const float*, int, int, double, double*, double*, double*,
                                         cudaStream_t);
template cudaError_t delta_fields<__half>(const __half*, int, int, double, double*, double*,
                                          double*, cudaStream_t);
template cudaError_t delta_energy<float>(const float*, const float*, int, int,
                                         const StepArgs<float>&, double*, double*, unsigned int*,
                                         cudaStream_t);
template cudaError_t delta_energy<__half>(const __half*, const float*, int, int,
                                          const StepArgs<__half>&, double*, double*,
                                          unsigned int*, cudaStream_t);

}  // namespace lbsc

// lb_device.cuh — device helpers shared by the FP32/FP16 step kernels: the
// per-site physics of one lattice Boltzmann step (Chibbaro et al.,
// arXiv:1008.2865) and the deterministic CTA/grid reductions.
#pragma once

#include "lb_internal.h"

namespace lbsc {
namespace dev {

__device__ __forceinline__ float ldg_(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st_(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ float lds_(const float* p) { return *p; }
__device__ __forceinline__ float lds_(const __half* p) { return __half2float(*p); }
// a pair of adjacent populations (lb_internal.h): one 8-byte or 4-byte access
__device__ __forceinline__ void ldg_pair(const float* p, float& a, float& b)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ldg_pair(const __half* p, float& a, float& b)
{
    const float2 v = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void lds_pair(const float* p, float& a, float& b)
{
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void lds_pair(const __half* p, float& a, float& b)
{
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void st_pair(float* p, float a, float b)
{
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st_pair(__half* p, float a, float b)
{
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}

__device__ __forceinline__ int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// Element offsets within a tile of the tiled population layout (lb_internal.h),
// relative to the column offsets tsingle(x) (populations 0, 2, 4) and tpair(x)
// (the pairs (1, 3), (5, 6), (7, 8); A and B are a pair's first and second
// member).
template <typename T>
struct Tile;
template <>
struct Tile<float> {   // paired: a pair is two adjacent elements
    static constexpr bool kPaired = true;
    static constexpr int P0 = 0, P2 = 32, P4 = 64;
    static constexpr int A13 = 96, B13 = 97, A56 = 160, B56 = 161, A78 = 224, B78 = 225;
};
template <>
struct Tile<__half> {  // the same element offsets: a pair is one 4-byte access
    static constexpr bool kPaired = true;
    static constexpr int P0 = 0, P2 = 32, P4 = 64;
    static constexpr int A13 = 96, B13 = 97, A56 = 160, B56 = 161, A78 = 224, B78 = 225;
};
__device__ __forceinline__ int tsingle(int x) { return (x >> 5) * kTileElems + (x & (kTileW - 1)); }
template <typename T>
__device__ __forceinline__ int tpair(int x)
{
    return (x >> 5) * kTileElems + (Tile<T>::kPaired ? 2 : 1) * (x & (kTileW - 1));
}

// A pair (members at p + OA and p + OB) from global memory, shared memory, or
// into global memory: one access in the paired layout, two otherwise.
template <int OA, int OB, typename T>
__device__ __forceinline__ void ld2(const T* __restrict__ p, float& a, float& b)
{
    if (Tile<T>::kPaired) {
        ldg_pair(p + OA, a, b);
    } else {
        a = ldg_(p + OA);
        b = ldg_(p + OB);
    }
}
template <int OA, int OB, typename T>
__device__ __forceinline__ void lds2(const T* p, float& a, float& b)
{
    if (Tile<T>::kPaired) {
        lds_pair(p + OA, a, b);
    } else {
        a = lds_(p + OA);
        b = lds_(p + OB);
    }
}
template <int OA, int OB, typename T>
__device__ __forceinline__ void st2(T* p, float a, float b)
{
    if (Tile<T>::kPaired) {
        st_pair(p + OA, a, b);
    } else {
        st_(p + OA, a);
        st_(p + OB, b);
    }
}

// The 9 populations of one site from a row pointer and the column's offsets
// cs = tsingle(x), cp = tpair<T>(x).
template <typename T>
__device__ __forceinline__ void load_site(float f[9], const T* __restrict__ row, int cs, int cp)
{
    using L = Tile<T>;
    f[0] = ldg_(row + cs + L::P0);
    f[2] = ldg_(row + cs + L::P2);
    f[4] = ldg_(row + cs + L::P4);
    ld2<L::A13, L::B13>(row + cp, f[1], f[3]);
    ld2<L::A56, L::B56>(row + cp, f[5], f[6]);
    ld2<L::A78, L::B78>(row + cp, f[7], f[8]);
}

// The 9 populations of site (x, y) of a tiled buffer with `pitch` elements per row.
template <typename T>
__device__ __forceinline__ void load_site_xy(float f[9], const T* __restrict__ g, int pitch, int x,
                                             int y)
{
    load_site(f, g + (size_t)y * pitch, tsingle(x), tpair<T>(x));
}

// Two-belt force sums of Eq. FORCE in pair form. r[k] points at the stencil
// centre's column in the dpsi row y + k - 2 (k = 0..4), so r[k][dx] is
// dpsi(x + dx, y + k - 2). Returns S = sum_c K_c c dpsi(x + c), grouped by
// |c|^2; the constant psi_ref cancels inside every pair (c, -c).
template <typename T>
__device__ __forceinline__ void force_sums(const float* const r[5], const StepArgs<T>& a,
                                           float& Sx, float& Sy)
{
    const float *rM2 = r[0], *rM1 = r[1], *rC = r[2], *rP1 = r[3], *rP2 = r[4];
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

// force_sums and, with E (a reduction step), also the Sec. 5 energies from the
// same neighbour values. Only lattice totals of the energies are wanted, and on
// the periodic lattice sum_x psi(x) psi(x + c) = sum_x psi(x) psi(x - c)
// (translate x by c), so each class sum takes one member of every pair
// (c, -c), doubled: the totals equal those of energy_site's full class sums,
// the per-site terms do not. The energies are weighted by `on` (1 for an
// output site, 0 otherwise) instead of a branch.
template <bool E, typename T>
__device__ __forceinline__ void force_energy(const float* const r[5], const StepArgs<T>& a,
                                             float& Sx, float& Sy, float on, float pc, float& es,
                                             float& em, float& eb)
{
    const float *rM2 = r[0], *rM1 = r[1], *rC = r[2], *rP1 = r[3], *rP2 = r[4];
    const float xp1 = rC[1], xm1 = rC[-1], yp1 = rP1[0], ym1 = rM1[0];        // |c|^2 = 1
    const float pp = rP1[1], mm = rM1[-1], pm = rM1[1], mp = rP1[-1];         // |c|^2 = 2
    const float xp2 = rC[2], xm2 = rC[-2], yp2 = rP2[0], ym2 = rM2[0];        // |c|^2 = 4
    const float a21 = rP1[2], am2m1 = rM1[-2], b12 = rP2[1], bm1m2 = rM2[-1]; // |c|^2 = 5
    const float cm12 = rP2[-1], c1m2 = rM2[1], dm21 = rP1[-2], d2m1 = rM1[2];
    const float e22 = rP2[2], em2m2 = rM2[-2], f2m2 = rM2[2], fm22 = rP2[-2]; // |c|^2 = 8
    const float d10 = xp1 - xm1, d01 = yp1 - ym1;
    const float d11 = pp - mm, d1m = pm - mp;
    const float d20 = xp2 - xm2, d02 = yp2 - ym2;
    const float da = a21 - am2m1, db = b12 - bm1m2, dc = cm12 - c1m2, dd = dm21 - d2m1;
    const float e1 = e22 - em2m2, e2 = f2m2 - fm22;
    Sx = a.K1 * d10 + a.K2 * (d11 + d1m) + 2.f * a.K4 * d20 +
         a.K5 * (2.f * (da - dd) + (db - dc)) + 2.f * a.K8 * (e1 + e2);
    Sy = a.K1 * d01 + a.K2 * (d11 - d1m) + 2.f * a.K4 * d02 +
         a.K5 * ((da + dd) + 2.f * (db + dc)) + 2.f * a.K8 * (e1 - e2);
    if (E) {
        const float pr = a.psi_ref;
        const float H1 = xp1 + yp1;                        // (1,0), (0,1)
        const float H2 = pp + pm;                          // (1,1), (1,-1)
        const float H4 = xp2 + yp2;                        // (2,0), (0,2)
        const float H5 = (a21 + b12) + (cm12 + dm21);      // (2,1), (1,2), (-1,2), (-2,1)
        const float H8 = e22 + f2m2;                       // (2,2), (2,-2)
        const float b1 = a.K0 * pc + a.K1 * fmaf(2.f, H1, 4.f * pr) + a.K2 * fmaf(2.f, H2, 4.f * pr);
        const float b2 = a.K4 * fmaf(2.f, H4, 4.f * pr) + a.K5 * fmaf(2.f, H5, 8.f * pr) +
                         a.K8 * fmaf(2.f, H8, 4.f * pr);
        const float hp = 0.5f * on * pc;
        es = fmaf(hp, b1, es);
        em = fmaf(hp, b2, em);
        eb = fmaf(a.half_A1 * on * pc, pc, eb);
    }
}

// Sec. 5 pseudo-energy densities of one site with psi = psi_ref + dpsi:
// belt 1 with the rest coupling K0, belt 2, and the bulk term A1/2 psi^2.
template <typename T>
__device__ __forceinline__ void energy_site(const float* const r[5], float pc,
                                            const StepArgs<T>& a, float& es, float& em,
                                            float& eb)
{
    const float *rM2 = r[0], *rM1 = r[1], *rC = r[2], *rP1 = r[3], *rP2 = r[4];
    const float pr = a.psi_ref;
    const float S1 = (rC[1] + rC[-1]) + (rP1[0] + rM1[0]);
    const float S2 = (rP1[1] + rP1[-1]) + (rM1[1] + rM1[-1]);
    const float S4 = (rC[2] + rC[-2]) + (rP2[0] + rM2[0]);
    const float S5 = ((rP1[2] + rP1[-2]) + (rM1[2] + rM1[-2])) +
                     ((rP2[1] + rP2[-1]) + (rM2[1] + rM2[-1]));
    const float S8 = (rP2[2] + rP2[-2]) + (rM2[2] + rM2[-2]);
    const float b1 = a.K0 * pc + a.K1 * fmaf(4.f, pr, S1) + a.K2 * fmaf(4.f, pr, S2);
    const float b2 = a.K4 * fmaf(4.f, pr, S4) + a.K5 * fmaf(8.f, pr, S5) + a.K8 * fmaf(4.f, pr, S8);
    es = fmaf(0.5f * pc, b1, es);
    em = fmaf(0.5f * pc, b2, em);
    eb = fmaf(a.half_A1 * pc, pc, eb);
}

// Moments (Eqs. 2-3) and BGK relaxation (Eq. 1) of the deviations
// f_i - w_i rho_ref towards the Eq. 4 equilibrium at u + F/(omega rho),
// written as deviations again:
//   g*_i = (1 - omega) g_i + omega w_i d + omega w_i rho (3 c.u + 9/2 (c.u)^2 - 3/2 u^2)
// with d = rho - rho_ref. OM1 drops the (1 - omega) g_i terms (omega = 1,
// the paper's tau = 1). Returns d.
template <bool OM1, typename T>
__device__ __forceinline__ float collide(const float f[9], float Fx, float Fy,
                                         const StepArgs<T>& a, float gs[9])
{
    const float d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const float rho = a.rho_ref + d;
    const float inv = __frcp_rn(rho);
    const float ux = fmaf(Fx, a.inv_omega, jx) * inv;
    const float uy = fmaf(Fy, a.inv_omega, jy) * inv;
    const float usq15 = 1.5f * fmaf(ux, ux, uy * uy);
    const float orho = OM1 ? rho : a.omega * rho;
    const float od = OM1 ? d : a.omega * d;
    const float A0 = orho * a.w0, A1 = orho * a.w1, A2 = orho * a.w2;
    const float D0 = od * a.w0, D1 = od * a.w1, D2 = od * a.w2;
    float e[9];
    e[0] = fmaf(A0, -usq15, D0);
    {
        const float s = fmaf(4.5f * ux, ux, -usq15), t3 = 3.f * ux;
        e[1] = fmaf(A1, s + t3, D1);
        e[3] = fmaf(A1, s - t3, D1);
    }
    {
        const float s = fmaf(4.5f * uy, uy, -usq15), t3 = 3.f * uy;
        e[2] = fmaf(A1, s + t3, D1);
        e[4] = fmaf(A1, s - t3, D1);
    }
    {
        const float c = ux + uy;
        const float s = fmaf(4.5f * c, c, -usq15), t3 = 3.f * c;
        e[5] = fmaf(A2, s + t3, D2);
        e[7] = fmaf(A2, s - t3, D2);
    }
    {
        const float c = uy - ux;
        const float s = fmaf(4.5f * c, c, -usq15), t3 = 3.f * c;
        e[6] = fmaf(A2, s + t3, D2);
        e[8] = fmaf(A2, s - t3, D2);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) gs[i] = OM1 ? e[i] : fmaf(a.omc, f[i], e[i]);
    return d;
}

// psi(rho) - psi_ref = -sqrt(rho0) e^{-rho_ref/rho0} expm1(-(rho - rho_ref)/rho0)
template <typename T>
__device__ __forceinline__ float dpsi_of(float d, const StepArgs<T>& a)
{
    return a.cpsi * expm1f(-d * a.inv_rho0);
}

// Deterministic sum of 4 doubles over a CTA of NT threads (NT a multiple of
// 32, at most 1024); the result is valid in thread 0. The threads' values meet
// in shared memory and warp 0 alone does the FP64 adds (fixed strided order,
// then a fixed shuffle tree): FP64 issues slowly on this part, so the adds of
// one warp instead of every warp's shuffle tree.
// `red` is 4 NT doubles of shared memory (k-major); each thread writes only its
// own slots before the first barrier, so a buffer whose slot (k, tid) the
// thread itself last used may serve.
template <int NT>
__device__ void block_sum4(double v[4], double* red)
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k * NT + tid] = v[k];
    __syncthreads();
    if (tid < 32) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double w = red[k * NT + tid];
#pragma unroll
            for (int j = tid + 32; j < NT; j += 32) w += red[k * NT + j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
            v[k] = w;
        }
    }
    __syncthreads();
}
template <int NT>
__device__ void block_sum4(double v[4])
{
    __shared__ double red[4 * NT];
    block_sum4<NT>(v, red);
}

// Sum of n 4-double partials p[0..n) over a CTA of NT threads: thread k adds
// partials k, k + NT, k + 2 NT, ... in that order, then block_sum4's tree; the
// total is valid in thread 0. The loads of U partials are issued together
// (one L2 round trip instead of U); U does not change the order of the adds.
template <int NT, int U = 4>
__device__ void sum_partials(const double* partials, unsigned int nblocks, double w[4],
                             double* red)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = 0.0;
    unsigned int j = threadIdx.x;
    for (; j + (U - 1) * NT < nblocks; j += U * NT) {
        double2 q[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const double2* p2 = reinterpret_cast<const double2*>(partials + 4 * (size_t)(j + u * NT));
            q[u][0] = __ldcg(p2);
            q[u][1] = __ldcg(p2 + 1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            w[0] += q[u][0].x;
            w[1] += q[u][0].y;
            w[2] += q[u][1].x;
            w[3] += q[u][1].y;
        }
    }
    for (; j < nblocks; j += NT) {
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] += __ldcg(partials + 4 * (size_t)j + k);
    }
    block_sum4<NT>(w, red);
}

// Store this CTA's partial, and if it is the last CTA to arrive, sum all
// partials (sum_partials) and return true in thread 0 with the total in v.
// Resets the counter for the next use. `red`: the block sums' shared buffer
// (4 NT doubles, as block_sum4).
template <int NT>
__device__ bool last_block_total(double v[4], double* partials, unsigned int* counter,
                                 unsigned int nblocks, double* red)
{
    __shared__ bool s_last;
    const unsigned int b = blockIdx.y * gridDim.x + blockIdx.x;
    block_sum4<NT>(v, red);
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
    double w[4];
    sum_partials<NT>(partials, nblocks, w, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = w[k];
        *counter = 0u;
    }
    return threadIdx.x == 0;
}
template <int NT>
__device__ bool last_block_total(double v[4], double* partials, unsigned int* counter,
                                 unsigned int nblocks)
{
    __shared__ double red[4 * NT];
    return last_block_total<NT>(v, partials, counter, nblocks, red);
}

// Grid sum of a reduction step in two levels, so that the FP64 adds (a slow
// pipe on this part) spread over many SMs instead of the one last CTA: CTA row
// y of the step's grid left its nbx partials at cta[y nbx .. y nbx + nbx); one
// CTA per row sums them (sum_partials) into rows[y], and the last row of the
// lattice to finish (arrival counter, reset here) sums rows[0 .. nby) the same
// way. Returns true in thread 0 of that CTA, with the total in w.
template <int NT>
__device__ bool row_then_total(const double* cta, int nbx, int nby, int y, double* rows,
                               unsigned int* counter, double w[4], double* red)
{
    __shared__ bool s_last;
    sum_partials<NT, 1>(cta + 4 * (size_t)y * nbx, nbx, w, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) rows[4 * (size_t)y + k] = w[k];
        __threadfence();
        s_last = atomicAdd(counter, 1u) == (unsigned int)nby - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    sum_partials<NT, 1>(rows, nby, w, red);
    if (threadIdx.x == 0) *counter = 0u;
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

}  // namespace dev
}  // namespace lbsc

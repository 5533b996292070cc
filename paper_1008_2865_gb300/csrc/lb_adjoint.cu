// lb_adjoint.cu — lb_adjoint: the gradient of
//   J = E_s(T) + E_m(T) + sum_x (rho(x, T) - rho*(x))^2
// (Sec. 5 pseudo-energy of the final state plus a squared misfit to a target
// density) with respect to the initial density field and the couplings G1, G2
// of Eq. FORCE, for an FP32 state, by a hand-written reverse sweep of the
// fused step with sqrt(T) checkpointing.
//
// Forward (Eqs. 1-4, Eq. FORCE):  rho, j = moments of f;  psi(rho);
//   F = -psi(x) S(x), S = sum_c K_c c psi(x+c);  v = (j + F/omega)/rho;
//   f*_i = (1-omega) f_i + omega feq_i(rho, v);  f_i(x + c_i, t+1) = f*_i(x).
// Reverse, with l' = dJ/df(t+1) and l* the streamed-back adjoint
// l*_i(x) = l'_i(x + c_i):
//   pass A (per site x):
//     rho-bar = omega sum_i l*_i feq_i / rho - (v-bar . v) / rho
//     v-bar   = omega rho sum_i l*_i w_i (3 c_i + 9 (c_i.v) c_i - 3 v)
//     j-bar   = v-bar / rho,  F-bar = v-bar / (omega rho)
//     psi-bar(x) gets -F-bar . S (the leading psi(x) of F(x)); Q = psi F-bar
//     dJ/dG1 += -psi F-bar . S_w,  dJ/dG2 += -psi F-bar . S_p  (S = G1 S_w + G2 S_p)
//   pass B (per site y): psi-bar(y) += sum_c K_c c . Q(y + c) (the transpose of the
//     force stencil; K_c = K_{-c}); rho-bar += psi'(rho) psi-bar;
//     l_i(y) = (1 - omega) l*_i(y) + rho-bar(y) + c_i . j-bar(y).
// Terminal: l_i(y, T) = psi'(rho) sum_{c incl. rest} K_c psi(y+c) + 2 (rho - rho*).
// Start: dJ/drho_init(x) = sum_i w_i l_i(x, 0).
// The state and the adjoint are FP32; J and the G1, G2 gradients accumulate
// in FP64 (per-thread, then deterministic CTA and grid sums).
#include <cmath>
#include <new>
#include <vector>

#include "lb_device.cuh"

using namespace lbsc;
using namespace lbsc::dev;

namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjMaxBlocks = 152 * (2048 / kAdjThreads);   // one full wave of threads

// Periodic neighbourhood of site (x, y), computed once per site (nx, ny >= 5):
// columns x-2 .. x+2 and row offsets (y-2 .. y+2) * nx.
struct Nbr5 {
    int xo[5];
    int yo[5];
};

__device__ __forceinline__ Nbr5 nbr5(int x, int y, int nx, int ny)
{
    Nbr5 n;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        int xx = x + k - 2, yy = y + k - 2;
        xx += xx < 0 ? nx : 0;
        xx -= xx >= nx ? nx : 0;
        yy += yy < 0 ? ny : 0;
        yy -= yy >= ny ? ny : 0;
        n.xo[k] = xx;
        n.yo[k] = yy * nx;
    }
    return n;
}

// The 5 x 5 neighbourhood of a periodic FP32 field: v[k][m] = field(x + m - 2, y + k - 2).
// For a column away from the periodic x edges (2 <= x < nx - 2, `xin`) each row is
// one pointer with immediate offsets; otherwise every column offset is wrapped.
__device__ __forceinline__ void gather5(const float* __restrict__ fld, const Nbr5& nb, int x,
                                        bool xin, float v[5][5])
{
    if (xin) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float* r = fld + nb.yo[k] + x;
#pragma unroll
            for (int m = 0; m < 5; ++m) v[k][m] = __ldg(r + (m - 2));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
#pragma unroll
            for (int m = 0; m < 5; ++m) v[k][m] = __ldg(fld + nb.yo[k] + nb.xo[m]);
        }
    }
}

// The same for the (Qx, Qy) pairs of pass B: one 8-byte load per stencil site.
__device__ __forceinline__ void gather5x2(const float2* __restrict__ fld, const Nbr5& nb, int x,
                                          bool xin, float vx[5][5], float vy[5][5])
{
    if (xin) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float2* r = fld + nb.yo[k] + x;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const float2 q = __ldg(r + (m - 2));
                vx[k][m] = q.x;
                vy[k][m] = q.y;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const float2 q = __ldg(fld + nb.yo[k] + nb.xo[m]);
                vx[k][m] = q.x;
                vy[k][m] = q.y;
            }
        }
    }
}

// D2Q9 speeds in the order of the populations (compile-time in unrolled loops).
__host__ __device__ constexpr int cx_of(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int cy_of(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}

// Deviations f_i(x, y) - w_i rho_ref of state t, read from the tiled populations.
template <typename T>
__device__ __forceinline__ void site_f(const T* __restrict__ g, int pitch, int x, int y,
                                       float f[9])
{
    load_site_xy(f, g, pitch, x, y);
}

struct AdjArgs {
    StepArgs<float> a;        // couplings, weights, rho_ref, psi_ref, omega of the state
    StepArgs<float> aw;       // couplings replaced by the D2Q9 weights (S_w)
    StepArgs<float> ap;       // couplings replaced by the E(8) weights (S_p)
    float G1, G2;
    float inv_sqrt_rho0;      // 1 / sqrt(rho0): psi'(rho) = exp(-rho/rho0) / sqrt(rho0)
    const float* g;           // tiled f(t) - w rho_ref
    const float* dpsi;        // dpsi(t)
    const float* lam_next;    // [9][N] dJ/df(t+1)
    float* lam;               // [9][N] dJ/df(t)
    float4* site;             // per site (j-bar x, j-bar y, rho-bar so far, psi'(rho))
    float2* Q;                // per site psi F-bar (x, y), read by pass B as a stencil
    const double* rho_target; // terminal kernel
    double* partials;
    unsigned int* counter;
    double* acc;              // [4] FP64 accumulators
};

// s += x with Kahan's compensation c (the rounding error of the previous adds).
// The operations must not be reassociated: nvcc does not, and fmaf is not used.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

template <int NT>
__device__ void accumulate_grid(double v[4], const AdjArgs& A)
{
    if (last_block_total<NT>(v, A.partials, A.counter, gridDim.x)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) A.acc[k] += v[k];
    }
}

// Grid sum of two per-thread values added into A.acc[0..1] with little FP64
// work (FP64 issues slowly on this part) and no long dependent chains: the
// CTA's values meet in shared memory, each lane of warp 0 adds NT/32 of them in
// FP32 in a fixed order, the 32 lane sums go to FP64 and a fixed shuffle tree
// adds them; the last CTA to finish sums the CTA partials in FP64 in CTA order
// (loads issued four at a time). Error: each FP32 lane sum adds at most NT/32
// per-thread values, so its relative error is below (NT/32) 2^-24 of the sum of
// their magnitudes; everything above it is FP64.
template <int NT>
__device__ void accumulate_grid2(float v0, float v1, const AdjArgs& A)
{
    __shared__ float sh[2][NT];
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    sh[0][tid] = v0;
    sh[1][tid] = v1;
    __syncthreads();
    if (tid < 32) {
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int k = tid; k < NT; k += 32) {
            a0 += sh[0][k];
            a1 += sh[1][k];
        }
        double w0 = a0, w1 = a1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w0 += __shfl_down_sync(0xffffffffu, w0, o);
            w1 += __shfl_down_sync(0xffffffffu, w1, o);
        }
        if (tid == 0) {
            reinterpret_cast<double2*>(A.partials)[blockIdx.x] = make_double2(w0, w1);
            __threadfence();
            s_last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double w0 = 0.0, w1 = 0.0;
    const double2* p2 = reinterpret_cast<const double2*>(A.partials);
    unsigned int j = tid;
    for (; j + 3 * NT < gridDim.x; j += 4 * NT) {
        double2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldcg(p2 + j + u * NT);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            w0 += q[u].x;
            w1 += q[u].y;
        }
    }
    for (; j < gridDim.x; j += NT) {
        const double2 q = __ldcg(p2 + j);
        w0 += q.x;
        w1 += q.y;
    }
    double v[4] = {w0, w1, 0.0, 0.0};
    block_sum4<NT>(v);
    if (tid == 0) {
        A.acc[0] += v[0];
        A.acc[1] += v[1];
        *A.counter = 0u;
    }
}

// J of the state (A.g / gT, A.dpsi) and the terminal adjoint l(T) (skipped when
// A.lam is null: lb_objective). T is the population storage type.
template <typename T>
__global__ void __launch_bounds__(kAdjThreads) k_adj_terminal(const AdjArgs A,
                                                              const T* __restrict__ gT)
{
    const StepArgs<float>& a = A.a;
    const int nx = a.nx, ny = a.ny, N = (int)a.N;
    double v[4] = {0.0, 0.0, 0.0, 0.0};   // E, misfit, dE/dG1, dE/dG2
    for (int s = blockIdx.x * kAdjThreads + threadIdx.x; s < N; s += gridDim.x * kAdjThreads) {
        const int y = s / nx, x = s % nx;
        float f[9];
        site_f(gT, a.pitch, x, y, f);
        const float d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        const float rho = a.rho_ref + d;
        const Nbr5 nb = nbr5(x, y, nx, ny);
        const bool xin = x >= 2 && x < nx - 2;
        float p[5][5];
        gather5(A.dpsi, nb, x, xin, p);
        const float pr = a.psi_ref;
        const float pc = pr + p[2][2];
        // class sums of psi (not deviations) around the site
        const float S1 = fmaf(4.f, pr, (p[2][3] + p[2][1]) + (p[3][2] + p[1][2]));
        const float S2 = fmaf(4.f, pr, (p[3][3] + p[3][1]) + (p[1][3] + p[1][1]));
        const float S4 = fmaf(4.f, pr, (p[2][4] + p[2][0]) + (p[4][2] + p[0][2]));
        const float S5 = fmaf(8.f, pr, ((p[3][4] + p[3][0]) + (p[1][4] + p[1][0])) +
                                           ((p[4][3] + p[4][1]) + (p[0][3] + p[0][1])));
        const float S8 = fmaf(4.f, pr, (p[4][4] + p[4][0]) + (p[0][4] + p[0][0]));
        const float dEdpsi = a.K0 * pc + a.K1 * S1 + a.K2 * S2 + a.K4 * S4 + a.K5 * S5 + a.K8 * S8;
        const float sw = A.aw.K0 * pc + A.aw.K1 * S1 + A.aw.K2 * S2;
        const float sp = A.ap.K0 * pc + A.ap.K1 * S1 + A.ap.K2 * S2 + A.ap.K4 * S4 +
                         A.ap.K5 * S5 + A.ap.K8 * S8;
        const float dpr = __expf(-rho * a.inv_rho0) * A.inv_sqrt_rho0;
        const double mis = (double)rho - A.rho_target[s];
        if (A.lam) {
            const float lam = dpr * dEdpsi + (float)(2.0 * mis);
#pragma unroll
            for (int i = 0; i < 9; ++i) A.lam[i * N + s] = lam;
        }
        v[0] += 0.5 * (double)pc * dEdpsi;
        v[1] += mis * mis;
        v[2] += 0.5 * (double)pc * sw;
        v[3] += 0.5 * (double)pc * sp;
    }
    accumulate_grid<kAdjThreads>(v, A);
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_pass_a(const AdjArgs A)
{
    const StepArgs<float>& a = A.a;
    const int nx = a.nx, ny = a.ny, N = (int)a.N;
    const float om = a.omega;
    const float w[9] = {a.w0, a.w1, a.w1, a.w1, a.w1, a.w2, a.w2, a.w2, a.w2};
    // dJ/dG1, dJ/dG2: per thread a compensated FP32 sum (Kahan: the running sum
    // stays within about one FP32 rounding of the exact sum of its terms, however
    // many sites the thread visits), then accumulate_grid2
    float f1 = 0.f, f2 = 0.f, c1 = 0.f, c2 = 0.f;
    for (int s = blockIdx.x * kAdjThreads + threadIdx.x; s < N; s += gridDim.x * kAdjThreads) {
        const int y = s / nx, x = s % nx;
        float f[9];
        site_f(A.g, a.pitch, x, y, f);
        const float d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
        const float rho = a.rho_ref + d;
        const Nbr5 nb = nbr5(x, y, nx, ny);
        const bool xin = x >= 2 && x < nx - 2;
        float p[5][5];
        gather5(A.dpsi, nb, x, xin, p);
        const float* rows[5] = {&p[0][2], &p[1][2], &p[2][2], &p[3][2], &p[4][2]};
        float Swx, Swy, Spx, Spy;
        force_sums(rows, A.aw, Swx, Swy);
        force_sums(rows, A.ap, Spx, Spy);
        const float Sx = A.G1 * Swx + A.G2 * Spx, Sy = A.G1 * Swy + A.G2 * Spy;
        const float pc = a.psi_ref + p[2][2];
        const float Fx = -pc * Sx, Fy = -pc * Sy;
        const float inv = __frcp_rn(rho);
        const float vx = fmaf(Fx, a.inv_omega, jx) * inv, vy = fmaf(Fy, a.inv_omega, jy) * inv;
        const float usq = vx * vx + vy * vy;
        // rho-bar gets omega sum_i l*_i feq_i / rho = omega sum_i l*_i w_i (1 + 3 c.v + ...);
        // v-bar = omega rho sum_i l*_i w_i (3 c_i + 9 (c_i.v) c_i - 3 v)
        float rb = 0.f, vbx = 0.f, vby = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ci = cx_of(i), cj = cy_of(i);
            // l*_i(x) = l'_i(x + c_i): the adjoint streamed back
            const float lw = w[i] * __ldg(A.lam_next + i * N + nb.yo[2 + cj] + nb.xo[2 + ci]);
            const float cu = ci * vx + cj * vy;
            rb += lw * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * usq);
            const float t9 = 9.f * cu;
            vbx += lw * (3.f * ci + t9 * ci - 3.f * vx);
            vby += lw * (3.f * cj + t9 * cj - 3.f * vy);
        }
        rb *= om;
        vbx *= om * rho;
        vby *= om * rho;
        const float Fbx = vbx * inv * a.inv_omega, Fby = vby * inv * a.inv_omega;
        rb -= (vbx * vx + vby * vy) * inv;
        const float dpr = __expf(-rho * a.inv_rho0) * A.inv_sqrt_rho0;
        A.site[s] = make_float4(vbx * inv, vby * inv, rb + dpr * (-(Fbx * Sx + Fby * Sy)), dpr);
        A.Q[s] = make_float2(pc * Fbx, pc * Fby);
        kahan_add(f1, c1, -pc * (Fbx * Swx + Fby * Swy));
        kahan_add(f2, c2, -pc * (Fbx * Spx + Fby * Spy));
    }
    accumulate_grid2<kAdjThreads>(f1, f2, A);
}

__global__ void __launch_bounds__(kAdjThreads) k_adj_pass_b(const AdjArgs A)
{
    const StepArgs<float>& a = A.a;
    const int nx = a.nx, ny = a.ny, N = (int)a.N;
    const float omc = a.omc;
    for (int s = blockIdx.x * kAdjThreads + threadIdx.x; s < N; s += gridDim.x * kAdjThreads) {
        const int y = s / nx, x = s % nx;
        // sum_c K_c c . Q(y + c): the x part is the force stencil of Qx, the y part of
        // Qy (one 8-byte load per stencil site for both)
        const Nbr5 nb = nbr5(x, y, nx, ny);
        const bool xin = x >= 2 && x < nx - 2;
        float qx[5][5], qy[5][5];
        gather5x2(A.Q, nb, x, xin, qx, qy);
        const float* rx[5] = {&qx[0][2], &qx[1][2], &qx[2][2], &qx[3][2], &qx[4][2]};
        const float* ry[5] = {&qy[0][2], &qy[1][2], &qy[2][2], &qy[3][2], &qy[4][2]};
        float sx, sy, tx, ty;
        force_sums(rx, a, sx, sy);
        force_sums(ry, a, tx, ty);
        const float4 sv = __ldg(A.site + s);
        const float rb = sv.z + sv.w * (sx + ty);
        const float jbx = sv.x, jby = sv.y;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ci = cx_of(i), cj = cy_of(i);
            const float ls = __ldg(A.lam_next + i * N + nb.yo[2 + cj] + nb.xo[2 + ci]);
            A.lam[i * N + s] = fmaf(omc, ls, rb + ci * jbx + cj * jby);
        }
    }
}

__global__ void k_adj_grad_init(const float* __restrict__ lam, int N, float w0, float w1, float w2,
                                double* __restrict__ out)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const double g = (double)w0 * lam[s] +
                         (double)w1 * (((double)lam[N + s] + lam[2 * N + s]) +
                                       ((double)lam[3 * N + s] + lam[4 * N + s])) +
                         (double)w2 * (((double)lam[5 * N + s] + lam[6 * N + s]) +
                                       ((double)lam[7 * N + s] + lam[8 * N + s]));
        out[s] = g;
    }
}

int adj_grid(long long n)
{
    long long b = (n + kAdjThreads - 1) / kAdjThreads;
    if (b > kAdjMaxBlocks) b = kAdjMaxBlocks;
    return (int)(b < 1 ? 1 : b);
}

bool dev_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

StepArgs<float> with_weights(StepArgs<float> a, bool e8)
{
    // the same stencil code with unit couplings: the D2Q9 weights (belt 1 and
    // rest) or the E(8) weights (both belts and rest, Table 1, Eq. weights_1)
    if (!e8) {
        a.K0 = 4.f / 9.f; a.K1 = 1.f / 9.f; a.K2 = 1.f / 36.f; a.K4 = 0.f; a.K5 = 0.f; a.K8 = 0.f;
    } else {
        a.K0 = (float)(247.0 / 420.0); a.K1 = 4.f / 63.f; a.K2 = 4.f / 135.f;
        a.K4 = 1.f / 180.f; a.K5 = 2.f / 945.f; a.K8 = 1.f / 15120.f;
    }
    return a;
}

}  // namespace

extern "C" lb_status lb_adjoint(lb_state* s, long steps, const double* rho_target,
                                int checkpoint_every, double* J_out, double* grad_rho,
                                double* grad_G)
{
    NvtxRange nvtx_range("lb_adjoint");
    if (!s || steps < 0 || !rho_target || !J_out || !grad_rho || !grad_G || checkpoint_every < 0)
        return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    if (s->p.prec != LB_FP32 || s->t != 0) return LB_ERR_STATE;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return LB_ERR_CUDA;
    const int N = (int)s->N;
    const long long T = steps;
    long long C = checkpoint_every > 0 ? checkpoint_every : (long long)std::ceil(std::sqrt((double)T));
    if (C < 1) C = 1;
    const long long K = T > 0 ? (T + C - 1) / C : 0;     // checkpoints at t = 0, C, 2C, ...
    const size_t GE = (size_t)g_elems(s->p.nx, s->p.ny);
    const size_t slot = GE + (size_t)N;                   // populations (GE) then dpsi (N), floats
    cudaStream_t st = s->stream;

    // ---- working memory of one call (freed on return): checkpoints, two segment
    // buffers (states 1 .. C-1 of a segment; state 0 is its checkpoint), the
    // adjoint ping-pong, per-site scratch, and a second stream with its events
    float *ck = nullptr, *seg = nullptr, *lam = nullptr, *scr = nullptr;
    double *tgt = nullptr, *acc = nullptr, *part = nullptr, *grad_dev = nullptr;
    unsigned int* cnt = nullptr;
    cudaStream_t rs = nullptr;                       // recomputation stream
    cudaEvent_t ev_fwd = nullptr, ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    auto release = [&]() {
        void* ptrs[] = {ck, seg, lam, scr, tgt, acc, part, grad_dev, cnt};
        for (void* q : ptrs)
            if (q) cudaFree(q);
        cudaEvent_t evs[] = {ev_fwd, ev_ready[0], ev_ready[1], ev_free[0], ev_free[1]};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        if (rs) cudaStreamDestroy(rs);
        cudaGetLastError();
    };
    const size_t seg_slots = (size_t)(C > 1 ? C - 1 : 1);
    const bool grad_on_dev = dev_ptr(grad_rho);
    bool ok = cudaMalloc((void**)&ck, sizeof(float) * slot * (size_t)(K > 0 ? K : 1)) == cudaSuccess &&
              cudaMalloc((void**)&seg, sizeof(float) * slot * 2 * seg_slots) == cudaSuccess &&
              cudaMalloc((void**)&lam, sizeof(float) * 18 * (size_t)N) == cudaSuccess &&
              cudaMalloc((void**)&scr, sizeof(float) * 6 * (size_t)N) == cudaSuccess &&
              cudaMalloc((void**)&tgt, sizeof(double) * N) == cudaSuccess &&
              cudaMalloc((void**)&acc, sizeof(double) * 8) == cudaSuccess &&
              cudaMalloc((void**)&part, sizeof(double) * 4 * kAdjMaxBlocks) == cudaSuccess &&
              cudaMalloc((void**)&cnt, sizeof(unsigned int)) == cudaSuccess &&
              (grad_on_dev || cudaMalloc((void**)&grad_dev, sizeof(double) * N) == cudaSuccess);
    if (!ok) {
        release();
        return LB_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_fwd, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_ready[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_ready[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_free[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_free[1], cudaEventDisableTiming) != cudaSuccess) {
        release();
        return LB_ERR_CUDA;
    }
    auto fail = [&]() {
        release();
        s->poisoned = true;
        return LB_ERR_CUDA;
    };
    if (cudaMemcpyAsync(tgt, rho_target, sizeof(double) * N, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemsetAsync(acc, 0, sizeof(double) * 8, st) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st) != cudaSuccess)
        return fail();

    auto save = [&](float* dst, int cur) -> bool {
        return cudaMemcpyAsync(dst, s->g[cur], sizeof(float) * GE, cudaMemcpyDeviceToDevice,
                               st) == cudaSuccess &&
               cudaMemcpyAsync(dst + GE, s->dpsi[cur], sizeof(float) * N,
                               cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    };
    // ---- forward, checkpointing the state (g(t), dpsi(t)) at t = kC. The
    // register-prefetch kernel is used here and in the recomputation below, so
    // the recomputed states are bit-identical to the checkpointed trajectory.
    Fp32Launch L = s->launch;
    L.pipeline = 0;
    for (long long t = 0; t < T; ++t) {
        if (t % C == 0 && !save(ck + slot * (t / C), s->cur)) return fail();
        const bool reduce = s->p.trace_every > 0 && (s->t % s->p.trace_every) == 0;
        if (fp32_step(state_args<float>(s, s->cur), L, reduce, st) != cudaSuccess) return fail();
        s->cur ^= 1;
        s->t += 1;
    }

    AdjArgs A{};
    A.a = state_args<float>(s, s->cur);
    A.aw = with_weights(A.a, false);
    A.ap = with_weights(A.a, true);
    A.G1 = (float)s->p.G1;
    A.G2 = (float)s->p.G2;
    A.inv_sqrt_rho0 = (float)(1.0 / std::sqrt(s->p.rho0));
    A.rho_target = tgt;
    A.partials = part;
    A.counter = cnt;
    // the float4 array first, at the allocation's (256-byte aligned) start, then
    // the float2 array at 16 N bytes (8-byte aligned for any N)
    A.site = reinterpret_cast<float4*>(scr);
    A.Q = reinterpret_cast<float2*>(scr + 4 * (size_t)N);
    float* lamA = lam;
    float* lamB = lam + 9 * (size_t)N;
    const int grid = adj_grid(N);

    // ---- terminal: J and l(T)
    A.g = static_cast<const float*>(s->g[s->cur]);
    A.dpsi = s->dpsi[s->cur];
    A.lam = lamA;
    A.acc = acc;             // acc[0..3] = E, misfit, dE/dG1, dE/dG2
    k_adj_terminal<float><<<grid, kAdjThreads, 0, st>>>(A, A.g);
    if (cudaGetLastError() != cudaSuccess) return fail();

    // ---- reverse over the segments. Segment k (states kC .. kC + n - 1) is
    // recomputed from its checkpoint into segment buffer k & 1 on the second
    // stream while the reverse sweep of segment k + 1 runs on the caller's
    // stream (both are latency-bound on lattices that fit in L2, so the two
    // overlap); events order the buffer reuse and the hand-over.
    A.acc = acc + 4;         // acc[4], acc[5] = the steps' dJ/dG1, dJ/dG2
    const StepArgs<float> base = state_args<float>(s, 0);
    auto seg_len = [&](long long k) { return (k + 1) * C <= T ? C : T - k * C; };
    auto state_at = [&](long long k, long long j) -> float* {
        return j == 0 ? ck + slot * k : seg + slot * ((size_t)(k & 1) * seg_slots + (j - 1));
    };
    bool used[2] = {false, false};
    auto recompute = [&](long long k) -> bool {
        const int b = (int)(k & 1);
        if (used[b] && cudaStreamWaitEvent(rs, ev_free[b], 0) != cudaSuccess) return false;
        used[b] = true;
        for (long long j = 0; j + 1 < seg_len(k); ++j) {
            StepArgs<float> a = base;
            const float* in = state_at(k, j);
            float* out = state_at(k, j + 1);
            a.g_in = in;
            a.g_out = out;
            a.dpsi_in = in + GE;
            a.dpsi_out = out + GE;
            if (fp32_step(a, L, false, rs) != cudaSuccess) return false;
        }
        return cudaEventRecord(ev_ready[b], rs) == cudaSuccess;
    };
    if (cudaEventRecord(ev_fwd, st) != cudaSuccess || cudaStreamWaitEvent(rs, ev_fwd, 0) != cudaSuccess)
        return fail();
    if (K > 0 && !recompute(K - 1)) return fail();
    for (long long k = K - 1; k >= 0; --k) {
        const long long n = seg_len(k);
        if (k > 0 && !recompute(k - 1)) return fail();
        if (cudaStreamWaitEvent(st, ev_ready[k & 1], 0) != cudaSuccess) return fail();
        for (long long j = n - 1; j >= 0; --j) {
            const float* state = state_at(k, j);
            A.g = state;
            A.dpsi = state + GE;
            A.lam_next = lamA;
            A.lam = lamB;
            k_adj_pass_a<<<grid, kAdjThreads, 0, st>>>(A);
            k_adj_pass_b<<<grid, kAdjThreads, 0, st>>>(A);
            if (cudaGetLastError() != cudaSuccess) return fail();
            float* tmp = lamA;
            lamA = lamB;
            lamB = tmp;
        }
        if (cudaEventRecord(ev_free[k & 1], st) != cudaSuccess) return fail();
    }
    double* gout = grad_on_dev ? grad_rho : grad_dev;
    k_adj_grad_init<<<adj_grid(N), kAdjThreads, 0, st>>>(lamA, N, A.a.w0, A.a.w1, A.a.w2, gout);
    if (cudaGetLastError() != cudaSuccess) return fail();
    double h[8];
    if (cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return fail();
    if (!grad_on_dev &&
        cudaMemcpyAsync(grad_rho, grad_dev, sizeof(double) * N, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return fail();
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail();
    release();
    *J_out = h[0] + h[1];
    grad_G[0] = h[2] + h[4];
    grad_G[1] = h[3] + h[5];
    if (!std::isfinite(*J_out) || !std::isfinite(grad_G[0]) || !std::isfinite(grad_G[1]))
        return LB_ERR_NONFINITE;
    return LB_OK;
}

namespace {

__global__ void __launch_bounds__(256) k_misfit64(const double* __restrict__ rho,
                                                  const double* __restrict__ tgt, long long n,
                                                  double* partials, unsigned int* counter,
                                                  double* out)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long s = blockIdx.x * 256LL + threadIdx.x; s < n; s += (long long)gridDim.x * 256) {
        const double m = rho[s] - tgt[s];
        v[0] += m * m;
    }
    if (last_block_total<256>(v, partials, counter, gridDim.x)) *out = v[0];
}

}  // namespace

namespace lbsc {

cudaError_t objective_delta(const lb_state* s, const double* tgt, double* acc, cudaStream_t st)
{
    AdjArgs A{};
    A.a = state_args<float>(s, s->cur);
    A.aw = with_weights(A.a, false);
    A.ap = with_weights(A.a, true);
    A.G1 = (float)s->p.G1;
    A.G2 = (float)s->p.G2;
    A.inv_sqrt_rho0 = (float)(1.0 / std::sqrt(s->p.rho0));
    A.dpsi = s->dpsi[s->cur];
    A.rho_target = tgt;
    A.partials = s->partials;
    A.counter = s->counter;
    A.acc = acc;
    A.lam = nullptr;
    cudaError_t e = cudaMemsetAsync(acc, 0, 4 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int grid = adj_grid(s->N);
    if (s->p.prec == LB_FP16_DELTA)
        k_adj_terminal<__half><<<grid, kAdjThreads, 0, st>>>(A, static_cast<const __half*>(s->g[s->cur]));
    else
        k_adj_terminal<float><<<grid, kAdjThreads, 0, st>>>(A, static_cast<const float*>(s->g[s->cur]));
    return cudaGetLastError();
}

cudaError_t misfit64(const double* rho, const double* tgt, long long n, double* partials,
                     unsigned int* counter, double* out, cudaStream_t st)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    k_misfit64<<<(int)(b < 1 ? 1 : b), 256, 0, st>>>(rho, tgt, n, partials, counter, out);
    return cudaGetLastError();
}

}  // namespace lbsc

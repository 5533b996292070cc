// lb_api.cu — the C ABI of liblbsc.so (include/lb.h): parameter validation,
// device memory of a state, launch sequencing on the caller's stream, and
// host<->device transfers at the boundary.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>
#include <vector>

#include "lb_internal.h"

using namespace lbsc;

namespace lbsc {

// Test hook: allocations left before one is made to fail (-1: never).
static std::atomic<int> g_fail_allocs_after{-1};

void* state_alloc(lb_state* s, size_t bytes)
{
    {
        int left = g_fail_allocs_after.load();
        while (left >= 0 && !g_fail_allocs_after.compare_exchange_weak(left, left - 1)) {
        }
        if (left == 0) return nullptr;   // the hook's failure (counter is now -1: disarmed)
    }
    // round the usable size up so the tail guard starts 256-byte aligned
    const size_t body = (bytes + kGuardBytes - 1) / kGuardBytes * kGuardBytes;
    void* base = nullptr;
    if (cudaMalloc(&base, body + 2 * kGuardBytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    char* b = static_cast<char*>(base);
    if (cudaMemsetAsync(b, kGuardByte, kGuardBytes, s->stream) != cudaSuccess ||
        cudaMemsetAsync(b + kGuardBytes + body, kGuardByte, kGuardBytes, s->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(base);
        return nullptr;
    }
    s->allocs.push_back({base, body});
    return b + kGuardBytes;
}

Couplings couplings(double G1, double G2)
{
    // Table 1 weights; p_s0 = 1 - sum of the 24 link weights (Eq. weights_1)
    const double p1 = 4.0 / 63.0, p2 = 4.0 / 135.0, p4 = 1.0 / 180.0, p5 = 2.0 / 945.0,
                 p8 = 1.0 / 15120.0;
    const double p0 = 1.0 - (4 * p1 + 4 * p2 + 4 * p4 + 8 * p5 + 4 * p8);
    Couplings c;
    c.K0 = G1 * (4.0 / 9.0) + G2 * p0;
    c.K1 = G1 * (1.0 / 9.0) + G2 * p1;
    c.K2 = G1 * (1.0 / 36.0) + G2 * p2;
    c.K4 = G2 * p4;
    c.K5 = G2 * p5;
    c.K8 = G2 * p8;
    return c;
}

// Where a kernel can read or write an array directly: device (or managed) memory
// as it is, pinned host memory through its device alias (read or written over
// the host link by the kernel, no staging copy); nullptr for pageable host memory.
double* device_view(double* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
    if (at.type == cudaMemoryTypeHost && at.devicePointer)
        return static_cast<double*>(at.devicePointer);
    return nullptr;
}

}  // namespace lbsc

namespace {

lb_status validate(const lb_params* p)
{
    if (!p) return LB_ERR_ARG;
    if (p->nx < 5 || p->ny < 5) return LB_ERR_ARG;
    if ((long long)p->nx * p->ny * 9 >= (1LL << 31)) return LB_ERR_ARG;
    if (g_elems(p->nx, p->ny) >= (1LL << 31)) return LB_ERR_ARG;   // 32-bit indices in the steps
    if (!(p->omega > 0.0 && p->omega < 2.0)) return LB_ERR_ARG;
    if (!std::isfinite(p->G1) || !std::isfinite(p->G2)) return LB_ERR_ARG;
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return LB_ERR_ARG;
    if (p->psi_form != LB_PSI_SC_EXP) return LB_ERR_ARG;
    if (p->prec != LB_FP32 && p->prec != LB_FP64 && p->prec != LB_FP16_DELTA) return LB_ERR_ARG;
    if (p->trace_every < 0) return LB_ERR_ARG;
    if (!std::isfinite(p->rho_ref)) return LB_ERR_ARG;
    if (p->device < 0) return LB_ERR_ARG;
    return LB_OK;
}

// Default launch shape: the register-prefetch pipeline (measured faster than
// the bulk-copy rings on GB300 for the 8192^2 lattice; the tuner may still pick
// the rings) with 128-thread strips, or 64-thread strips for lattices whose
// state fits in L2 (512^2: 11.1 us per step against 12.5 us); rows chosen for
// about five waves of 40 resident warps per SM on a 152-SM part (8192^2: 72
// rows, 4.95 waves, the tuned shape), at least 8
// (small lattices have few columns, so short chunks are what gives them enough
// CTAs: 512^2 steps in 11.1 us with 8-row chunks against 15.2 us with 16).
Fp32Launch default_launch(int nx, int ny, lb_precision prec)
{
    (void)prec;
    Fp32Launch L{128, 64, 0};
    if ((long long)nx * ny * 80 <= (128LL << 20)) L.block_x = 64;
    const long long strips = (nx + L.block_x - 3) / (L.block_x - 2);
    const long long target = 152LL * (40 * 32 / L.block_x) * 5;
    long long rows = (strips * ny + target - 1) / target;
    if (rows < 8) rows = 8;
    if (rows > 512) rows = 512;
    L.rows = (int)rows;
    return L;
}

// CTA count of a launch shape (the CTA-partial buffer is sized for the largest)
size_t step_blocks(const lb_state* s, Fp32Launch L)
{
    if (L.pipeline == 1)
        return (size_t)bulk_grid_blocks(s->p.nx, s->p.ny, (int)elem_size(s->p.prec), L);
    return (size_t)fp32_grid_blocks(s->p.nx, s->p.ny, L);
}

template <typename T>
StepArgs<T> make_args(const lb_state* s)
{
    return lbsc::state_args<T>(s, s->cur);
}

}  // namespace

namespace lbsc {

template <typename T>
StepArgs<T> state_args(const lb_state* s, int cur)
{
    const lb_params& p = s->p;
    const Couplings K = couplings(p.G1, p.G2);
    StepArgs<T> a{};
    a.g_in = static_cast<const T*>(s->g[cur]);
    a.g_out = static_cast<T*>(s->g[cur ^ 1]);
    a.dpsi_in = s->dpsi[cur];
    a.dpsi_out = s->dpsi[cur ^ 1];
    a.nx = p.nx;
    a.ny = p.ny;
    a.rows = s->launch.rows;
    a.N = s->N;
    a.pitch = g_pitch(p.nx);
    a.npitch = (int)g_elems(p.nx, p.ny);
    a.omega = (float)p.omega;
    a.omc = (float)(1.0 - p.omega);
    a.inv_omega = (float)(1.0 / p.omega);
    a.w0 = (float)(4.0 / 9.0);
    a.w1 = (float)(1.0 / 9.0);
    a.w2 = (float)(1.0 / 36.0);
    a.K0 = (float)K.K0;
    a.K1 = (float)K.K1;
    a.K2 = (float)K.K2;
    a.K4 = (float)K.K4;
    a.K5 = (float)K.K5;
    a.K8 = (float)K.K8;
    a.rho_ref = (float)s->rho_ref;
    a.psi_ref = (float)(std::sqrt(p.rho0) * -std::expm1(-s->rho_ref / p.rho0));
    a.cpsi = (float)(-std::sqrt(p.rho0) * std::exp(-s->rho_ref / p.rho0));
    a.inv_rho0 = (float)(1.0 / p.rho0);
    a.half_A1 = (float)(0.5 * (p.G1 + p.G2));
    a.partials = s->partials;
    a.counter = s->counter;
    a.trace = s->trace;
    a.trace_count = s->trace_count;
    a.t = s->t;
    a.err = s->err;
    a.wait_cycles = s->wait_cycles;
    a.skip_unit0 = s->skip_unit0;
    return a;
}

template StepArgs<float> state_args<float>(const lb_state*, int);
template StepArgs<__half> state_args<__half>(const lb_state*, int);

size_t elem_size(lb_precision p) { return p == LB_FP16_DELTA ? 2 : 4; }

}  // namespace lbsc

namespace {

lb_status fail_cuda(lb_state* s)
{
    if (s) s->poisoned = true;
    cudaGetLastError();
    return LB_ERR_CUDA;
}

// Read the kernels' error flags (synchronises the stream): bit 1, a bounded
// wait ran out (the state is poisoned); bit 2, a fused reduction produced a
// non-finite mass or energy (the lattice has blown up).
lb_status check_err(lb_state* s)
{
    int e = 0;
    if (cudaMemcpyAsync(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return fail_cuda(s);
    if (e & 1) {
        s->poisoned = true;
        return LB_ERR_TIMEOUT;
    }
    if (e & 2) return LB_ERR_NONFINITE;
    return LB_OK;
}

#define LB_CUDA(s, call)                          \
    do {                                          \
        if ((call) != cudaSuccess) return fail_cuda(s); \
    } while (0)

void free_state(lb_state* s)
{
    if (!s) return;
    DeviceScope dev(s->p.device);
    cudaStreamSynchronize(s->stream);
    for (const lb_state::Alloc& a : s->allocs) cudaFree(a.base);
    cudaGetLastError();
    delete s;
}

lb_status step_fp32(lb_state* s, long n)
{
    for (long k = 0; k < n; ++k) {
        const bool reduce = s->p.trace_every > 0 && (s->t % s->p.trace_every) == 0;
        cudaError_t e;
        const bool bulk = s->launch.pipeline == 1;
        if (s->p.prec == LB_FP32)
            e = bulk ? fp32_step_bulk(make_args<float>(s), s->launch, reduce, s->stream)
                     : fp32_step(make_args<float>(s), s->launch, reduce, s->stream);
        else
            e = bulk ? fp16_step_bulk(make_args<__half>(s), s->launch, reduce, s->stream)
                     : fp16_step(make_args<__half>(s), s->launch, reduce, s->stream);
        if (e != cudaSuccess) return fail_cuda(s);
        s->cur ^= 1;
        s->t += 1;
    }
    return LB_OK;
}

Fp64Args make64(const lb_state* s)
{
    Fp64Args a;
    a.f_in = s->f64[s->cur];
    a.f_out = s->f64[s->cur ^ 1];
    a.psi = s->psi64;
    a.rho = s->rho64;
    a.nx = s->p.nx;
    a.ny = s->p.ny;
    a.omega = s->p.omega;
    a.G1 = s->p.G1;
    a.G2 = s->p.G2;
    a.rho0 = s->p.rho0;
    return a;
}

lb_status step_fp64(lb_state* s, long n)
{
    for (long k = 0; k < n; ++k) {
        const Fp64Args a = make64(s);
        LB_CUDA(s, fp64_psi(a, s->stream));
        if (s->p.trace_every > 0 && (s->t % s->p.trace_every) == 0)
            LB_CUDA(s, fp64_energy(a, s->partials, s->counter, s->res, s->trace, s->trace_count,
                                   s->t, s->stream));
        LB_CUDA(s, fp64_collide_stream(a, s->stream));
        s->cur ^= 1;
        s->t += 1;
    }
    return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_status_str(lb_status st)
{
    switch (st) {
    case LB_OK: return "ok";
    case LB_ERR_ARG: return "invalid argument";
    case LB_ERR_CUDA: return "CUDA error (state poisoned)";
    case LB_ERR_OOM: return "device allocation failed";
    case LB_ERR_NONFINITE: return "non-finite density or energy";
    case LB_ERR_STATE: return "call not valid in the current state";
    case LB_ERR_TIMEOUT: return "an in-kernel wait ran out (state poisoned)";
    }
    return "unknown status";
}

lb_status lb_init(lb_state** out, const lb_params* p, const double* rho_init, void* stream)
{
    NvtxRange nvtx_range("lb_init");
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    if (validate(p) != LB_OK || !rho_init) return LB_ERR_ARG;
    lb_state* s = new (std::nothrow) lb_state();
    if (!s) return LB_ERR_OOM;
    s->p = *p;
    s->stream = static_cast<cudaStream_t>(stream);
    s->N = (long long)p->nx * p->ny;
    const long long N = s->N;
    DeviceScope dev(p->device);
    if (!dev.ok) {
        delete s;
        return LB_ERR_CUDA;
    }
    auto alloc = [&](void** q, size_t bytes) -> bool {
        *q = state_alloc(s, bytes);
        return *q != nullptr;
    };
    s->launch = default_launch(p->nx, p->ny, p->prec);
    size_t nblk_step = (size_t)fp32_grid_blocks(p->nx, p->ny, Fp32Launch{64, kMinRows, 0});
    const size_t nblk_bulk =
        (size_t)bulk_grid_blocks(p->nx, p->ny, (int)elem_size(p->prec), Fp32Launch{64, kMinRows, 1});
    if (nblk_bulk > nblk_step) nblk_step = nblk_bulk;
    s->partials_cap = nblk_step > 152 * 16 ? nblk_step : 152 * 16;
    // the reduction step's grid sum keeps one total per CTA row after the CTA partials
    s->max_cta_rows = (p->ny + kMinRows - 1) / kMinRows;
    s->partials_cap += (size_t)s->max_cta_rows;
    bool ok = alloc((void**)&s->partials, 4 * sizeof(double) * s->partials_cap) &&
              alloc((void**)&s->counter, sizeof(unsigned int)) &&
              alloc((void**)&s->trace, sizeof(double) * kTraceCap * kTraceCols) &&
              alloc((void**)&s->trace_count, sizeof(int)) &&
              alloc((void**)&s->res, 4 * sizeof(double)) && alloc((void**)&s->flag, sizeof(int)) &&
              alloc((void**)&s->err, sizeof(int));
    if (ok && p->prec == LB_FP64) {
        ok = alloc((void**)&s->f64[0], 9 * sizeof(double) * N) &&
             alloc((void**)&s->f64[1], 9 * sizeof(double) * N) &&
             alloc((void**)&s->psi64, sizeof(double) * N) &&
             alloc((void**)&s->rho64, sizeof(double) * N);
    } else if (ok) {
        const size_t es = elem_size(p->prec);
        const size_t gb = es * (size_t)g_elems(p->nx, p->ny);
        ok = alloc(&s->g[0], gb) && alloc(&s->g[1], gb) &&
             alloc((void**)&s->dpsi[0], sizeof(float) * N) &&
             alloc((void**)&s->dpsi[1], sizeof(float) * N);
    }
    if (!ok) {
        free_state(s);
        return LB_ERR_OOM;
    }
    // rho_init is copied once (one DMA transfer, whatever memory it is in) into the
    // second population buffer, which holds nothing until the first step writes it
    // and is at least 8 N bytes in every precision; the checks and the
    // initialisation then read device memory only.
    double* rho_in = static_cast<double*>(p->prec == LB_FP64 ? (void*)s->f64[1] : s->g[1]);
    auto bail = [&](lb_status st) {
        cudaGetLastError();
        free_state(s);
        return st;
    };
    if (cudaMemcpyAsync(rho_in, rho_init, sizeof(double) * N, cudaMemcpyDefault, s->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(s->counter, 0, sizeof(unsigned int), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->trace_count, 0, sizeof(int), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->err, 0, sizeof(int), s->stream) != cudaSuccess)
        return bail(LB_ERR_CUDA);
    if (rho_check_sum(rho_in, N, s->partials, s->counter, s->res, s->flag, s->stream) !=
        cudaSuccess)
        return bail(LB_ERR_CUDA);
    double sum = 0.0;
    int flag = 0;
    // after this synchronisation the caller's rho_init is no longer read
    if (cudaMemcpyAsync(&sum, s->res, sizeof(double), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&flag, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return bail(LB_ERR_CUDA);
    if (flag) return bail(LB_ERR_ARG);
    // The reference density is rounded to FP32 once: the kernels add it in FP32,
    // the deviations at init and the mass/field reconstructions use it in FP64,
    // and all of them must mean the same number.
    s->rho_ref = (double)(float)(p->rho_ref > 0.0 ? p->rho_ref : sum / (double)N);
    const bool padded = p->prec != LB_FP64 && g_pitch(p->nx) != 9 * p->nx;
    const size_t gbytes = elem_size(p->prec) * (size_t)g_elems(p->nx, p->ny);
    if (padded && cudaMemsetAsync(s->g[0], 0, gbytes, s->stream) != cudaSuccess)
        return bail(LB_ERR_CUDA);
    cudaError_t e;
    if (p->prec == LB_FP64)
        e = fp64_init(s->f64[0], rho_in, p->nx, p->ny, s->stream);
    else if (p->prec == LB_FP32)
        e = delta_init<float>(static_cast<float*>(s->g[0]), s->dpsi[0], rho_in, p->nx, p->ny,
                              s->rho_ref, p->rho0, s->stream);
    else
        e = delta_init<__half>(static_cast<__half*>(s->g[0]), s->dpsi[0], rho_in, p->nx, p->ny,
                               s->rho_ref, p->rho0, s->stream);
    if (e != cudaSuccess) return bail(LB_ERR_CUDA);
    // the padding columns of the tiled populations hold zeros in both buffers (nx
    // not a multiple of 32; otherwise every element of g[0] is written by the
    // initialisation and every element of g[1] by the first step); g[1] is
    // cleared after the initialisation has read rho_init from it
    if (padded && cudaMemsetAsync(s->g[1], 0, gbytes, s->stream) != cudaSuccess)
        return bail(LB_ERR_CUDA);
    *out = s;
    return LB_OK;
}

lb_status lb_step(lb_state* s, long n)
{
    NvtxRange nvtx_range("lb_step");
    if (!s || n < 0) return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    if (n == 0) return LB_OK;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    return s->p.prec == LB_FP64 ? step_fp64(s, n) : step_fp32(s, n);
}

lb_status lb_energy(lb_state* s, double out[4])
{
    NvtxRange nvtx_range("lb_energy");
    if (!s || !out) return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    if (s->p.prec == LB_FP64) {
        const Fp64Args a = make64(s);
        LB_CUDA(s, fp64_psi(a, s->stream));
        LB_CUDA(s, fp64_energy(a, s->partials, s->counter, s->res, nullptr, nullptr, s->t,
                               s->stream));
    } else if (s->p.prec == LB_FP32) {
        const StepArgs<float> a = make_args<float>(s);
        LB_CUDA(s, delta_energy<float>(a.g_in, a.dpsi_in, s->p.nx, s->p.ny, a, s->res,
                                       s->partials, s->counter, s->stream));
    } else {
        const StepArgs<__half> a = make_args<__half>(s);
        LB_CUDA(s, delta_energy<__half>(a.g_in, a.dpsi_in, s->p.nx, s->p.ny, a, s->res,
                                        s->partials, s->counter, s->stream));
    }
    double h[4];
    LB_CUDA(s, cudaMemcpyAsync(h, s->res, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    {
        const lb_status st = check_err(s);
        if (st != LB_OK) return st;
    }
    for (int k = 0; k < 4; ++k) out[k] = h[k];
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(h[k])) return LB_ERR_NONFINITE;
    return LB_OK;
}

lb_status lb_objective(lb_state* s, const double* rho_target, double* J)
{
    NvtxRange nvtx_range("lb_objective");
    if (!s || !rho_target || !J) return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    const long long N = s->N;
    // the target where a kernel can read it: in place, or copied into the
    // state's field buffer (allocated on first use, as by lb_fields)
    const double* tgt = device_view(const_cast<double*>(rho_target));
    if (!tgt) {
        if (!s->field_tmp) {
            s->field_tmp = static_cast<double*>(state_alloc(s, sizeof(double) * N));
            if (!s->field_tmp) return LB_ERR_OOM;
        }
        LB_CUDA(s, cudaMemcpyAsync(s->field_tmp, rho_target, sizeof(double) * N,
                                   cudaMemcpyHostToDevice, s->stream));
        tgt = s->field_tmp;
    }
    double h[4] = {0.0, 0.0, 0.0, 0.0};
    if (s->p.prec == LB_FP64) {
        // psi and rho of the current state, the Sec. 5 sums, then the misfit
        const Fp64Args a = make64(s);
        LB_CUDA(s, fp64_psi(a, s->stream));
        LB_CUDA(s, fp64_energy(a, s->partials, s->counter, s->res, nullptr, nullptr, s->t,
                               s->stream));
        LB_CUDA(s, cudaMemcpyAsync(h, s->res, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                   s->stream));
        LB_CUDA(s, misfit64(s->rho64, tgt, N, s->partials, s->counter, s->res, s->stream));
        LB_CUDA(s, cudaMemcpyAsync(h + 2, s->res, sizeof(double), cudaMemcpyDeviceToHost,
                                   s->stream));
        LB_CUDA(s, cudaStreamSynchronize(s->stream));
        *J = (h[0] + h[1]) + h[2];
    } else {
        // the terminal sums of lb_adjoint (same kernel, grid and order)
        LB_CUDA(s, objective_delta(s, tgt, s->res, s->stream));
        LB_CUDA(s, cudaMemcpyAsync(h, s->res, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                   s->stream));
        LB_CUDA(s, cudaStreamSynchronize(s->stream));
        *J = h[0] + h[1];
    }
    {
        const lb_status st = check_err(s);
        if (st != LB_OK) return st;
    }
    return std::isfinite(*J) ? LB_OK : LB_ERR_NONFINITE;
}

static cudaError_t fields_into(lb_state* s, double* r, double* x, double* y)
{
    if (s->p.prec == LB_FP64) return fp64_fields(s->f64[s->cur], s->p.nx, s->p.ny, r, x, y, s->stream);
    if (s->p.prec == LB_FP32)
        return delta_fields<float>(static_cast<const float*>(s->g[s->cur]), s->p.nx, s->p.ny,
                                   s->rho_ref, r, x, y, s->stream);
    return delta_fields<__half>(static_cast<const __half*>(s->g[s->cur]), s->p.nx, s->p.ny,
                                s->rho_ref, r, x, y, s->stream);
}

lb_status lb_fields(lb_state* s, double* rho, double* ux, double* uy)
{
    NvtxRange nvtx_range("lb_fields");
    if (!s) return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    const long long N = s->N;
    double* outs[3] = {rho, ux, uy};
    double* views[3];
    for (int k = 0; k < 3; ++k) views[k] = device_view(outs[k]);
    // every output a kernel can write directly: one pass over the populations
    if (views[0] || views[1] || views[2]) {
        if (fields_into(s, views[0], views[1], views[2]) != cudaSuccess) return fail_cuda(s);
    }
    // pageable host outputs: through a device buffer, one field at a time
    for (int k = 0; k < 3; ++k) {
        if (!outs[k] || views[k]) continue;
        if (!s->field_tmp) {
            s->field_tmp = static_cast<double*>(state_alloc(s, sizeof(double) * N));
            if (!s->field_tmp) {
                cudaGetLastError();
                s->field_tmp = nullptr;
                return LB_ERR_OOM;
            }
        }
        double* t = s->field_tmp;
        if (fields_into(s, k == 0 ? t : nullptr, k == 1 ? t : nullptr, k == 2 ? t : nullptr) !=
            cudaSuccess)
            return fail_cuda(s);
        LB_CUDA(s, cudaMemcpyAsync(outs[k], t, sizeof(double) * N, cudaMemcpyDeviceToHost,
                                   s->stream));
    }
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    return check_err(s);
}

lb_status lb_trace(lb_state* s, double* buf, int cap, int* count)
{
    NvtxRange nvtx_range("lb_trace");
    if (!s || !count || cap < 0 || (cap > 0 && !buf)) return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    int total = 0;
    LB_CUDA(s, cudaMemcpyAsync(&total, s->trace_count, sizeof(int), cudaMemcpyDeviceToHost,
                               s->stream));
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    const int stored = total < kTraceCap ? total : kTraceCap;
    const int n = stored < cap ? stored : cap;
    // rows total-n .. total-1, oldest first; row r lives in ring slot r % kTraceCap,
    // so the rows form at most two contiguous runs of the ring
    int done = 0;
    while (done < n) {
        const int slot = (total - n + done) % kTraceCap;
        int run = kTraceCap - slot;
        if (run > n - done) run = n - done;
        LB_CUDA(s, cudaMemcpyAsync(buf + (size_t)done * kTraceCols,
                                   s->trace + (size_t)slot * kTraceCols,
                                   sizeof(double) * kTraceCols * run, cudaMemcpyDeviceToHost,
                                   s->stream));
        done += run;
    }
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    *count = n;
    return check_err(s);
}

namespace {
struct SavedHeader {
    char magic[8];            // "LBSCSTAT"
    int version, nx, ny, prec;
    long long t;
    double rho_ref;
    long long payload;        // bytes after the header
};
constexpr int kSaveVersion = 4;   // 4: tiled populations of state t (pairs side by side, FP16 too)

size_t payload_bytes(const lb_state* s)
{
    if (s->p.prec == LB_FP64) return sizeof(double) * 9 * (size_t)s->N;
    return elem_size(s->p.prec) * (size_t)g_elems(s->p.nx, s->p.ny) +
           sizeof(float) * (size_t)s->N;
}
}  // namespace

lb_status lb_check_guards(lb_state* s, int* damaged)
{
    NvtxRange nvtx_range("lb_check_guards");
    if (!s || !damaged) return LB_ERR_ARG;
    *damaged = 0;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    std::vector<unsigned char> h(2 * kGuardBytes);
    for (const lb_state::Alloc& a : s->allocs) {
        const char* b = static_cast<const char*>(a.base);
        LB_CUDA(s, cudaMemcpy(h.data(), b, kGuardBytes, cudaMemcpyDeviceToHost));
        LB_CUDA(s, cudaMemcpy(h.data() + kGuardBytes, b + kGuardBytes + a.bytes, kGuardBytes,
                              cudaMemcpyDeviceToHost));
        for (unsigned char c : h)
            if (c != kGuardByte) {
                ++*damaged;
                break;
            }
    }
    return LB_OK;
}

void lb_debug_fail_alloc(int after)
{
    lbsc::g_fail_allocs_after.store(after < 0 ? -1 : after);
}

lb_status lb_debug_damage_guard(lb_state* s, int buffer)
{
    NvtxRange nvtx_range("lb_debug_damage_guard");
    if (!s || buffer < 0 || buffer >= (int)s->allocs.size()) return LB_ERR_ARG;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    const lb_state::Alloc& a = s->allocs[(size_t)buffer];
    char* tail = static_cast<char*>(a.base) + kGuardBytes + a.bytes;
    LB_CUDA(s, cudaMemsetAsync(tail + 17, 0x00, 1, s->stream));
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    return LB_OK;
}

size_t lb_state_bytes(const lb_state* s)
{
    return s ? sizeof(SavedHeader) + payload_bytes(s) : 0;
}

lb_status lb_save_state(lb_state* s, void* dst, size_t bytes)
{
    NvtxRange nvtx_range("lb_save_state");
    if (!s || !dst || bytes < lb_state_bytes(s)) return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    SavedHeader h{};
    std::memcpy(h.magic, "LBSCSTAT", 8);
    h.version = kSaveVersion;
    h.nx = s->p.nx;
    h.ny = s->p.ny;
    h.prec = (int)s->p.prec;
    h.t = s->t;
    h.rho_ref = s->rho_ref;
    h.payload = (long long)payload_bytes(s);
    char* d = static_cast<char*>(dst);
    const cudaMemcpyKind k = cudaMemcpyDefault;
    LB_CUDA(s, cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyDefault, s->stream));
    d += sizeof(h);
    if (s->p.prec == LB_FP64) {
        LB_CUDA(s, cudaMemcpyAsync(d, s->f64[s->cur], sizeof(double) * 9 * s->N, k, s->stream));
    } else {
        const size_t gb = elem_size(s->p.prec) * (size_t)g_elems(s->p.nx, s->p.ny);
        LB_CUDA(s, cudaMemcpyAsync(d, s->g[s->cur], gb, k, s->stream));
        LB_CUDA(s, cudaMemcpyAsync(d + gb, s->dpsi[s->cur], sizeof(float) * s->N, k, s->stream));
    }
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    return LB_OK;
}

lb_status lb_load_state(lb_state* s, const void* src, size_t bytes)
{
    NvtxRange nvtx_range("lb_load_state");
    if (!s || !src || bytes < sizeof(SavedHeader)) return LB_ERR_ARG;
    if (s->poisoned) return LB_ERR_STATE;
    DeviceScope dev(s->p.device);
    if (!dev.ok) return fail_cuda(s);
    SavedHeader h{};
    LB_CUDA(s, cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDefault, s->stream));
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    if (std::memcmp(h.magic, "LBSCSTAT", 8) != 0 || h.version != kSaveVersion ||
        h.nx != s->p.nx || h.ny != s->p.ny || h.prec != (int)s->p.prec ||
        h.payload != (long long)payload_bytes(s) || bytes < lb_state_bytes(s) || h.t < 0)
        return LB_ERR_ARG;
    if (s->p.prec != LB_FP64 && h.rho_ref != s->rho_ref) return LB_ERR_ARG;
    const char* d = static_cast<const char*>(src) + sizeof(h);
    const cudaMemcpyKind k = cudaMemcpyDefault;
    if (s->p.prec == LB_FP64) {
        LB_CUDA(s, cudaMemcpyAsync(s->f64[0], d, sizeof(double) * 9 * s->N, k, s->stream));
    } else {
        const size_t gb = elem_size(s->p.prec) * (size_t)g_elems(s->p.nx, s->p.ny);
        LB_CUDA(s, cudaMemcpyAsync(s->g[0], d, gb, k, s->stream));
        LB_CUDA(s, cudaMemcpyAsync(s->dpsi[0], d + gb, sizeof(float) * s->N, k, s->stream));
    }
    LB_CUDA(s, cudaStreamSynchronize(s->stream));
    s->cur = 0;
    s->t = h.t;
    return LB_OK;
}

lb_status lb_get_launch(const lb_state* s, int* block_x, int* rows_per_cta, int* pipeline)
{
    if (!s || !block_x || !rows_per_cta || !pipeline) return LB_ERR_ARG;
    if (s->p.prec == LB_FP64) return LB_ERR_STATE;
    *block_x = s->launch.block_x;
    *rows_per_cta = s->launch.rows;
    *pipeline = s->launch.pipeline;
    return LB_OK;
}

lb_status lb_set_launch(lb_state* s, int block_x, int rows_per_cta, int pipeline)
{
    if (!s) return LB_ERR_ARG;
    if (s->p.prec == LB_FP64) return LB_ERR_STATE;
    if (rows_per_cta < kMinRows || rows_per_cta > kMaxRows) return LB_ERR_ARG;
    if (pipeline == 0) {
        if (block_x != 64 && block_x != 96 && block_x != 128 && block_x != 192 && block_x != 256)
            return LB_ERR_ARG;
    } else if (pipeline == 1) {
        if (block_x != 64 && block_x != 128 && block_x != 256) return LB_ERR_ARG;
        if (!bulk_supported(s->p.nx, s->p.ny, (int)elem_size(s->p.prec), block_x))
            return LB_ERR_ARG;
    } else {
        return LB_ERR_ARG;
    }
    const Fp32Launch L{block_x, rows_per_cta, pipeline};
    // the CTA-partial buffer was sized for the smallest CTAs (64 threads, kMinRows rows)
    // and one row total per CTA row
    if (step_blocks(s, L) + (size_t)s->max_cta_rows > s->partials_cap) return LB_ERR_ARG;
    s->launch = L;
    return LB_OK;
}

lb_status lb_set_wait_limit(lb_state* s, long long cycles, int test_skip_copies)
{
    if (!s || cycles <= 0 || (test_skip_copies != 0 && test_skip_copies != 1)) return LB_ERR_ARG;
    s->wait_cycles = cycles;
    s->skip_unit0 = test_skip_copies;
    return LB_OK;
}

long lb_time(const lb_state* s) { return s ? (long)s->t : -1; }

void lb_destroy(lb_state* s)
{
    NvtxRange nvtx_range("lb_destroy");
    free_state(s);
}

}  // extern "C"

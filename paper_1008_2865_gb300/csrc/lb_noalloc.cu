// lb_noalloc.cu — lb_energy_noalloc: the pseudo-energy / mass reduction of the
// FP64 path, for callers that cannot allocate device memory. The CTA partial
// sums, the arrival counter and the result live in one file-scope static
// device array instead of memory from cudaMalloc; the caller passes the
// fields in and receives the four sums. Nothing in this file allocates.
#include <cmath>
#include <mutex>

#include "lb_internal.h"

namespace lbsc {
namespace {

// Scratch layout, in doubles: [0] arrival counter (its first 4 bytes, as an
// unsigned int), [4..7] the result, [8 ..) the per-CTA partials (4 each).
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocSitesPerThread = 64;
constexpr long long kNoAllocSitesPerCta = (long long)kNoAllocThreads * kNoAllocSitesPerThread;
constexpr int kNoAllocMaxCtas = 8192;
constexpr int kNoAllocHeader = 8;
constexpr int kNoAllocDoubles = kNoAllocHeader + 4 * kNoAllocMaxCtas;   // 262,208 bytes

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device addresses of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ int wrap(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ double at(const double* f, int x, int y, int nx, int ny)
{
    return f[(long long)wrap(y, ny) * nx + wrap(x, nx)];
}

// Per site (Sec. 5): 1/2 psi sum_{i=0..8} (G1 w_i + G2 p_si) psi(x + c_i),
// 1/2 psi sum_{belt 2} G2 p_mi psi(x + c_mi), (G1 + G2)/2 psi^2, and rho.
// Each CTA covers kNoAllocSitesPerCta consecutive sites; the last CTA to
// arrive sums the partials in CTA order and writes the result.
__global__ void __launch_bounds__(kNoAllocThreads)
k_energy_noalloc(const double* __restrict__ psi, const double* __restrict__ rho, int nx, int ny,
                 double K0, double K1, double K2, double K4, double K5, double K8, double halfA1,
                 double* scratch)
{
    const long long N = (long long)nx * ny;
    const long long s0 = (long long)blockIdx.x * kNoAllocSitesPerCta;
    const long long s1 = s0 + kNoAllocSitesPerCta < N ? s0 + kNoAllocSitesPerCta : N;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long s = s0 + threadIdx.x; s < s1; s += kNoAllocThreads) {
        const int y = (int)(s / nx), x = (int)(s % nx);
        const double p = psi[s];
        const double S1 = at(psi, x + 1, y, nx, ny) + at(psi, x - 1, y, nx, ny) +
                          at(psi, x, y + 1, nx, ny) + at(psi, x, y - 1, nx, ny);
        const double S2 = at(psi, x + 1, y + 1, nx, ny) + at(psi, x - 1, y + 1, nx, ny) +
                          at(psi, x + 1, y - 1, nx, ny) + at(psi, x - 1, y - 1, nx, ny);
        const double S4 = at(psi, x + 2, y, nx, ny) + at(psi, x - 2, y, nx, ny) +
                          at(psi, x, y + 2, nx, ny) + at(psi, x, y - 2, nx, ny);
        double S5 = 0.0;
        for (int a = -2; a <= 2; a += 4)
            for (int b = -1; b <= 1; b += 2)
                S5 += at(psi, x + a, y + b, nx, ny) + at(psi, x + b, y + a, nx, ny);
        const double S8 = at(psi, x + 2, y + 2, nx, ny) + at(psi, x - 2, y + 2, nx, ny) +
                          at(psi, x + 2, y - 2, nx, ny) + at(psi, x - 2, y - 2, nx, ny);
        v[0] += 0.5 * p * (K0 * p + K1 * S1 + K2 * S2);
        v[1] += 0.5 * p * (K4 * S4 + K5 * S5 + K8 * S8);
        v[2] += halfA1 * p * p;
        v[3] += rho[s];
    }
    // deterministic CTA sum: warp shuffles, then the warps in order
    __shared__ double red[kNoAllocThreads / 32][4];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < 4; ++k) red[warp][k] = v[k];
    __syncthreads();
    double* partials = scratch + kNoAllocHeader;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNoAllocThreads / 32; ++w)
            for (int k = 0; k < 4; ++k) v[k] += red[w][k];
        for (int k = 0; k < 4; ++k) partials[4 * blockIdx.x + k] = v[k];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double w[4] = {0.0, 0.0, 0.0, 0.0};
        for (unsigned int j = 0; j < gridDim.x; ++j)
            for (int k = 0; k < 4; ++k) w[k] += __ldcg(partials + 4 * j + k);
        for (int k = 0; k < 4; ++k) scratch[4 + k] = w[k];
        *counter = 0u;
    }
}

// Device ordinal of device (or managed) memory p; -1 for host memory, an
// unknown pointer or NULL.
int device_of(const void* p)
{
    if (!p) return -1;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return at.device;
    return -1;
}

// The device address of the scratch array on the current device (looked up
// on the first call per device with that device current).
double* scratch_address(int dev)
{
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    return g_addr[dev];
}

}  // namespace
}  // namespace lbsc

extern "C" lb_status lb_energy_noalloc(const double* psi, const double* rho, int nx, int ny,
                                       double G1, double G2, double* out, void* stream)
{
    using namespace lbsc;
    NvtxRange nvtx_range("lb_energy_noalloc");
    if (!psi || !rho || !out) return LB_ERR_ARG;
    if (nx < 5 || ny < 5) return LB_ERR_ARG;
    if (!std::isfinite(G1) || !std::isfinite(G2)) return LB_ERR_ARG;
    const long long N = (long long)nx * ny;
    const long long ctas = (N + kNoAllocSitesPerCta - 1) / kNoAllocSitesPerCta;
    if (ctas > kNoAllocMaxCtas) return LB_ERR_ARG;   // more sites than the scratch array covers
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LB_ERR_CUDA;
    }
    // the fields must live on the current device (the kernel reads them there)
    if (device_of(psi) != dev || device_of(rho) != dev) return LB_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int out_dev = device_of(out);
    if (out_dev >= 0 && out_dev != dev) return LB_ERR_ARG;
    const bool dev_out = out_dev == dev;
    if (!dev_out) {
        // a host result needs a stream synchronisation, which a capture forbids
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            return LB_ERR_CUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return LB_ERR_ARG;
    }
    double* scratch = scratch_address(dev);
    if (!scratch) return LB_ERR_CUDA;
    const Couplings K = couplings(G1, G2);
    // the arrival counter must start at zero; the partials are overwritten
    if (cudaMemsetAsync(scratch, 0, sizeof(double), st) != cudaSuccess) {
        cudaGetLastError();
        return LB_ERR_CUDA;
    }
    k_energy_noalloc<<<(unsigned int)ctas, kNoAllocThreads, 0, st>>>(
        psi, rho, nx, ny, K.K0, K.K1, K.K2, K.K4, K.K5, K.K8, 0.5 * (G1 + G2), scratch);
    if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;
    if (cudaMemcpyAsync(out, scratch + 4, 4 * sizeof(double),
                        dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        st) != cudaSuccess) {
        cudaGetLastError();
        return LB_ERR_CUDA;
    }
    if (!dev_out) {
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return LB_ERR_CUDA;
        }
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(out[k])) return LB_ERR_NONFINITE;
    }
    return LB_OK;
}

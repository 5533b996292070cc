// lb_bulk.cu — the fused step of lb_fp32.cu with its input rows staged in
// shared memory by the bulk-copy (TMA) engine: cp.async.bulk copies into
// rings of row buffers, completion signalled through mbarrier transaction
// counts, D rows ahead of the compute. The number of bytes in flight per SM is
// then set by the rings in shared memory rather than by registers, which is
// what a 25-point stencil streaming 80 bytes per site needs to keep HBM busy.
//
// Geometry (T = float or __half, AE = 16 / sizeof(T) elements per 16 bytes):
//   a CTA of BX threads owns TX = AE * floor((BX - 2) / AE) output columns
//   (float: BX - 4) starting at x0 = blockIdx.x * TX (a multiple of AE), and marches
//   over `rows` output rows. Thread k computes the collision at column
//   x0 - 1 + k for k <= TX + 1 (the two halo columns included); the
//   remaining threads repeat column TX + 1 without storing.
//   Row unit j (j = 0, 1, ...) is {g* row y0 - 2 + j (all 9 populations,
//   columns [x0 - AE, x0 + TX + AE)), dpsi row y0 + 1 + j (columns
//   [x0 - 4, x0 + TX + 4))}; units -4..-1 carry only the dpsi rows
//   y0 - 3 .. y0. Collision row r = y0 - 1 + it needs units up to it + 2.
//   Periodic wrap in x splits a window into at most three aligned copies.
// Schedule: units 0..D are issued before the first row; iteration it waits
// for unit it+2 and, after the previous iteration's barrier, issues unit
// it+1+D. A g* row is read by iterations j-2..j and a dpsi row by j..j+4, so
// the slot a new unit overwrites was last read by iteration it-1 when
// NG = D + 2 and NP = D + 6; the barrier it re-arms belongs to unit it,
// waited at iteration it-2, when NB = D + 1.
//
// Every wait on an mbarrier is bounded by a clock limit; a CTA whose wait
// runs out sets the state's error flag and all its threads leave together at
// the next per-row barrier (__syncthreads_or), after a bounded wait for the
// copies they issued. No wait in this file can spin forever.
#include "lb_device.cuh"

#include <cstdint>

namespace lbsc {
namespace {

using namespace dev;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, giving up after
// `limit` SM clock cycles. Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Copy the window [xs, xs + w) of a periodic row (row base `src`, nx
// elements) into dst, splitting at the row ends. All boundaries are
// multiples of 16 bytes; nx >= w so the window wraps at most once.
template <typename E>
__device__ __forceinline__ void copy_window(E* dst, const E* src, int xs, int w, int nx,
                                            uint64_t* bar)
{
    if (xs < 0) {
        bulk_g2s(dst, src + (nx + xs), (uint32_t)(-xs) * sizeof(E), bar);
        bulk_g2s(dst - xs, src, (uint32_t)(w + xs) * sizeof(E), bar);
    } else if (xs + w > nx) {
        const int k = nx - xs;
        bulk_g2s(dst, src + xs, (uint32_t)k * sizeof(E), bar);
        bulk_g2s(dst + k, src, (uint32_t)(w - k) * sizeof(E), bar);
    } else {
        bulk_g2s(dst, src + xs, (uint32_t)w * sizeof(E), bar);
    }
}

template <typename T, int BX>
struct BulkGeom {
    static constexpr int AE = 16 / (int)sizeof(T);      // elements per 16 bytes
    static constexpr int TX = ((BX - 2) / AE) * AE;     // output columns per CTA
    static constexpr int WG = TX + 2 * AE;              // g* window width
    static constexpr int WP = TX + 8;                   // dpsi window width
};

template <typename T, int BX, int D, bool REDUCE, bool OM1>
__global__ void __launch_bounds__(BX) k_step_bulk(const StepArgs<T> a)
{
    using G = BulkGeom<T, BX>;
    constexpr int AE = G::AE, TX = G::TX, WG = G::WG, WP = G::WP;
    constexpr int NG = D + 2, NP = D + 6, NB = D + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* gring = reinterpret_cast<T*>(smem_raw);                                  // [NG][9][WG]
    float* pring = reinterpret_cast<float*>(smem_raw + sizeof(T) * NG * 9 * WG); // [NP][WP]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * NG * 9 * WG +
                                                 sizeof(float) * NP * WP);    // [NB + 1]
    __shared__ float4 exR[2][BX + 2];
    __shared__ float4 exL[2][BX + 2];

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int N = (int)a.N;
    const int x0 = blockIdx.x * TX;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, ny);
    const int H = y1 - y0;
    const int last_unit = H + 3;                 // units 0..H+3 are consumed
    const int txe = min(TX, nx - x0);
    const bool out_col = tid >= 1 && tid <= txe;
    const int tcol = min(tid, TX + 1);
    const int gpos = tcol + AE - 1;              // thread column in the g* window
    const int ppos = tcol + 3;                   // thread column in the dpsi window
    const int xc = x0 - 1 + tid;                 // output column (out_col threads)
    const long long limit = a.wait_cycles;
    const uint32_t unit_bytes = (uint32_t)(9 * WG * sizeof(T) + WP * sizeof(float)) + a.extra_tx;

    // ---- producer: lanes 0..9 of warp 0 issue the copies of one unit
    auto issue_unit = [&](int j) {
        const int lane = tid;                    // only called by warp 0
        uint64_t* bar = &bars[j < 0 ? NB : j % NB];
        if (lane == 0) {
            const uint32_t bytes = j < 0 ? 4u * WP * sizeof(float) + a.extra_tx : unit_bytes;
            mbar_arrive_expect_tx(bar, bytes);
        }
        __syncwarp();
        if (j < 0) {
            // the four leading dpsi rows y0-3 .. y0 (units -4 .. -1)
            if (lane < 4) {
                const int q = wrapi(y0 - 3 + lane, ny);
                copy_window(pring + (lane % NP) * WP, a.dpsi_in + q * nx, x0 - 4, WP, nx, bar);
            }
            return;
        }
        if (lane < 9) {
            const int s = wrapi(y0 - 2 + j, ny);
            copy_window(gring + ((j % NG) * 9 + lane) * WG, a.g_in + (lane * N + s * nx),
                        x0 - AE, WG, nx, bar);
        } else if (lane == 9) {
            const int q = wrapi(y0 + 1 + j, ny);
            copy_window(pring + ((j + 4) % NP) * WP, a.dpsi_in + q * nx, x0 - 4, WP, nx, bar);
        }
    };

    if (tid == 0) {
        for (int k = 0; k <= NB; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid < 32) {
        issue_unit(-1);
        for (int j = 0; j <= D && j <= last_unit; ++j) issue_unit(j);
    }

    // the leading dpsi rows and units 0, 1 (g* rows y0-2, y0-1) before the first row;
    // the barrier after the waits lets iterations 0 and 1 re-arm those barriers
    bool fail = !mbar_wait_bounded(&bars[NB], 0, limit);
    fail |= !mbar_wait_bounded(&bars[0], 0, limit);
    fail |= !mbar_wait_bounded(&bars[1], 0, limit);
    __syncthreads();

    float acc_m = 0.f, acc_0 = 0.f;
    float es = 0.f, em = 0.f, eb = 0.f, ms = 0.f;
    double d_es = 0.0, d_em = 0.0, d_eb = 0.0, d_ms = 0.0;

    for (int it = 0; it <= H + 1; ++it) {
        const int r = y0 - 1 + it;
        // ---- keep D units in flight (slots freed by the previous iteration's barrier);
        // a barrier is re-armed only after warp 0 has seen its previous phase complete
        if (tid < 32 && it + 1 + D <= last_unit && !__any_sync(0xffffffffu, fail)) {
            fence_proxy_async_smem();
            issue_unit(it + 1 + D);
        }
        // ---- unit it+2 completes rows r+1 (g*) and r+4 (dpsi)
        {
            const int j = it + 2;
            fail |= !mbar_wait_bounded(&bars[j % NB], (uint32_t)((j / NB) & 1), limit);
        }
        // ---- pull f_i(x, r) = f*_i(x - c_i) from the g* ring (rows r-1, r, r+1)
        const T* gm = gring + (it % NG) * 9 * WG + gpos;          // row r - 1
        const T* gc = gring + ((it + 1) % NG) * 9 * WG + gpos;    // row r
        const T* gp = gring + ((it + 2) % NG) * 9 * WG + gpos;    // row r + 1
        float f[9];
        f[0] = lds_(gc);
        f[1] = lds_(gc + WG - 1);
        f[2] = lds_(gm + 2 * WG);
        f[3] = lds_(gc + 3 * WG + 1);
        f[4] = lds_(gp + 4 * WG);
        f[5] = lds_(gm + 5 * WG - 1);
        f[6] = lds_(gm + 6 * WG + 1);
        f[7] = lds_(gp + 7 * WG + 1);
        f[8] = lds_(gp + 8 * WG - 1);
        // ---- dpsi rows r-2 .. r+2 (ring slots it .. it+4)
        const float* rows[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) rows[k] = pring + ((it + k) % NP) * WP + ppos;
        const float pc = a.psi_ref + rows[2][0];
        float Sx, Sy;
        force_sums(rows, a, Sx, Sy);
        float gs[9];
        const float d = collide<OM1>(f, -pc * Sx, -pc * Sy, a, gs);

        if (out_col && r >= y0 && r < y1) {
            T* o = a.g_out + (r * nx + xc);
#pragma unroll
            for (int i = 0; i < 9; ++i) st_(o + i * N, gs[i]);
            if (REDUCE) {
                energy_site(rows, pc, a, es, em, eb);
                ms += d;
                if (((r - y0) & 15) == 15) {
                    d_es += es; d_em += em; d_eb += eb; d_ms += ms;
                    es = em = eb = ms = 0.f;
                }
            }
        }
        // ---- hand post-collision values to the neighbouring columns
        exR[it & 1][tid + 1] = make_float4(gs[8], gs[1], gs[5], 0.f);
        exL[it & 1][tid + 1] = make_float4(gs[7], gs[3], gs[6], 0.f);
        if (__syncthreads_or(fail)) {
            if (tid == 0) atomicOr(a.err, 1);
            // bounded wait for every unit this CTA issued and has not consumed
            if (tid == 0) {
                for (int j = it + 3; j <= it + 1 + D && j <= last_unit; ++j)
                    mbar_wait_bounded(&bars[j % NB], (uint32_t)((j / NB) & 1), limit);
            }
            return;
        }
        const float4 R = exR[it & 1][tid];
        const float4 L = exL[it & 1][tid + 2];
        acc_m += gs[4] + (R.x + L.x);
        acc_0 += gs[0] + (R.y + L.y);
        const float acc_p = gs[2] + (R.z + L.z);
        if (out_col && r - 1 >= y0) a.dpsi_out[(r - 1) * nx + xc] = dpsi_of(acc_m, a);
        acc_m = acc_0;
        acc_0 = acc_p;
    }

    if (REDUCE) {
        double v[4] = {d_es + es, d_em + em, d_eb + eb, d_ms + ms};
        const unsigned int nb = gridDim.x * gridDim.y;
        if (last_block_total<BX>(v, a.partials, a.counter, nb)) {
            const double mass = (double)a.N * (double)a.rho_ref + v[3];
            write_trace_row(a.trace, a.trace_count, a.t, mass, v[0], v[1], v[2]);
            if (!isfinite(mass) || !isfinite(v[0]) || !isfinite(v[1])) atomicOr(a.err, 2);
        }
    }
}

template <typename T, int BX, int D, bool REDUCE, bool OM1>
cudaError_t launch_bulk(const StepArgs<T>& a, int rows, cudaStream_t s)
{
    using G = BulkGeom<T, BX>;
    constexpr int NG = D + 2, NP = D + 6, NB = D + 1;
    const size_t smem = sizeof(T) * NG * 9 * G::WG + sizeof(float) * NP * G::WP +
                        sizeof(uint64_t) * (NB + 1);
    auto kern = k_step_bulk<T, BX, D, REDUCE, OM1>;
    // the dynamic shared memory opt-in is a per-device function attribute
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(__atomic_load_n(&configured, __ATOMIC_ACQUIRE) & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        __atomic_fetch_or(&configured, bit, __ATOMIC_RELEASE);
    }
    dim3 grid((a.nx + G::TX - 1) / G::TX, (a.ny + rows - 1) / rows);
    kern<<<grid, BX, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int BX>
cudaError_t launch_bulk_bx(const StepArgs<T>& a, int rows, bool reduce, bool om1, cudaStream_t s)
{
    constexpr int D = 3;
    if (reduce)
        return om1 ? launch_bulk<T, BX, D, true, true>(a, rows, s)
                   : launch_bulk<T, BX, D, true, false>(a, rows, s);
    return om1 ? launch_bulk<T, BX, D, false, true>(a, rows, s)
               : launch_bulk<T, BX, D, false, false>(a, rows, s);
}

template <typename T>
cudaError_t launch_bulk_any(const StepArgs<T>& a, Fp32Launch L, bool reduce, cudaStream_t s)
{
    const bool om1 = a.omega == 1.0f;
    switch (L.block_x) {
    case 64: return launch_bulk_bx<T, 64>(a, L.rows, reduce, om1, s);
    case 128: return launch_bulk_bx<T, 128>(a, L.rows, reduce, om1, s);
    case 256: return launch_bulk_bx<T, 256>(a, L.rows, reduce, om1, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
int bulk_tx(int block_x)
{
    switch (block_x) {
    case 64: return BulkGeom<T, 64>::TX;
    case 128: return BulkGeom<T, 128>::TX;
    case 256: return BulkGeom<T, 256>::TX;
    default: return 0;
    }
}

template <typename T>
int bulk_wg(int block_x)
{
    switch (block_x) {
    case 64: return BulkGeom<T, 64>::WG;
    case 128: return BulkGeom<T, 128>::WG;
    case 256: return BulkGeom<T, 256>::WG;
    default: return 0;
    }
}

}  // namespace

bool bulk_supported(int nx, int ny, int elem_bytes, int block_x)
{
    (void)ny;
    const int ae = 16 / elem_bytes;
    const int tx = elem_bytes == 2 ? bulk_tx<__half>(block_x) : bulk_tx<float>(block_x);
    const int wg = elem_bytes == 2 ? bulk_wg<__half>(block_x) : bulk_wg<float>(block_x);
    if (tx <= 0) return false;
    // every row and population plane starts on a 16-byte boundary, windows wrap at most once
    return nx % ae == 0 && nx % 4 == 0 && nx >= wg && nx >= tx + 8;
}

int bulk_grid_blocks(int nx, int ny, int elem_bytes, Fp32Launch L)
{
    const int tx = elem_bytes == 2 ? bulk_tx<__half>(L.block_x) : bulk_tx<float>(L.block_x);
    if (tx <= 0) return 0;
    return ((nx + tx - 1) / tx) * ((ny + L.rows - 1) / L.rows);
}

cudaError_t fp32_step_bulk(const StepArgs<float>& a, Fp32Launch L, bool reduce, cudaStream_t s)
{
    return launch_bulk_any<float>(a, L, reduce, s);
}

cudaError_t fp16_step_bulk(const StepArgs<__half>& a, Fp32Launch L, bool reduce, cudaStream_t s)
{
    return launch_bulk_any<__half>(a, L, reduce, s);
}

}  // namespace lbsc

// lb_bulk.cu — the fused step of lb_fp32.cu with its input rows staged in
// shared memory by the bulk-copy (TMA) engine: cp.async.bulk copies into
// rings of row buffers, completion signalled through mbarrier transaction
// counts, D rows ahead of the compute, so that the loads in flight do not
// occupy registers. On GB300 the shallowest ring (D = 1) is the fastest: every
// extra row of ring costs resident CTAs, and the step is bound by latency per
// warp rather than by the depth of the prefetch.
//
// Geometry (T = float or __half; nx a multiple of 32):
//   a CTA of BX threads owns TX = 4 floor((BX - 2) / 4) output columns
//   starting at x0 = blockIdx.x * TX (a multiple of 4, so every dpsi window
//   starts on a 16-byte boundary) and marches over `rows` output rows.
//   Thread k computes the collision at column x0 - 1 + k for k <= TX + 1 (the
//   two halo columns included); the remaining threads repeat column TX + 1
//   without storing.
//   Row unit j (j = 0, 1, ...) is {the populations of row y0 - 1 + j: the
//   whole 32-column tiles covering columns [x0 - 1, x0 + TX], contiguous in the
//   tiled layout; dpsi row y0 + 1 + j, columns [x0 - 4, x0 + TX + 4)}; a
//   leading unit carries the dpsi rows y0 - 3 .. y0. Collision row r = y0 - 1
//   + it needs unit it. Periodic wrap in x splits a copy in two.
// Schedule: units 0..D-1 are issued before the first row; iteration it waits
// for unit it and, after the previous iteration's barrier, issues unit it+D.
// A population row is read by its own iteration only and a dpsi row by five,
// so the slot a new unit overwrites was last read by iteration it-1 when
// NG = D + 1 and NP = D + 5; the barrier it re-arms belongs to unit it-1,
// waited at iteration it-1, when NB = D + 1.
//
// Every wait on an mbarrier is bounded by a clock limit; a CTA whose wait
// runs out sets the state's error flag and all its threads leave together at
// the next per-row barrier (__syncthreads_or), after a bounded wait for the
// copies they issued. No wait in this file can spin forever. The test hook of
// lb_set_wait_limit arms unit 0's barrier and issues none of its copies: that
// wait runs out with no copy of the unit in flight, and the units issued
// before the timeout complete before the CTA leaves.
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
    static constexpr int TX = ((BX - 2) / 4) * 4;          // output columns per CTA
    static constexpr int KT = (TX + 64) / kTileW;          // tiles in a population window (max)
    static constexpr int WG = KT * kTileElems;             // elements of a population window
    static constexpr int WP = TX + 8;                      // dpsi window width
};

template <typename T, int BX, int D, bool REDUCE, bool OM1>
__global__ void __launch_bounds__(BX) k_step_bulk(const StepArgs<T> a)
{
    using G = BulkGeom<T, BX>;
    constexpr int TX = G::TX, WG = G::WG, WP = G::WP;
    constexpr int NG = D + 1, NP = D + 5, NB = D + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* gring = reinterpret_cast<T*>(smem_raw);                                   // [NG][WG]
    float* pring = reinterpret_cast<float*>(smem_raw + sizeof(T) * NG * WG);     // [NP][WP]
    uint64_t* bars =
        reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * NG * WG + sizeof(float) * NP * WP);
    __shared__ float4 exR[2][BX + 2];        // right-moving f*: speeds 8, 1, 5
    __shared__ float4 exL[2][BX + 2];        // left-moving f*: speeds 7, 3, 6

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int P = a.pitch;
    const int ntile = nx / kTileW;               // tiles per row
    const int x0 = blockIdx.x * TX;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, ny);
    const int H = y1 - y0;
    const int last_unit = H + 1;                 // units 0..H+1 are consumed
    const int txe = min(TX, nx - x0);
    const bool out_col = tid >= 1 && tid <= txe;
    const int xu = x0 - 1 + min(tid, TX + 1);    // thread column, unwrapped (-1 .. nx)
    const int ta = (x0 - 1) >> 5;                // first tile of the window, unwrapped
    const int nt = ((x0 + TX) >> 5) - ta + 1;    // tiles in this CTA's window
    // the thread column's single and pair offsets within the window of tiles
    using TL = Tile<T>;
    const int gps = ((xu >> 5) - ta) * kTileElems + (xu & (kTileW - 1));
    const int gpp = ((xu >> 5) - ta) * kTileElems + (TL::kPaired ? 2 : 1) * (xu & (kTileW - 1));
    const int ppos = min(tid, TX + 1) + 3;       // thread column in the dpsi window
    const int xc = x0 - 1 + tid;                 // output column (out_col threads)
    const int cs = tsingle(xc), cp = tpair<T>(xc);
    const long long limit = a.wait_cycles;
    const uint32_t unit_bytes = (uint32_t)(nt * kTileElems * sizeof(T) + WP * sizeof(float));

    // ---- producer: lanes 0..2 of warp 0 issue the copies of one unit
    auto issue_unit = [&](int j) {
        const int lane = tid;                    // only called by warp 0
        uint64_t* bar = &bars[j < 0 ? NB : j % NB];
        if (lane == 0) {
            const uint32_t bytes = j < 0 ? 4u * WP * sizeof(float) : unit_bytes;
            mbar_arrive_expect_tx(bar, bytes);
        }
        __syncwarp();
        // test hook: unit 0's barrier is armed for its bytes but none of its copies
        // is issued, so its wait runs out while nothing of that unit is in flight
        if (a.skip_unit0 && j == 0) return;
        if (j < 0) {
            // the four leading dpsi rows y0-3 .. y0
            if (lane < 4) {
                const int q = wrapi(y0 - 3 + lane, ny);
                copy_window(pring + lane * WP, a.dpsi_in + q * nx, x0 - 4, WP, nx, bar);
            }
            return;
        }
        if (lane == 0) {
            // whole tiles ta .. ta+nt-1 of population row y0-1+j, wrapped at the row ends
            const T* row = a.g_in + wrapi(y0 - 1 + j, ny) * P;
            T* dst = gring + (j % NG) * WG;
            copy_window(dst, row, ta * kTileElems, nt * kTileElems, ntile * kTileElems, bar);
        } else if (lane == 1) {
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
        for (int j = 0; j < D && j <= last_unit; ++j) issue_unit(j);
    }
    bool fail = !mbar_wait_bounded(&bars[NB], 0, limit);   // the leading dpsi rows

    float acc_m = 0.f, acc_0 = 0.f;
    float es = 0.f, em = 0.f, eb = 0.f, ms = 0.f;
    double d_es = 0.0, d_em = 0.0, d_eb = 0.0, d_ms = 0.0;
    // population row offsets (row * P) of rows r-1, r, r+1 for the stores
    int s0 = wrapi(y0 - 2, ny) * P;
    int s1 = wrapi(y0 - 1, ny) * P;
    int s2 = wrapi(y0, ny) * P;

    for (int it = 0; it <= H + 1; ++it) {
        const int r = y0 - 1 + it;
        // ---- keep D units in flight (slots freed by the previous iteration's barrier)
        if (tid < 32 && it + D <= last_unit && !__any_sync(0xffffffffu, fail)) {
            fence_proxy_async_smem();
            issue_unit(it + D);
        }
        // ---- unit it completes population row r and dpsi row r+2
        fail |= !mbar_wait_bounded(&bars[it % NB], (uint32_t)((it / NB) & 1), limit);
        const T* gr = gring + (it % NG) * WG;
        float f[9];
        f[0] = lds_(gr + gps + TL::P0);
        f[2] = lds_(gr + gps + TL::P2);
        f[4] = lds_(gr + gps + TL::P4);
        lds2<TL::A13, TL::B13>(gr + gpp, f[1], f[3]);
        lds2<TL::A56, TL::B56>(gr + gpp, f[5], f[6]);
        lds2<TL::A78, TL::B78>(gr + gpp, f[7], f[8]);
        // ---- dpsi rows r-2 .. r+2 (ring slots it .. it+4)
        const float* rows[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) rows[k] = pring + ((it + k) % NP) * WP + ppos;
        const float pc = a.psi_ref + rows[2][0];
        float Sx, Sy;
        force_sums(rows, a, Sx, Sy);
        float gs[9];
        const float d = collide<OM1>(f, -pc * Sx, -pc * Sy, a, gs);

        const bool out_site = out_col && r >= y0 && r < y1;
        if (REDUCE && out_site) {
            energy_site(rows, pc, a, es, em, eb);
            ms += d;
            if (((r - y0) & 63) == 63) {
                d_es += es; d_em += em; d_eb += eb; d_ms += ms;
                es = em = eb = ms = 0.f;
            }
        }
        // ---- stream on chip (Eq. 1) as in lb_fp32.cu: own-column speeds now,
        // the neighbouring columns' after the barrier
        exR[it & 1][tid + 1] = make_float4(gs[8], gs[1], gs[5], 0.f);
        exL[it & 1][tid + 1] = make_float4(gs[7], gs[3], gs[6], 0.f);
        const bool st_m = out_col && r - 1 >= y0;
        const bool st_0 = out_site;
        const bool st_p = out_col && r + 1 < y1;
        if (__syncthreads_or(fail)) {
            if (tid == 0) atomicOr(a.err, 1);
            // bounded wait for every unit this CTA issued and has not consumed
            if (tid == 0) {
                for (int j = it + 1; j <= it + D && j <= last_unit; ++j)
                    mbar_wait_bounded(&bars[j % NB], (uint32_t)((j / NB) & 1), limit);
            }
            return;
        }
        const float4 R = exR[it & 1][tid];
        const float4 L = exL[it & 1][tid + 2];
        if (st_m) {
            st_(a.g_out + (s0 + cs + TL::P4), gs[4]);
            st2<TL::A78, TL::B78>(a.g_out + (s0 + cp), L.x, R.x);
        }
        if (st_0) {
            st_(a.g_out + (s1 + cs + TL::P0), gs[0]);
            st2<TL::A13, TL::B13>(a.g_out + (s1 + cp), R.y, L.y);
        }
        if (st_p) {
            st_(a.g_out + (s2 + cs + TL::P2), gs[2]);
            st2<TL::A56, TL::B56>(a.g_out + (s2 + cp), R.z, L.z);
        }
        acc_m += gs[4] + (R.x + L.x);
        acc_0 += gs[0] + (R.y + L.y);
        const float acc_p = gs[2] + (R.z + L.z);
        if (st_m) a.dpsi_out[(r - 1) * nx + xc] = dpsi_of(acc_m, a);
        acc_m = acc_0;
        acc_0 = acc_p;
        s0 = s1;
        s1 = s2;
        s2 += P;
        if (s2 == a.npitch) s2 = 0;
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
    constexpr int NG = D + 1, NP = D + 5, NB = D + 1;
    const size_t smem = sizeof(T) * NG * G::WG + sizeof(float) * NP * G::WP +
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
    constexpr int D = 1;   // 8192^2 at 128 x 48: D = 1, 2, 3, 4 -> 0.915, 0.965, 0.972, 1.077 ms
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

}  // namespace

bool bulk_supported(int nx, int ny, int elem_bytes, int block_x)
{
    (void)ny;
    const int tx = elem_bytes == 2 ? bulk_tx<__half>(block_x) : bulk_tx<float>(block_x);
    if (tx <= 0) return false;
    // rows of whole tiles (every copy starts on a 16-byte boundary); a window
    // of tiles and a dpsi window wrap at most once
    return nx % kTileW == 0 && nx >= tx + 64;
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

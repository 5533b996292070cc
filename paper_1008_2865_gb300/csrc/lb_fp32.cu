// lb_fp32.cu — fused single-pass step of the two-belt Shan–Chen D2Q9 lattice
// Boltzmann method (Chibbaro et al., arXiv:1008.2865) for sm_103a, with the
// populations stored as deviations from the rest equilibrium at rho_ref.
//
// State between steps: g(t) = f(t) - w rho_ref, the streamed populations of
// state t at their own site (tiled layout, lb_internal.h), and dpsi(t) =
// psi(rho(t)) - psi(rho_ref) ([ny][nx]). One launch advances t -> t+1 and
// moves ~80 bytes per site in FP32: 36 B of g read, 36 B written, 4 B of dpsi
// read, 4 B written.
//
// Work decomposition. A CTA of BX threads owns a strip of BX-2 output
// columns and `rows` output rows; thread k sits on column x0-1+k, so the two
// edge threads are the one-column halo whose collisions the interior needs.
// The CTA marches over its rows; on lattices larger than L2, the steps march
// down in even row chunks and up in odd ones (so that the two CTAs reading a
// chunk boundary's halo row read it at about the same time, and the second
// read hits L2). For collision row r it
//   1. reads the 9 populations f_i(x, r) of its own site (one base address,
//      immediate offsets) — the loads of the next row are issued before row r
//      is computed;
//   2. forms rho, j (Eqs. 2-3) and reads psi(t) of the 25-site stencil from a
//      ring of 8 dpsi rows kept in shared memory (each dpsi row is read from
//      HBM once per CTA);
//   3. evaluates the two-belt force of Eq. FORCE in pair form, grouped by
//      |c|^2 (the constant psi_ref cancels in every antisymmetric pair);
//   4. relaxes towards the Eq. 4 equilibrium at u + F/(omega rho);
//   5. streams the post-collision values on chip (Eq. 1): the three
//      right-moving and three left-moving values go to the neighbouring
//      threads through shared memory, and every thread stores f(t+1) of its
//      own column — the speeds with c_y = -1, 0, +1 into rows r-1, r, r+1.
//      The same values, summed per speed group in a fixed order, give
//      rho(t+1); the row behind r is then complete and its dpsi(t+1) is written.
// One __syncthreads per row orders the exchange and the ring updates.
// REDUCE launches also accumulate mass and the Sec. 5 pseudo-energies of
// state t (FP32 per thread for 64 rows, then FP64) and reduce them per CTA in
// FP64; k_step_total then sums the CTA partials, row by row and then the row
// totals, in a fixed order into one trace row — deterministic for a given
// launch shape.
#include "lb_device.cuh"

#include <cmath>

namespace lbsc {
namespace {

using namespace dev;

// Resident warps per SM the register budget is cut for, the most that compile
// without spills: 40 warps (48 registers) for the plain steps (48 warps at 40
// registers spill, and run slower) and for the FP32 reduction step, whose
// energy/mass accumulators then live in shared memory (sacc; 0.900 ms at
// 8192^2 against 0.906 ms at 36 warps with register accumulators); 36 warps
// (56 registers, register accumulators) for the FP16 reduction step, which is
// bound by instruction issue and runs faster without the shared-memory traffic.
// The FP32 step is bound by the latency of its global loads.
template <typename T, bool REDUCE>
struct StepWarps {
    static constexpr bool sacc = REDUCE && sizeof(T) == 4;
    static constexpr int value = REDUCE && !sacc ? 36 : 40;
};

// Advance a row offset (row * stride, periodic over `total`) by one row in
// direction DIR (+1 down, -1 up).
template <int DIR>
__device__ __forceinline__ int step_row(int off, int stride, int total)
{
    if (DIR > 0) {
        off += stride;
        return off == total ? 0 : off;
    }
    return (off == 0 ? total : off) - stride;
}

// One CTA's tile of the step: output columns [bx (BX-2), +BX-2) and output
// rows [y0, y1) = [by rows, +rows), marched in direction DIR: down from row
// y0-1 (DIR = +1) or up from row y1 (DIR = -1). When neighbouring row chunks
// march in opposite directions, the two CTAs that read a chunk boundary's halo
// row reach it at about the same time and the second read hits L2. With
// REDUCE, v receives this thread's FP64 partial sums {E_s, E_m, E_bulk, sum of
// rho - rho_ref} of state t over its sites.
template <typename T, int BX, bool REDUCE, bool OM1, bool MIRROR, bool SACC, int DIR>
__device__ __forceinline__ void step_tile_dir(const StepArgs<T>& a, int bx, int by, double v[4],
                                              float (*win)[BX + 4], float4 (*exR)[BX + 2],
                                              float4 (*exL)[BX + 2], double* eacc, float* sacc)
{
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int N = (int)a.N;
    const int P = a.pitch, NP = a.npitch;
    const int x0 = bx * (BX - 2);
    const int y0 = by * a.rows;
    const int y1 = min(y0 + a.rows, ny);
    const int nrows = y1 - y0;
    const int txe = min(BX - 2, nx - x0);
    const bool out_col = tid >= 1 && tid <= txe;
    const int xc = wrapi(x0 - 1 + tid, nx);
    const int pc0 = wrapi(x0 - 3 + tid, nx);
    const int pc1 = wrapi(x0 - 3 + BX + (tid & 3), nx);
    using TL = Tile<T>;
    const int cs = tsingle(xc), cp = tpair<T>(xc);   // the column's single and pair offsets
    const int r0 = DIR > 0 ? y0 - 1 : y1;    // first collision row

    // ring slot q = row & 7 of dpsi row `row`; with MIRROR, slots 0..3 are
    // repeated in 8..11, so that the five rows r-2 .. r+2 sit in consecutive slots
    // from (r-2) & 7 and one base address serves the whole stencil
    for (int rr = r0 - 2; rr <= r0 + 2; ++rr) {
        const float* src = a.dpsi_in + wrapi(rr, ny) * nx;
        const float v0 = __ldg(src + pc0);
        const float v1 = tid < 4 ? __ldg(src + pc1) : 0.f;
        const int q = rr & 7;
        win[q][tid] = v0;
        if (tid < 4) win[q][BX + tid] = v1;
        if (MIRROR && q < 4) {
            win[q + 8][tid] = v0;
            if (tid < 4) win[q + 8][BX + tid] = v1;
        }
    }
    // Row offsets (row * P) of g, periodic, kept incrementally: at the top of
    // iteration r, sb, sc, sa hold rows r-DIR (behind), r, r+DIR (ahead) and oq
    // the dpsi row r+3 DIR.
    int sb = wrapi(r0 - DIR, ny) * P;
    int sc = wrapi(r0, ny) * P;
    int sa = wrapi(r0 + DIR, ny) * P;
    int oq = wrapi(r0 + 3 * DIR, ny) * nx;

    float f[9];
    load_site(f, a.g_in + sc, cs, cp);
    __syncthreads();

    // rho(t+1) of a row from its three speed groups (c_y = +1, 0, -1), summed as
    // (G+ + G0) + G- whatever the direction: hb = ahead-group sum of the behind
    // row, zb = zero-group sum of the behind row, hc = ahead-group sum of row r.
    float hb = 0.f, zb = 0.f, hc = 0.f;
    // energy/mass sums: FP32 for up to 64 rows, then added into FP64 slots of this
    // thread in shared memory (eacc[q BX + tid]), which keeps the FP64 accumulators
    // out of the registers of the row loop. With SACC the FP32 accumulators are
    // shared-memory slots too (sacc), so that the FP32 reduction step fits the
    // plain step's 48 registers and 40 warps per SM; otherwise registers.
    float es = 0.f, em = 0.f, eb = 0.f, ms = 0.f;
    if (REDUCE) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            eacc[q * BX + tid] = 0.0;
            if (SACC) sacc[q * BX + tid] = 0.f;
        }
    }

    for (int k = 0; k <= nrows + 1; ++k) {
        const int r = r0 + DIR * k;
        // ---- prefetch: dpsi row r+3 DIR and the populations of row r+DIR
        const bool more = k <= nrows;
        float pn0 = 0.f, pn1 = 0.f;
        if (more) {
            const float* src = a.dpsi_in + oq;
            pn0 = __ldg(src + pc0);
            if (tid < 4) pn1 = __ldg(src + pc1);
        }
        oq = step_row<DIR>(oq, nx, N);
        float fn[9];
        if (more) load_site(fn, a.g_in + sa, cs, cp);

        // ---- force from the dpsi(t) ring, then moments and collision
        const float* rows[5];
#pragma unroll
        for (int j = 0; j < 5; ++j)
            rows[j] = MIRROR ? &win[((r - 2) & 7) + j][tid + 2] : &win[(r - 2 + j) & 7][tid + 2];
        const float pc = a.psi_ref + rows[2][0];
        const bool out_site = out_col && k >= 1 && k <= nrows;
        float Sx, Sy;
        // the force, and on reduction steps the Sec. 5 energies of state t at (x, r)
        if (SACC) {
            es = sacc[0 * BX + tid];
            em = sacc[1 * BX + tid];
            eb = sacc[2 * BX + tid];
        }
        force_energy<REDUCE>(rows, a, Sx, Sy, out_site ? 1.f : 0.f, pc, es, em, eb);
        if (SACC) {
            sacc[0 * BX + tid] = es;
            sacc[1 * BX + tid] = em;
            sacc[2 * BX + tid] = eb;
        }
        float gs[9];
        const float d = collide<OM1>(f, -pc * Sx, -pc * Sy, a, gs);
        if (SACC) sacc[3 * BX + tid] = fmaf(out_site ? 1.f : 0.f, d, sacc[3 * BX + tid]);
        else if (REDUCE) ms = fmaf(out_site ? 1.f : 0.f, d, ms);

        // ---- exchange post-collision values with the neighbouring columns
        exR[r & 1][tid + 1] = make_float4(gs[8], gs[1], gs[5], 0.f);
        exL[r & 1][tid + 1] = make_float4(gs[7], gs[3], gs[6], 0.f);
        if (more) {
            const int q = (r + 3 * DIR) & 7;
            win[q][tid] = pn0;
            if (tid < 4) win[q][BX + tid] = pn1;
            if (MIRROR && q < 4) {
                win[q + 8][tid] = pn0;
                if (tid < 4) win[q + 8][BX + tid] = pn1;
            }
        }
        // ---- f(t+1) = f*(x - c_i) (Eq. 1) for the own column: the speeds with
        // c_y = -DIR land in the behind row, c_y = 0 in row r, c_y = +DIR in the
        // ahead row. The own-column speeds are stored now, the six from the
        // neighbouring columns after the barrier.
        const int rb = r - DIR;
        // rows r - DIR, r, r + DIR are output rows for k >= 2, 1 <= k <= nrows, k < nrows
        const bool st_b = out_col && k >= 2;
        const bool st_0 = out_site;
        const bool st_a = out_col && k < nrows;
        constexpr int ib = DIR > 0 ? 4 : 2, ia = DIR > 0 ? 2 : 4;   // own speeds with c_y = -DIR, +DIR
        constexpr int ob = DIR > 0 ? TL::P4 : TL::P2, oa = DIR > 0 ? TL::P2 : TL::P4;
        if (st_b) st_(a.g_out + (sb + cs + ob), gs[ib]);
        if (st_0) st_(a.g_out + (sc + cs + TL::P0), gs[0]);
        if (st_a) st_(a.g_out + (sa + cs + oa), gs[ia]);
        const float own_b = gs[ib], own_0 = gs[0], own_a = gs[ia];
        __syncthreads();
        const float4 R = exR[r & 1][tid];       // from column x-1: speeds 8, 1, 5
        const float4 L = exL[r & 1][tid + 2];   // from column x+1: speeds 7, 3, 6
        const float Rb = DIR > 0 ? R.x : R.z, Lb = DIR > 0 ? L.x : L.z;
        const float Ra = DIR > 0 ? R.z : R.x, La = DIR > 0 ? L.z : L.x;
        // the two values from the neighbouring columns form one pair of the layout:
        // behind row (7, 8) = (L, R) marching down, (5, 6) = (R, L) marching up;
        // row r (1, 3) = (R, L); ahead row (5, 6) = (R, L) down, (7, 8) = (L, R) up
        if (st_b) {
            if (DIR > 0) st2<TL::A78, TL::B78>(a.g_out + (sb + cp), Lb, Rb);
            else st2<TL::A56, TL::B56>(a.g_out + (sb + cp), Rb, Lb);
        }
        if (st_0) st2<TL::A13, TL::B13>(a.g_out + (sc + cp), R.y, L.y);
        if (st_a) {
            if (DIR > 0) st2<TL::A56, TL::B56>(a.g_out + (sa + cp), Ra, La);
            else st2<TL::A78, TL::B78>(a.g_out + (sa + cp), La, Ra);
        }
        const float gb = own_b + (Rb + Lb);     // behind-group sum into row r-DIR
        const float g0 = own_0 + (R.y + L.y);   // zero-group sum of row r
        const float ga = own_a + (Ra + La);     // ahead-group sum into row r+DIR
        // rho(t+1) of the behind row is complete: (G+ + G0) + G-
        if (st_b) {
            const float rho1 = DIR > 0 ? (hb + zb) + gb : (gb + zb) + hb;
            a.dpsi_out[rb * nx + xc] = dpsi_of(rho1, a);
        }
        hb = hc;
        zb = g0;
        hc = ga;
        sb = sc;
        sc = sa;
        sa = step_row<DIR>(sa, P, NP);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fn[i];
        if (REDUCE) {
            if ((k & 63) == 63) {
                if (SACC) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        eacc[q * BX + tid] += sacc[q * BX + tid];
                        sacc[q * BX + tid] = 0.f;
                    }
                } else {
                    eacc[0 * BX + tid] += es;
                    eacc[1 * BX + tid] += em;
                    eacc[2 * BX + tid] += eb;
                    eacc[3 * BX + tid] += ms;
                    es = em = eb = ms = 0.f;
                }
            }
        }
    }

    if (REDUCE) {
        if (SACC) {
            es = sacc[0 * BX + tid];
            em = sacc[1 * BX + tid];
            eb = sacc[2 * BX + tid];
            ms = sacc[3 * BX + tid];
        }
        v[0] = eacc[0 * BX + tid] + es;
        v[1] = eacc[1 * BX + tid] + em;
        v[2] = eacc[2 * BX + tid] + eb;
        v[3] = eacc[3 * BX + tid] + ms;
    }
}

// The tile of chunk `by`. With ALTERNATE and `alternate` (marches_alternate:
// states larger than L2), the tile marches down in even chunks and up in odd
// ones, otherwise down. Fields do not depend on the direction (each site's
// arithmetic, and the order of the rho(t+1) sum, are the same either way); the
// per-thread energy and mass sums of a reduction step do, so a batch replica
// takes the direction its lattice takes alone, and its trace stays
// bit-identical to that run's. MIRROR: the ring's stencil rows from one base
// address (single-lattice plain steps; the reduction and batch kernels keep
// the 8-slot ring, measured faster there).
template <typename T, int BX, bool REDUCE, bool OM1, bool ALTERNATE, bool MIRROR, bool SACC>
__device__ __forceinline__ void step_tile(const StepArgs<T>& a, int bx, int by, double v[4],
                                          double* eacc, bool alternate = true)
{
    __shared__ float win[MIRROR ? 12 : 8][BX + 4];   // dpsi(t) rows, slot = row & 7
    __shared__ float4 exR[2][BX + 2];        // right-moving f*: speeds 8, 1, 5 (cy = -1, 0, +1)
    __shared__ float4 exL[2][BX + 2];        // left-moving f*: speeds 7, 3, 6
    __shared__ float sacc[SACC ? 4 * BX : 1];      // FP32 energy/mass slots of the threads
    if (ALTERNATE && alternate && (by & 1))
        step_tile_dir<T, BX, REDUCE, OM1, MIRROR, SACC, -1>(a, bx, by, v, win, exR, exL, eacc, sacc);
    else
        step_tile_dir<T, BX, REDUCE, OM1, MIRROR, SACC, +1>(a, bx, by, v, win, exR, exL, eacc, sacc);
}

template <typename T, int BX, bool REDUCE, bool OM1>
__global__ void __launch_bounds__(BX, StepWarps<T, REDUCE>::value * 32 / BX)
    k_step(const StepArgs<T> a, bool alternate)
{
    __shared__ double eacc[REDUCE ? 4 * BX : 1];   // FP64 energy/mass slots, then the block sums
    double v[4];
    step_tile<T, BX, REDUCE, OM1, true, !REDUCE, StepWarps<T, REDUCE>::sacc>(a, blockIdx.x, blockIdx.y,
                                                                              v, eacc, alternate);
    if (REDUCE) {
        // the CTA partial; k_step_total forms the grid sum and the trace row
        block_sum4<BX>(v, eacc);
        if (threadIdx.x == 0) {
            double* p = a.partials + 4 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
#pragma unroll
            for (int k = 0; k < 4; ++k) p[k] = v[k];
        }
    }
}

// The grid sum of a reduction step of k_step (grid nbx x nby, launched after
// it on the same stream): one CTA per CTA row, row_then_total, then the trace
// row of state t. The row totals follow the CTA partials in a.partials.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_step_total(const StepArgs<T> a, int nbx)
{
    __shared__ double red[4 * NT];
    const int nby = gridDim.x;
    double* rows = a.partials + 4 * (size_t)nbx * nby;
    double w[4];
    if (row_then_total<NT>(a.partials, nbx, nby, blockIdx.x, rows, a.counter, w, red)) {
        const double mass = (double)a.N * (double)a.rho_ref + w[3];
        write_trace_row(a.trace, a.trace_count, a.t, mass, w[0], w[1], w[2]);
        if (!isfinite(mass) || !isfinite(w[0]) || !isfinite(w[1])) atomicOr(a.err, 2);
    }
}

// ---------------------------------------------------------------- batches
// Several lattices (replicas, each with its own size and couplings) advanced by
// one launch: a persistent grid strides over a work list of tiles, each tile
// = (replica, strip, row chunk) of that replica's own launch shape, and runs
// exactly the per-tile code of k_step. The replica's arguments are staged in
// shared memory once per tile. A tile marches as k_step marches it (tl.w: the
// replica alternates; ALTERNATE: some replica does, and its kernels get a
// 36-warp register budget). With REDUCE each tile's CTA partial (the same block
// sum k_step forms) goes to tile_partials; k_batch_reduce then sums a
// replica's partials in the order k_step_total uses, so a replica's fields
// and trace are bit-identical to running it alone with the same shape.
// (Measured on the 96-replica sweep and not kept: tiles handed out by an
// atomic counter, 1.2% slower; alternating march directions for replicas that
// fit in L2, no gain.)
template <typename T, int BX, bool REDUCE, bool OM1, bool ALTERNATE>
__global__ void __launch_bounds__(BX, (REDUCE ? 28 : ALTERNATE ? 36 : 40) * 32 / BX)
    k_step_batch(const StepArgs<T>* __restrict__ args, const int4* __restrict__ tiles, int ntiles,
                 double* __restrict__ tile_partials)
{
    __shared__ StepArgs<T> sa;
    __shared__ int sa_rep;                          // replica whose arguments sa holds
    __shared__ double eacc[REDUCE ? 4 * BX : 1];   // FP64 energy/mass slots, then the block sum
    static_assert(sizeof(StepArgs<T>) % 4 == 0, "arguments are copied as 4-byte words");
    // (measured on the 96-replica sweep: the warp-wide copy 1.2% faster than one
    // thread copying the struct; CTAs taking consecutive items instead of every
    // gridDim.x-th, so that a replica's arguments would stay in sa, 31% slower)
    if (threadIdx.x == 0) sa_rep = -1;
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const int4 tl = tiles[k];                   // (replica, strip, chunk, alternate)
        __syncthreads();                            // previous tile done with sa and smem rings
        if (threadIdx.x < 32 && tl.x != sa_rep) {   // warp 0 copies the arguments, 4 B a lane
            const int* src = reinterpret_cast<const int*>(args + tl.x);
            int* dst = reinterpret_cast<int*>(&sa);
            for (int w = threadIdx.x; w < (int)(sizeof(StepArgs<T>) / 4); w += 32)
                dst[w] = __ldg(src + w);
            __syncwarp();
            if (threadIdx.x == 0) sa_rep = tl.x;
        }
        __syncthreads();
        double v[4];
        step_tile<T, BX, REDUCE, OM1, ALTERNATE, false, false>(sa, tl.y, tl.z, v, eacc, tl.w != 0);
        if (REDUCE) {
            block_sum4<BX>(v, eacc);
            if (threadIdx.x == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) tile_partials[4 * (size_t)k + q] = v[q];
            }
        }
    }
}

// The grid sums of a batch's reduction step: one CTA per (replica, row chunk)
// (rowmap), row_then_total over the replica's tile partials (tiles first ..
// first + ntiles - 1, in the replica's own CTA order), exactly as k_step_total
// sums k_step's CTA partials; then one trace row (t = rows already written x
// trace_every) into the replica's trace ring.
template <int NT>
__global__ void __launch_bounds__(NT)
    k_batch_reduce(double* __restrict__ tile_partials, const BatchRep* __restrict__ reps,
                   const int2* __restrict__ rowmap, int trace_every)
{
    __shared__ double red[4 * NT];
    const int2 m = rowmap[blockIdx.x];            // (replica, row chunk)
    const BatchRep r = reps[m.x];
    const int nty = r.ntiles / r.ntx;
    double w[4];
    if (row_then_total<NT>(tile_partials + 4 * (size_t)r.first_tile, r.ntx, nty, m.y,
                           tile_partials + 4 * (size_t)r.first_row, r.counter, w, red)) {
        const double mass = (double)r.N * r.rho_ref + w[3];
        const long long t = (long long)(*r.trace_count) * trace_every;
        write_trace_row(r.trace, r.trace_count, t, mass, w[0], w[1], w[2]);
        if (!isfinite(mass) || !isfinite(w[0]) || !isfinite(w[1])) atomicOr(r.err, 2);
    }
}

// ---------------------------------------------------------------- helpers

// The helpers below cover the lattice row by row (blockIdx.y strides over rows,
// the threads of a block over the columns of a row), so that no site index is
// divided by nx.
template <typename T>
__global__ void __launch_bounds__(256) k_delta_init(T* __restrict__ g, float* __restrict__ dpsi,
                                                    const double* __restrict__ rho, int nx,
                                                    int ny, double rho_ref, double inv_rho0,
                                                    float cpsi)
{
    const int pitch = g_pitch(nx);
    const float w0 = 4.f / 9.f, w1 = 1.f / 9.f, w2 = 1.f / 36.f;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        for (int x = blockIdx.x * 256 + threadIdx.x; x < nx; x += gridDim.x * 256) {
            const size_t s = (size_t)y * nx + x;
            // f_i(x, 0) = w_i rho_init(x): the fluid at rest, stored as w_i (rho - rho_ref)
            const double d = rho[s] - rho_ref;
            const float df = (float)d;
            T* row = g + (size_t)y * pitch;
            using TL = Tile<T>;
            const int cs = tsingle(x), cp = tpair<T>(x);
            st_(row + cs + TL::P0, w0 * df);
            st_(row + cs + TL::P2, w1 * df);
            st_(row + cs + TL::P4, w1 * df);
            st2<TL::A13, TL::B13>(row + cp, w1 * df, w1 * df);
            st2<TL::A56, TL::B56>(row + cp, w2 * df, w2 * df);
            st2<TL::A78, TL::B78>(row + cp, w2 * df, w2 * df);
            dpsi[s] = cpsi * expm1f((float)(-d * inv_rho0));
        }
    }
}

// rho = rho_ref + sum_i g_i and u = sum_i c_i g_i / rho (Eqs. 2-3): the sums in
// FP32 in the order of the step's moments, u by an IEEE FP32 division, stored as
// doubles (rho in FP64: rho_ref + d).
template <typename T>
__global__ void __launch_bounds__(256) k_delta_fields(const T* __restrict__ g, int nx, int ny,
                                                      double rho_ref, double* __restrict__ rho,
                                                      double* __restrict__ ux,
                                                      double* __restrict__ uy)
{
    const int pitch = g_pitch(nx);
    const float rref = (float)rho_ref;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        for (int x = blockIdx.x * 256 + threadIdx.x; x < nx; x += gridDim.x * 256) {
            float f[9];
            load_site_xy(f, g, pitch, x, y);
            const float d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
            const float r = rref + d;
            const size_t s = (size_t)y * nx + x;
            if (rho) rho[s] = rho_ref + (double)d;
            if (ux) ux[s] = (double)__fdiv_rn(jx, r);
            if (uy) uy[s] = (double)__fdiv_rn(jy, r);
        }
    }
}

// lb_energy: the Sec. 5 sums and the mass of state t. Row by row (blockIdx.y
// strides over rows, the threads of a block over columns; a column away from
// the periodic x edges reads its stencil rows with immediate offsets). The
// class sums of the psi deviations (|c|^2 = 1, 2, 4, 5, 8) and the site's
// deviation sum are FP32 sums of 4-9 FP32 values (within a few units of
// 2^-24 of their magnitude, ~1e-9 here); the products with the couplings and
// every accumulation are FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_delta_energy(const T* __restrict__ g,
                                                      const float* __restrict__ dpsi,
                                                      const StepArgs<T> a, double* out4)
{
    const int nx = a.nx, ny = a.ny;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const double pr = a.psi_ref;
    const double K0 = a.K0, K1 = a.K1, K2 = a.K2, K4 = a.K4, K5 = a.K5, K8 = a.K8;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const float* rw[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) rw[k] = dpsi + (size_t)wrapi(y + k - 2, ny) * nx;
        for (int x = blockIdx.x * 256 + threadIdx.x; x < nx; x += gridDim.x * 256) {
            float q[5][5];          // q[k][m] = dpsi(x + m - 2, y + k - 2)
            if (x >= 2 && x < nx - 2) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
#pragma unroll
                    for (int m = 0; m < 5; ++m) q[k][m] = __ldg(rw[k] + x + m - 2);
                }
            } else {
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    const int xx = wrapi(x + m - 2, nx);
#pragma unroll
                    for (int k = 0; k < 5; ++k) q[k][m] = __ldg(rw[k] + xx);
                }
            }
            const float S1 = (q[2][3] + q[2][1]) + (q[3][2] + q[1][2]);
            const float S2 = (q[3][3] + q[3][1]) + (q[1][3] + q[1][1]);
            const float S4 = (q[2][4] + q[2][0]) + (q[4][2] + q[0][2]);
            const float S5 = ((q[3][4] + q[3][0]) + (q[1][4] + q[1][0])) +
                             ((q[4][3] + q[4][1]) + (q[0][3] + q[0][1]));
            const float S8 = (q[4][4] + q[4][0]) + (q[0][4] + q[0][0]);
            const double pc = pr + (double)q[2][2];
            const double b1 = K0 * pc + K1 * (4 * pr + (double)S1) + K2 * (4 * pr + (double)S2);
            const double b2 =
                K4 * (4 * pr + (double)S4) + K5 * (8 * pr + (double)S5) + K8 * (4 * pr + (double)S8);
            v[0] += 0.5 * pc * b1;
            v[1] += 0.5 * pc * b2;
            v[2] += (double)a.half_A1 * pc * pc;
            float f[9];
            load_site_xy(f, g, a.pitch, x, y);
            const float d =
                ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            v[3] += (double)d;
        }
    }
    if (last_block_total<256>(v, a.partials, a.counter, gridDim.x * gridDim.y)) {
        out4[0] = v[0];
        out4[1] = v[1];
        out4[2] = v[2];
        out4[3] = (double)a.N * (double)a.rho_ref + v[3];
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
    const bool om1 = a.omega == 1.0f;
    const bool alt = marches_alternate(a.N);
    if (reduce) {
        if (om1) k_step<T, BX, true, true><<<grid, BX, 0, s>>>(a, alt);
        else k_step<T, BX, true, false><<<grid, BX, 0, s>>>(a, alt);
        if (cudaPeekAtLastError() != cudaSuccess) return cudaGetLastError();
        k_step_total<T, BX><<<grid.y, BX, 0, s>>>(a, (int)grid.x);
    } else {
        if (om1) k_step<T, BX, false, true><<<grid, BX, 0, s>>>(a, alt);
        else k_step<T, BX, false, false><<<grid, BX, 0, s>>>(a, alt);
    }
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

template <typename T, int BX>
cudaError_t launch_batch_bx(const BatchLaunch<T>& b, bool reduce, cudaStream_t s)
{
    auto pick = [&](auto kern) -> cudaError_t {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BX, 0);
        if (e != cudaSuccess) return e;
        long long grid = (long long)per_sm * b.num_sms;
        if (grid > b.ntiles) grid = b.ntiles;
        if (grid < 1) grid = 1;
        kern<<<(unsigned int)grid, BX, 0, s>>>(b.args, b.tiles, b.ntiles, b.tile_partials);
        return cudaGetLastError();
    };
    cudaError_t e;
    if (b.alternate) {
        if (reduce)
            e = b.om1 ? pick(k_step_batch<T, BX, true, true, true>)
                      : pick(k_step_batch<T, BX, true, false, true>);
        else
            e = b.om1 ? pick(k_step_batch<T, BX, false, true, true>)
                      : pick(k_step_batch<T, BX, false, false, true>);
    } else {
        if (reduce)
            e = b.om1 ? pick(k_step_batch<T, BX, true, true, false>)
                      : pick(k_step_batch<T, BX, true, false, false>);
        else
            e = b.om1 ? pick(k_step_batch<T, BX, false, true, false>)
                      : pick(k_step_batch<T, BX, false, false, false>);
    }
    if (e != cudaSuccess || !reduce) return e;
    k_batch_reduce<BX><<<b.nrows, BX, 0, s>>>(b.tile_partials, b.reps, b.rowmap, b.trace_every);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch(const BatchLaunch<T>& b, bool reduce, cudaStream_t s)
{
    switch (b.block_x) {
    case 64: return launch_batch_bx<T, 64>(b, reduce, s);
    case 96: return launch_batch_bx<T, 96>(b, reduce, s);
    case 128: return launch_batch_bx<T, 128>(b, reduce, s);
    case 192: return launch_batch_bx<T, 192>(b, reduce, s);
    case 256: return launch_batch_bx<T, 256>(b, reduce, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fp32_batch_step(const BatchLaunch<float>& b, bool reduce, cudaStream_t s)
{
    return launch_batch<float>(b, reduce, s);
}

cudaError_t fp16_batch_step(const BatchLaunch<__half>& b, bool reduce, cudaStream_t s)
{
    return launch_batch<__half>(b, reduce, s);
}

static int helper_grid(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

// Grid of the row-wise helpers: enough blocks per row to cover it, all rows
// (grid-stride beyond 65535).
static dim3 row_grid(int nx, int ny)
{
    const int bx = (nx + 255) / 256;
    return dim3((unsigned)(bx < 64 ? bx : 64), (unsigned)(ny < 65535 ? ny : 65535));
}

template <typename T>
cudaError_t delta_init(T* g, float* dpsi, const double* rho_init, int nx, int ny, double rho_ref,
                       double rho0, cudaStream_t s)
{
    const float cpsi = (float)(-std::sqrt(rho0) * std::exp(-rho_ref / rho0));
    k_delta_init<T><<<row_grid(nx, ny), 256, 0, s>>>(g, dpsi, rho_init, nx, ny, rho_ref,
                                                     1.0 / rho0, cpsi);
    return cudaGetLastError();
}

template <typename T>
cudaError_t delta_fields(const T* g, int nx, int ny, double rho_ref, double* rho, double* ux,
                         double* uy, cudaStream_t s)
{
    k_delta_fields<T><<<row_grid(nx, ny), 256, 0, s>>>(g, nx, ny, rho_ref, rho, ux, uy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t delta_energy(const T* g, const float* dpsi, int nx, int ny, const StepArgs<T>& a,
                         double* out4, double* partials, unsigned int* counter, cudaStream_t s)
{
    StepArgs<T> b = a;
    b.partials = partials;
    b.counter = counter;
    // at most 152 x 16 CTAs (the state's partial buffer holds at least that many)
    int bx = (nx + 255) / 256;
    if (bx > 32) bx = 32;
    int by = 152 * 16 / bx;
    if (by > ny) by = ny;
    k_delta_energy<T><<<dim3(bx, by), 256, 0, s>>>(g, dpsi, b, out4);
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

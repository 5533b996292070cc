// lb_internal.h — declarations shared by the translation units of liblbsc.so
// (state layout, launch helpers). Not installed; the public interface is
// include/lb.h.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lb.h"

namespace lbsc {

// NVTX range for the duration of an ABI call (visible in Nsight timelines).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Makes `dev` the calling thread's current device for the duration of an ABI
// call and gives the caller's current device back on return, so that a call on
// a state of another device does not move the caller's thread (a torch caller
// working on device 1 stays on device 1). ok is false if the switch failed.
struct DeviceScope {
    int prev = -1;
    bool ok = false;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    ~DeviceScope()
    {
        int now = -1;
        if (prev >= 0 && (cudaGetDevice(&now) != cudaSuccess || now != prev)) {
            cudaSetDevice(prev);
            cudaGetLastError();
        }
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

constexpr int kTraceCap = 65536;     // rows kept in the device trace ring
constexpr int kTraceCols = 5;        // (t, mass, E_s, E_m, E_bulk)

// Couplings of the 24 links grouped by |c|^2 (Eq. FORCE with Table 1):
//   K1 = G1/9 + 4 G2/63, K2 = G1/36 + 4 G2/135, K4 = G2/180,
//   K5 = 2 G2/945, K8 = G2/15120; K0 = G1 4/9 + G2 p_s0 is the rest coupling
//   of the belt-1 energy (p_s0 = 247/420 from Eq. weights_1).
struct Couplings {
    double K0, K1, K2, K4, K5, K8;
};
Couplings couplings(double G1, double G2);

// Populations of an FP32 / FP16 state ("tiled" layout): rows of 32-column
// tiles of 288 elements; the tile of column x in row y starts at
//   y * g_pitch(nx) + (x / 32) * 288.
// FP32 ("paired"): a tile holds its 32 sites' populations 0, 2 and 4 as three
// runs of 32 (elements 0-31, 32-63, 64-95, at x % 32 within each run), then the
// pairs (1, 3), (5, 6) and (7, 8) as three runs of 32 pairs (elements 96-159,
// 160-223, 224-287, the pair of column x % 32 at 2 (x % 32), first member
// first). The pairs are the populations a thread of the fused step always
// writes together (the two that arrive from the neighbouring columns in one
// row), so each pair is one 8-byte access.
// FP16: the same element layout, so a pair is one 4-byte access (8192^2:
// 92.6k against 91.5k MLUPS with nine runs of 32).
// Columns past nx in the last tile of a row are padding (zero, never read by a
// step).
constexpr int kTileW = 32;
constexpr int kTileElems = 9 * kTileW;
__host__ __device__ inline int g_pitch(int nx) { return kTileElems * ((nx + kTileW - 1) / kTileW); }
__host__ __device__ inline long long g_elems(int nx, int ny) { return (long long)ny * g_pitch(nx); }

// Arguments of the fused FP32 step (deviation storage, see lb.h LB_FP32).
template <typename T>
struct StepArgs {
    const T* __restrict__ g_in;      // tiled f(t) - w rho_ref: populations of state t
    T* __restrict__ g_out;           // tiled f(t+1) - w rho_ref
    const float* __restrict__ dpsi_in;   // [ny][nx] psi(t) - psi_ref
    float* __restrict__ dpsi_out;        // [ny][nx] psi(t+1) - psi_ref
    int nx, ny;
    int rows;                        // output rows per CTA
    long long N;                     // nx*ny
    int pitch;                       // g_pitch(nx): elements per row of g
    int npitch;                      // g_elems(nx, ny): elements per g buffer
    float omega, omc, inv_omega;     // omega, 1-omega, 1/omega
    float w0, w1, w2;                // D2Q9 weights
    float K1, K2, K4, K5, K8;        // force couplings
    float rho_ref, psi_ref, cpsi, inv_rho0;  // dpsi = cpsi * expm1(-(rho-rho_ref)/rho0)
    // energy/mass reduction (REDUCE launches only)
    float K0, half_A1;
    double* partials;                // [gridDim.x*gridDim.y + gridDim.y][4]: CTA, row totals
    unsigned int* counter;           // arrival counter of the grid sums (zero between uses)
    double* trace;                   // [kTraceCap][5] ring
    int* trace_count;                // rows ever written
    long long t;                     // time level of the reduced state
    // bounded waits of the bulk-copy kernel
    int* err;                        // error flags: 1 a wait ran out, 2 a reduction was not finite
    long long wait_cycles;           // clock limit of one wait
    int skip_unit0;                  // test hook: the first row unit's barrier is armed, no copy issued
};

// Output rows per CTA accepted by lb_set_launch / lb_batch_set_launch.
constexpr int kMinRows = 4;
constexpr int kMaxRows = 4096;

// Launchers (lb_fp32.cu). All return the launch's cudaError_t.
struct Fp32Launch {
    int block_x;   // threads per CTA
    int rows;      // output rows per CTA
    int pipeline;  // 0: register prefetch (any shape), 1: bulk-copy rings (nx % 32 == 0)
};
int fp32_grid_blocks(int nx, int ny, Fp32Launch L);
cudaError_t fp32_step(const StepArgs<float>& a, Fp32Launch L, bool reduce, cudaStream_t s);
cudaError_t fp16_step(const StepArgs<__half>& a, Fp32Launch L, bool reduce, cudaStream_t s);
// Whether the steps of a lattice of n sites march in alternating directions
// (down in even row chunks, up in odd ones): only when its state does not fit in
// L2 (measured: 2% slower at 1024^2, faster from 2048^2 on). A batch replica
// follows the same rule as the lattice run alone.
inline bool marches_alternate(long long n) { return n * 80 > (128LL << 20); }

// Batches (lb_fp32.cu kernels, lb_batch.cu host code): one launch advances many
// replicas. tiles[k] = (replica, strip, chunk, alternate), grouped by replica in
// each replica's own CTA order; reps[r] locates replica r's tiles and its trace ring.
struct BatchRep {
    int first_tile, ntiles;
    int ntx;                   // tiles per row chunk
    int first_row;             // slot of the replica's row totals (after all tile partials)
    unsigned int* counter;     // the replica's arrival counter (its state's, zero between uses)
    long long N;
    double rho_ref;
    double* trace;
    int* trace_count;
    int* err;                  // the replica's error flags
};
template <typename T>
struct BatchLaunch {
    const StepArgs<T>* args;   // [nreps] arguments of this step's parity
    const int4* tiles;
    int ntiles;
    double* tile_partials;     // [ntiles + row chunks of all replicas][4]
    const BatchRep* reps;
    int nreps;
    const int2* rowmap;        // [nrows] (replica, row chunk) of each reduction CTA
    int nrows;
    int block_x;
    bool om1;                  // every replica has omega == 1
    int trace_every;
    int num_sms;
    bool alternate;            // some replica marches in alternating directions
};
cudaError_t fp32_batch_step(const BatchLaunch<float>& b, bool reduce, cudaStream_t s);
cudaError_t fp16_batch_step(const BatchLaunch<__half>& b, bool reduce, cudaStream_t s);
// bulk-copy pipelined step (lb_bulk.cu)
bool bulk_supported(int nx, int ny, int elem_bytes, int block_x);
int bulk_grid_blocks(int nx, int ny, int elem_bytes, Fp32Launch L);
cudaError_t fp32_step_bulk(const StepArgs<float>& a, Fp32Launch L, bool reduce, cudaStream_t s);
cudaError_t fp16_step_bulk(const StepArgs<__half>& a, Fp32Launch L, bool reduce, cudaStream_t s);
template <typename T>
cudaError_t delta_init(T* g, float* dpsi, const double* rho_init, int nx, int ny,
                       double rho_ref, double rho0, cudaStream_t s);
template <typename T>
cudaError_t delta_fields(const T* g, int nx, int ny, double rho_ref, double* rho, double* ux,
                         double* uy, cudaStream_t s);
template <typename T>
cudaError_t delta_energy(const T* g, const float* dpsi, int nx, int ny, const StepArgs<T>& a,
                         double* out4, double* partials, unsigned int* counter, cudaStream_t s);

// Input checks and sums (lb_fp32.cu): out[0] = sum rho, flag |= 1 if any rho is
// not finite or <= 0.
cudaError_t rho_check_sum(const double* rho, long long n, double* partials, unsigned int* counter,
                          double* out_sum, int* flag, cudaStream_t s);

// FP64 parity path (lb_fp64.cu, compiled without FMA contraction).
struct Fp64Args {
    double* f_in;        // [9][ny][nx] populations of state t (after streaming)
    double* f_out;       // [9][ny][nx] populations of state t+1
    double* psi;         // [ny][nx] psi(t)
    double* rho;         // [ny][nx] rho(t)
    int nx, ny;
    double omega, G1, G2, rho0;
};
cudaError_t fp64_init(double* f, const double* rho_init, int nx, int ny, cudaStream_t s);
cudaError_t fp64_psi(const Fp64Args& a, cudaStream_t s);
cudaError_t fp64_collide_stream(const Fp64Args& a, cudaStream_t s);
cudaError_t fp64_energy(const Fp64Args& a, double* partials, unsigned int* counter,
                        double* out4, double* trace, int* trace_count, long long t,
                        cudaStream_t s);
cudaError_t fp64_fields(const double* f, int nx, int ny, double* rho, double* ux, double* uy,
                        cudaStream_t s);
cudaError_t fp64_exp_cr(const double* x, double* y, long long n, cudaStream_t s);

}  // namespace lbsc

// The state behind the opaque lb_state* of the C ABI (lb_api.cu owns its
// lifetime; lb_batch.cu drives several of them with one launch per step).
struct lb_state {
    lb_params p;
    cudaStream_t stream = nullptr;
    long long t = 0;
    bool poisoned = false;
    long long N = 0;
    // FP32 / FP16 deviation storage (g tiled, lbsc::g_elems elements each)
    void* g[2] = {nullptr, nullptr};
    float* dpsi[2] = {nullptr, nullptr};
    int cur = 0;
    double rho_ref = 0.0;
    lbsc::Fp32Launch launch{128, 64, 0};
    int* err = nullptr;            // set by a kernel whose bounded wait ran out
    long long wait_cycles = 2000000000LL;
    int skip_unit0 = 0;            // test hook of lb_set_wait_limit
    // FP64 parity storage
    double* f64[2] = {nullptr, nullptr};
    double* psi64 = nullptr;
    double* rho64 = nullptr;
    // reductions, trace, scratch
    double* partials = nullptr;
    size_t partials_cap = 0;       // number of 4-double partials
    int max_cta_rows = 0;          // CTA rows of the step's grid at most (kMinRows-row chunks)
    unsigned int* counter = nullptr;
    double* trace = nullptr;
    int* trace_count = nullptr;
    double* res = nullptr;         // 4 doubles of results
    int* flag = nullptr;
    double* field_tmp = nullptr;   // N doubles, allocated on the first lb_fields into pageable host memory
    // every device buffer of the state, with a guard region on each side
    struct Alloc {
        void* base;
        size_t bytes;
    };
    std::vector<Alloc> allocs;
};

namespace lbsc {
constexpr size_t kGuardBytes = 256;              // guard region on each side of a buffer
constexpr unsigned char kGuardByte = 0xA5;       // the pattern the guards hold
// Allocate `bytes` for a state with guards on both sides (pattern written on
// the state's stream); returns the usable pointer or nullptr.
void* state_alloc(lb_state* s, size_t bytes);
}  // namespace lbsc

namespace lbsc {
template <typename T>
StepArgs<T> state_args(const lb_state* s, int cur);   // arguments of a step from buffers `cur`
size_t elem_size(lb_precision p);
// Where a kernel can read or write a double array directly: device memory as it
// is, pinned host memory through its device alias; nullptr for pageable memory.
double* device_view(double* p);
// Objective sums of lb_adjoint's terminal kernel for an FP32/FP16 state
// (lb_adjoint.cu): acc[0] = E_s + E_m of the current state, acc[1] = sum (rho -
// tgt)^2, acc[2..3] the explicit dE/dG1, dE/dG2; tgt is device memory.
cudaError_t objective_delta(const lb_state* s, const double* tgt, double* acc, cudaStream_t st);
// *out = sum (rho - tgt)^2 over n doubles in device memory, deterministic.
cudaError_t misfit64(const double* rho, const double* tgt, long long n, double* partials,
                     unsigned int* counter, double* out, cudaStream_t st);
}  // namespace lbsc

// lb_batch.cu — the lb_batch_* entry points of include/lb.h: many independent
// lattices (replicas of possibly different sizes and couplings, e.g. a G2
// sweep with distinct seeds) advanced together, one launch per step over a
// work list of all replicas' tiles (k_step_batch in lb_fp32.cu), replayed
// from a CUDA graph of one trace period. Each replica is an lb_state, so
// energies, fields and traces reuse the single-lattice code.
#include <algorithm>
#include <new>
#include <vector>

#include "lb_internal.h"

using namespace lbsc;

struct lb_batch {
    std::vector<lb_state*> reps;
    int device = 0;
    cudaStream_t stream = nullptr;
    lb_precision prec = LB_FP32;
    int trace_every = 0;
    int block_x = 128, rows = 32;
    bool use_graph = true;
    bool om1 = true;
    bool alternate = false;   // some replica marches in alternating directions
    int num_sms = 1;
    long long t = 0;
    int cur = 0;
    bool poisoned = false;
    // device tables
    void* d_args[2] = {nullptr, nullptr};   // StepArgs<T>[nreps] for buffers 0 and 1
    int4* d_tiles = nullptr;
    int ntiles = 0;
    int2* d_rowmap = nullptr;   // (replica, row chunk) of each grid-sum CTA
    int nrows = 0;
    double* d_partials = nullptr;
    BatchRep* d_reps = nullptr;
    // graph of one period of steps, starting at t % period == 0
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int period = 0;
};

namespace {

void free_tables(lb_batch* b)
{
    void* ptrs[] = {b->d_args[0], b->d_args[1], b->d_tiles, b->d_partials, b->d_reps,
                    b->d_rowmap};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    b->d_args[0] = b->d_args[1] = nullptr;
    b->d_tiles = nullptr;
    b->d_rowmap = nullptr;
    b->d_partials = nullptr;
    b->d_reps = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaGetLastError();
}

template <typename T>
bool upload_args(lb_batch* b)
{
    for (int c = 0; c < 2; ++c) {
        std::vector<StepArgs<T>> a(b->reps.size());
        for (size_t r = 0; r < b->reps.size(); ++r) {
            a[r] = state_args<T>(b->reps[r], c);
            a[r].rows = b->rows;
        }
        if (cudaMalloc(&b->d_args[c], sizeof(StepArgs<T>) * a.size()) != cudaSuccess ||
            cudaMemcpy(b->d_args[c], a.data(), sizeof(StepArgs<T>) * a.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
    }
    return true;
}

// Work list: replica by replica, each in its own CTA order (chunk-major).
lb_status build_tables(lb_batch* b)
{
    free_tables(b);
    std::vector<int4> tiles;
    std::vector<BatchRep> info;
    std::vector<int2> rowmap;
    int nrows_total = 0;
    for (size_t r = 0; r < b->reps.size(); ++r) {
        const lb_state* s = b->reps[r];
        const int ntx = (s->p.nx + b->block_x - 3) / (b->block_x - 2);
        const int nty = (s->p.ny + b->rows - 1) / b->rows;
        BatchRep ri;
        ri.first_tile = (int)tiles.size();
        ri.ntiles = ntx * nty;
        ri.ntx = ntx;
        ri.first_row = nrows_total;   // offset by the tile count below
        ri.counter = s->counter;
        for (int y = 0; y < nty; ++y) rowmap.push_back(make_int2((int)r, y));
        nrows_total += nty;
        ri.N = s->N;
        ri.rho_ref = s->rho_ref;
        ri.trace = s->trace;
        ri.trace_count = s->trace_count;
        ri.err = s->err;
        info.push_back(ri);
        for (int by = 0; by < nty; ++by)
            for (int bx = 0; bx < ntx; ++bx)
                tiles.push_back(make_int4((int)r, bx, by, marches_alternate(s->N) ? 1 : 0));
    }
    b->ntiles = (int)tiles.size();
    b->nrows = nrows_total;
    for (BatchRep& ri : info) ri.first_row += b->ntiles;
    const bool ok =
        (b->prec == LB_FP32 ? upload_args<float>(b) : upload_args<__half>(b)) &&
        cudaMalloc((void**)&b->d_tiles, sizeof(int4) * tiles.size()) == cudaSuccess &&
        cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(),
                   cudaMemcpyHostToDevice) == cudaSuccess &&
        cudaMalloc((void**)&b->d_partials, 4 * sizeof(double) * (tiles.size() + nrows_total)) ==
            cudaSuccess &&
        cudaMalloc((void**)&b->d_rowmap, sizeof(int2) * rowmap.size()) == cudaSuccess &&
        cudaMemcpy(b->d_rowmap, rowmap.data(), sizeof(int2) * rowmap.size(),
                   cudaMemcpyHostToDevice) == cudaSuccess &&
        cudaMalloc((void**)&b->d_reps, sizeof(BatchRep) * info.size()) == cudaSuccess &&
        cudaMemcpy(b->d_reps, info.data(), sizeof(BatchRep) * info.size(),
                   cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_tables(b);
        return LB_ERR_OOM;
    }
    return LB_OK;
}

// Enqueue step t (buffers `cur` in) of every replica on stream s.
cudaError_t enqueue_step(const lb_batch* b, cudaStream_t s, long long t, int cur)
{
    const bool reduce = b->trace_every > 0 && t % b->trace_every == 0;
    if (b->prec == LB_FP32) {
        BatchLaunch<float> L{static_cast<const StepArgs<float>*>(b->d_args[cur]), b->d_tiles,
                             b->ntiles, b->d_partials, b->d_reps, (int)b->reps.size(),
                             b->d_rowmap, b->nrows, b->block_x, b->om1, b->trace_every,
                             b->num_sms, b->alternate};
        return fp32_batch_step(L, reduce, s);
    }
    BatchLaunch<__half> L{static_cast<const StepArgs<__half>*>(b->d_args[cur]), b->d_tiles,
                          b->ntiles, b->d_partials, b->d_reps, (int)b->reps.size(),
                          b->d_rowmap, b->nrows, b->block_x, b->om1, b->trace_every,
                          b->num_sms, b->alternate};
    return fp16_batch_step(L, reduce, s);
}

// Capture one period of steps starting at an aligned time (t % period == 0,
// hence buffers 0 in) into a graph.
bool build_graph(lb_batch* b)
{
    if (b->exec) return true;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < b->period && e == cudaSuccess; ++k) e = enqueue_step(b, b->cap, k, k & 1);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    const cudaError_t e3 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        b->exec = nullptr;
        cudaGetLastError();
        return false;
    }
    return true;
}

lb_status poison(lb_batch* b)
{
    b->poisoned = true;
    for (lb_state* s : b->reps) s->poisoned = true;
    cudaGetLastError();
    return LB_ERR_CUDA;
}

}  // namespace

extern "C" {

lb_status lb_batch_init(lb_batch** out, int count, const lb_params* params,
                        const double* const* rho_init, void* stream)
{
    NvtxRange nvtx_range("lb_batch_init");
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !params || !rho_init) return LB_ERR_ARG;
    for (int r = 0; r < count; ++r) {
        const lb_params& p = params[r];
        if (p.prec != params[0].prec || p.trace_every != params[0].trace_every ||
            p.device != params[0].device || !rho_init[r])
            return LB_ERR_ARG;
    }
    if (params[0].prec != LB_FP32 && params[0].prec != LB_FP16_DELTA) return LB_ERR_ARG;
    if (params[0].trace_every < 0) return LB_ERR_ARG;
    lb_batch* b = new (std::nothrow) lb_batch();
    if (!b) return LB_ERR_OOM;
    b->device = params[0].device;
    b->stream = static_cast<cudaStream_t>(stream);
    b->prec = params[0].prec;
    b->trace_every = params[0].trace_every;
    for (int r = 0; r < count; ++r) {
        lb_state* s = nullptr;
        const lb_status st = lb_init(&s, &params[r], rho_init[r], stream);
        if (st != LB_OK) {
            lb_batch_destroy(b);
            return st;
        }
        b->reps.push_back(s);
        b->om1 = b->om1 && params[r].omega == 1.0;
        b->alternate = b->alternate || marches_alternate(s->N);
    }
    DeviceScope dev(b->device);
    if (!dev.ok ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        lb_batch_destroy(b);
        return LB_ERR_CUDA;
    }
    const int te = b->trace_every;
    b->period = te == 0 ? 2 : (te % 2 == 0 ? te : 2 * te);
    if (b->period > 1024) b->period = 0;   // long periods: direct launches only
    const lb_status st = build_tables(b);
    if (st != LB_OK) {
        lb_batch_destroy(b);
        return st;
    }
    *out = b;
    return LB_OK;
}

lb_status lb_batch_step(lb_batch* b, long n)
{
    NvtxRange nvtx_range("lb_batch_step");
    if (!b || n < 0) return LB_ERR_ARG;
    if (b->poisoned) return LB_ERR_STATE;
    DeviceScope dev(b->device);
    if (!dev.ok) return poison(b);
    while (n > 0) {
        if (b->use_graph && b->period > 0 && b->t % b->period == 0 && n >= b->period &&
            build_graph(b)) {
            if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return poison(b);
            b->t += b->period;
            n -= b->period;   // period is even: the buffers are back to 0
        } else {
            if (enqueue_step(b, b->stream, b->t, b->cur) != cudaSuccess) return poison(b);
            b->t += 1;
            b->cur ^= 1;
            n -= 1;
        }
    }
    for (lb_state* s : b->reps) {
        s->t = b->t;
        s->cur = b->cur;
    }
    return LB_OK;
}

lb_status lb_batch_energy(lb_batch* b, int replica, double out[4])
{
    if (!b || replica < 0 || replica >= (int)b->reps.size()) return LB_ERR_ARG;
    if (b->poisoned) return LB_ERR_STATE;
    return lb_energy(b->reps[replica], out);
}

lb_status lb_batch_fields(lb_batch* b, int replica, double* rho, double* ux, double* uy)
{
    if (!b || replica < 0 || replica >= (int)b->reps.size()) return LB_ERR_ARG;
    if (b->poisoned) return LB_ERR_STATE;
    return lb_fields(b->reps[replica], rho, ux, uy);
}

lb_status lb_batch_trace(lb_batch* b, int replica, double* buf, int cap, int* count)
{
    if (!b || replica < 0 || replica >= (int)b->reps.size()) return LB_ERR_ARG;
    if (b->poisoned) return LB_ERR_STATE;
    return lb_trace(b->reps[replica], buf, cap, count);
}

lb_status lb_batch_get_launch(const lb_batch* b, int* block_x, int* rows_per_cta, int* use_graph)
{
    if (!b || !block_x || !rows_per_cta || !use_graph) return LB_ERR_ARG;
    *block_x = b->block_x;
    *rows_per_cta = b->rows;
    *use_graph = b->use_graph ? 1 : 0;
    return LB_OK;
}

lb_status lb_batch_set_launch(lb_batch* b, int block_x, int rows_per_cta, int use_graph)
{
    if (!b) return LB_ERR_ARG;
    if (b->poisoned) return LB_ERR_STATE;
    if (block_x != 64 && block_x != 96 && block_x != 128 && block_x != 192 && block_x != 256)
        return LB_ERR_ARG;
    if (rows_per_cta < kMinRows || rows_per_cta > kMaxRows || (use_graph != 0 && use_graph != 1))
        return LB_ERR_ARG;
    NvtxRange nvtx_range("lb_batch_set_launch");
    DeviceScope dev(b->device);
    if (!dev.ok || cudaStreamSynchronize(b->stream) != cudaSuccess) return poison(b);
    b->block_x = block_x;
    b->rows = rows_per_cta;
    b->use_graph = use_graph == 1;
    return build_tables(b);
}

lb_status lb_batch_check_guards(lb_batch* b, int* damaged)
{
    if (!b || !damaged) return LB_ERR_ARG;
    *damaged = 0;
    for (lb_state* s : b->reps) {
        int d = 0;
        const lb_status st = lb_check_guards(s, &d);
        if (st != LB_OK) return st;
        *damaged += d;
    }
    return LB_OK;
}

int lb_batch_count(const lb_batch* b) { return b ? (int)b->reps.size() : -1; }

long lb_batch_time(const lb_batch* b) { return b ? (long)b->t : -1; }

void lb_batch_destroy(lb_batch* b)
{
    if (!b) return;
    NvtxRange nvtx_range("lb_batch_destroy");
    DeviceScope dev(b->device);
    cudaStreamSynchronize(b->stream);
    free_tables(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaGetLastError();
    for (lb_state* s : b->reps) lb_destroy(s);
    delete b;
}

}  // extern "C"

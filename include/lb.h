/*
 * lb.h — C ABI of the GB300 (sm_103a) two-belt Shan–Chen lattice Boltzmann
 * library (liblbsc.so).
 *
 * The method is the one of Chibbaro, Falcucci, Chen, Shan, Chiatti, Succi,
 * "Lattice Boltzmann models for non-ideal fluids with arrested
 * phase-separation" (arXiv:1008.2865): a periodic 2D D2Q9 BGK fluid (Sec. 2,
 * Eqs. 1-4) with the Shan–Chen pseudopotential psi(rho) (Sec. 2) acting
 * through a two-belt, 24-neighbour force (Sec. 3, Eq. FORCE and Table 1),
 * plus the Ising-like pseudo-energies E_s, E_m and E_bulk of Sec. 5.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an lb_status; the library never aborts, traps or
 *     prints. After LB_ERR_CUDA the state is poisoned: only lb_destroy (and
 *     lb_time) remain valid on it.
 *   - Fields are row-major [y][x] (x fastest), N = nx*ny doubles.
 *   - Inputs are copied; outputs go to caller-owned memory. Pointers may be
 *     host memory (pageable or pinned) or device memory of the state's
 *     device; the library tells them apart with cudaPointerGetAttributes.
 *   - The library owns the device memory of a state (allocated in lb_init,
 *     freed in lb_destroy). There is no global mutable state: several states
 *     may live on one device and be driven from different host threads, one
 *     thread per state at a time.
 *   - Work is enqueued on the stream given at init (a cudaStream_t, or NULL
 *     for the legacy default stream) on the device named in lb_params.device.
 *     lb_step is asynchronous; lb_energy, lb_fields and lb_trace synchronise
 *     that stream before they return and report what the kernels flagged
 *     since: LB_ERR_NONFINITE when a fused energy/mass reduction was not
 *     finite, LB_ERR_TIMEOUT when a bounded wait ran out.
 *   - Each call that enqueues device work, synchronises or frees opens an NVTX
 *     range named after it (Nsight timelines); the plain getters and setters
 *     (lb_time, lb_get_launch, lb_set_launch, lb_set_wait_limit, lb_status_str,
 *     lb_batch_count, lb_batch_time, lb_batch_get_launch) do not.
 *   - The calling thread's current CUDA device is the same on return as it was
 *     on entry: a call that works on a state of another device switches to that
 *     device for its duration only.
 */
#ifndef LBSC_LB_H
#define LBSC_LB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = -1,        /* invalid argument; nothing was changed */
    LB_ERR_CUDA = -2,       /* a CUDA call failed; the state is poisoned */
    LB_ERR_OOM = -3,        /* device allocation failed; nothing was created */
    LB_ERR_NONFINITE = -4,  /* a NaN/Inf density or energy (a fused reduction or the result) */
    LB_ERR_STATE = -5,      /* call not valid in the state's current condition */
    LB_ERR_TIMEOUT = -6     /* a bounded in-kernel wait ran out; the state is poisoned */
} lb_status;

/* Pseudopotential form. Sec. 2: psi = sqrt(rho0) (1 - exp(-rho/rho0)),
 * the Shan–Chen form the paper uses throughout (rho0 = 1 in Sec. 3). */
typedef enum { LB_PSI_SC_EXP = 0 } lb_psi_form;

/* Arithmetic of a state.
 *   LB_FP32: the throughput path. Populations are stored in FP32 as
 *            deviations g_i = f*_i - w_i rho_ref from the rest equilibrium at
 *            the reference density rho_ref, psi as psi - psi(rho_ref); all
 *            arithmetic is FP32 except the FP64 energy/mass accumulation.
 *   LB_FP64: the parity path: FP64 populations and arithmetic in the same
 *            operation order as a plain per-site evaluation of Eqs. 1-4 and
 *            Eq. FORCE, without fused multiply-add, with a correctly rounded
 *            exp; slow on GB300 and not meant for throughput.
 *   LB_FP16_DELTA: as LB_FP32 but g_i stored in IEEE half precision (FP32
 *            arithmetic, FP32 psi). */
typedef enum { LB_FP32 = 0, LB_FP64 = 1, LB_FP16_DELTA = 2 } lb_precision;

typedef struct {
    int nx, ny;             /* lattice size; both >= 5 (the force stencil reaches 2 sites) */
    double omega;           /* BGK relaxation frequency 1/tau, 0 < omega < 2 (Eq. 1; tau = 1 in Sec. 4) */
    double G1;              /* first-belt coupling on the D2Q9 weights w_i (Eq. FORCE); < 0 attracts */
    double G2;              /* coupling on the E(8) weights p of belts 1 and 2 (Eq. FORCE, Table 1) */
    double rho0;            /* psi density scale rho0 > 0 (Sec. 2) */
    lb_psi_form psi_form;   /* LB_PSI_SC_EXP */
    lb_precision prec;      /* arithmetic, see above */
    int trace_every;        /* record (t, mass, E_s, E_m, E_bulk) every this many steps; 0 = never */
    double rho_ref;         /* FP32/FP16 storage reference density; <= 0 means the mean of rho_init */
    int device;             /* CUDA device ordinal the state lives on */
} lb_params;

typedef struct lb_state lb_state;   /* opaque; owns device memory */

/* Create a state at t = 0 with f_i(x, 0) = w_i rho_init(x), the u = 0
 * equilibrium of Eq. 4 (the noisy-density start of Sec. 4).
 *   out       receives the new state (set to NULL on failure)
 *   p         parameters; validated: nx, ny >= 5, 0 < omega < 2, finite G1
 *             and G2, rho0 > 0, trace_every >= 0, known psi_form and prec,
 *             nx*ny*9 and 288*ceil(nx/32)*ny (the populations of an FP32 or
 *             FP16 state, stored in 32-column tiles) below 2^31
 *   rho_init  N initial densities, host or device, each finite and > 0
 *   stream    cudaStream_t (as void*) used by every later call on the state
 * Errors: LB_ERR_ARG (bad parameter or rho_init), LB_ERR_OOM, LB_ERR_CUDA. */
lb_status lb_init(lb_state** out, const lb_params* p, const double* rho_init, void* stream);

/* Advance n >= 0 steps of Eq. 1: psi(rho) (Sec. 2), the two-belt force of
 * Eq. FORCE taken with the attractive sign of Eq. forza, BGK collision
 * towards the Eq. 4 equilibrium at the shifted velocity u + F/(omega rho),
 * then streaming. States t with t % trace_every == 0 append a trace row.
 * Asynchronous. Errors: LB_ERR_ARG (n < 0), LB_ERR_STATE, LB_ERR_CUDA. */
lb_status lb_step(lb_state* s, long n);

/* Pseudo-energies and mass of the current state t (Sec. 5):
 *   out[0] = E_s    = 1/2 sum_x psi(x) sum_{i=0..8} (G1 w_i + G2 p_si) psi(x + c_i)
 *   out[1] = E_m    = 1/2 sum_x psi(x) sum_{i=1..16} G2 p_mi psi(x + c_mi)
 *   out[2] = E_bulk = (G1 + G2)/2 sum_x psi(x)^2                (Eq. Ebulk)
 *   out[3] = mass   = sum_x rho(x)
 * out is host memory (4 doubles). Synchronises the stream.
 * Errors: LB_ERR_ARG, LB_ERR_NONFINITE (any of the four is not finite),
 * LB_ERR_STATE, LB_ERR_CUDA. */
lb_status lb_energy(lb_state* s, double out[4]);

/* Density rho = sum f_i and velocity u = sum c_i f_i / rho (Eqs. 2-3) of the
 * current state, written as N doubles each into caller-owned host or device
 * arrays; any of the three may be NULL. Device and pinned host arrays are
 * written directly by one kernel pass; pageable host arrays go through a device
 * buffer of N doubles that the state keeps. Synchronises the stream.
 * Errors: LB_ERR_ARG, LB_ERR_STATE, LB_ERR_CUDA. */
lb_status lb_fields(lb_state* s, double* rho, double* ux, double* uy);

/* Copy the recorded trace rows (t, mass, E_s, E_m, E_bulk), oldest first,
 * into buf (host, cap rows of 5 doubles); *count receives the number of rows
 * written (the most recent ones if more than cap are stored; the device ring
 * keeps the last 65536). Synchronises the stream.
 * Errors: LB_ERR_ARG, LB_ERR_STATE, LB_ERR_CUDA. */
lb_status lb_trace(lb_state* s, double* buf, int cap, int* count);

/* Launch shape of the fused FP32/FP16 step kernel. A CTA of block_x threads
 * marches over rows_per_cta output rows of a strip of columns, one thread per
 * column plus a one-column halo on each side. pipeline selects how the input
 * rows reach the CTA:
 *   0  register prefetch: each thread loads its populations of the next row
 *      from global memory (any lattice shape; block_x in {64, 96, 128, 192, 256},
 *      block_x - 2 output columns per CTA);
 *   1  bulk-copy rings: the bulk-copy (TMA) engine stages whole rows in shared
 *      memory several rows ahead (block_x in {64, 128, 256}; needs nx a
 *      multiple of 32 and nx >= block_x + 64).
 * lb_init starts with pipeline 0 (measured the faster of the two on GB300 for
 * the 8192 x 8192 lattice). rows_per_cta is in
 * [4, 4096]. The shape changes how the work is split, not the trajectory;
 * only the FP32 rounding of the energy partial sums depends on it.
 * Errors: LB_ERR_ARG for NULL or unsupported values, LB_ERR_STATE for an FP64
 * state (whose kernels have no such shape). */
lb_status lb_get_launch(const lb_state* s, int* block_x, int* rows_per_cta, int* pipeline);
lb_status lb_set_launch(lb_state* s, int block_x, int rows_per_cta, int pipeline);

/* Bound on every in-kernel wait of the bulk-copy pipeline, in SM clock cycles
 * (default 2e9, about one second at GB300 clocks). A wait that runs out makes
 * the kernel record an error and return; the next synchronising call
 * (lb_energy, lb_fields, lb_trace) reports LB_ERR_TIMEOUT and poisons the
 * state, while the CUDA context stays usable. test_skip_copies is a test hook
 * (0 or 1): with 1, every CTA arms the barrier of its first row unit for the
 * unit's bytes but issues none of the unit's copies, so that wait runs out on
 * purpose with nothing of the unit in flight; use 0 otherwise.
 * Errors: LB_ERR_ARG (NULL, cycles <= 0, test_skip_copies not 0 or 1). */
lb_status lb_set_wait_limit(lb_state* s, long long cycles, int test_skip_copies);

/* Guard check (debugging without a memory checker). Every device buffer of a
 * state is allocated with a 256-byte guard region on each side holding the
 * byte 0xA5; *damaged receives the number of buffers whose guards no longer
 * hold it, i.e. that some kernel wrote outside. Synchronises the stream.
 * Errors: LB_ERR_ARG, LB_ERR_CUDA. */
lb_status lb_check_guards(lb_state* s, int* damaged);
/* Test hook for the guard check: overwrite one byte of the tail guard of the
 * state's buffer number `buffer` (0-based, in allocation order) with a host-side
 * cudaMemset. Errors: LB_ERR_ARG (NULL or no such buffer), LB_ERR_CUDA. */
lb_status lb_debug_damage_guard(lb_state* s, int buffer);
/* Test hook for the allocation-failure path: after `after` more state buffer
 * allocations succeed, the next one fails once (as if the device were out of
 * memory); a negative value disarms it. Process-wide. */
void lb_debug_fail_alloc(int after);

/* Checkpoint and resume. A saved state is a small header (lattice size,
 * precision, time step, reference density) followed by the populations and
 * psi of the current time step; loading it into a state of the same size and
 * precision (and, for FP32/FP16, the same rho_ref) continues the run bit for
 * bit as if it had not been interrupted. The trace ring is not part of it.
 *   lb_state_bytes   size of the saved form (0 for NULL)
 *   lb_save_state    write it to dst (host or device memory, >= that size)
 *   lb_load_state    read it from src into s (host or device memory)
 * Both synchronise the stream. Errors: LB_ERR_ARG (NULL, short buffer, a
 * header that does not match s), LB_ERR_STATE, LB_ERR_CUDA. */
size_t lb_state_bytes(const lb_state* s);
lb_status lb_save_state(lb_state* s, void* dst, size_t bytes);
lb_status lb_load_state(lb_state* s, const void* src, size_t bytes);

/* Gradient of J = E_s(T) + E_m(T) + sum_x (rho(x, T) - rho_target(x))^2 — the
 * Sec. 5 pseudo-energy of the state after `steps` steps plus the squared misfit
 * of its density to a target field — with respect to the initial density
 * field and the couplings G1, G2 of Eq. FORCE, by a hand-written reverse sweep
 * of the step (FP32 state and adjoint, FP64 accumulation of J and of the G1,
 * G2 gradients) with checkpointing: the forward run stores its state every
 * checkpoint_every steps (0 picks ceil(sqrt(steps))), and each segment is
 * recomputed from its checkpoint before the reverse sweep crosses it.
 *   s             an LB_FP32 state at t = 0 (fresh from lb_init); on return it
 *                 holds the state at t = steps (trace rows as from lb_step)
 *   rho_target    N doubles, host or device
 *   J             host double: the objective
 *   grad_rho      N doubles, host or device: dJ/drho_init(x)
 *   grad_G        host doubles {dJ/dG1, dJ/dG2}
 * Working memory (about 40 N (steps/C + C) bytes) is allocated for the call.
 * Errors: LB_ERR_ARG, LB_ERR_STATE (not FP32, t != 0, poisoned), LB_ERR_OOM,
 * LB_ERR_CUDA, LB_ERR_NONFINITE. */
lb_status lb_adjoint(lb_state* s, long steps, const double* rho_target, int checkpoint_every,
                     double* J, double* grad_rho, double* grad_G);

/* The objective of lb_adjoint evaluated on the current state, without the
 * gradient: J = E_s + E_m + sum_x (rho(x) - rho_target(x))^2 (the Sec. 5
 * pseudo-energy plus the squared density misfit), accumulated in FP64.
 * For LB_FP32 (and LB_FP16_DELTA) states it runs lb_adjoint's own terminal
 * kernel with the same grid and summation order, so lb_objective after
 * lb_step(T) equals the J that lb_adjoint(T) returns, bit for bit; for LB_FP64
 * states it evaluates the same sums on the FP64 populations.
 *   rho_target  N doubles, host or device (pageable host memory goes through a
 *               device buffer of N doubles that the state keeps, as in lb_fields)
 *   J           host double
 * Synchronises the stream. Errors: LB_ERR_ARG, LB_ERR_STATE, LB_ERR_OOM,
 * LB_ERR_CUDA, LB_ERR_NONFINITE. */
lb_status lb_objective(lb_state* s, const double* rho_target, double* J);

/* ---- Batches: many independent lattices advanced by one launch per step ----
 * A batch holds `count` replicas (each with its own size, couplings, omega,
 * rho_ref and initial density; all with the same prec — LB_FP32 or
 * LB_FP16_DELTA —, trace_every and device), e.g. a G2 sweep with distinct
 * seeds. lb_batch_step advances all of them: one persistent launch per step
 * strides over a work list of every replica's tiles, and steps are replayed
 * from a CUDA graph of one trace period when the batch time is aligned to it.
 * A replica's fields, energies and trace are bit-identical to those of the
 * same lattice run alone with the same launch shape (register-prefetch
 * pipeline). The paper runs its A2 scan (Sec. 4) as separate simulations;
 * batching is this library's way to run such sweeps on one GPU.
 *   params    array of count parameter sets (validated as in lb_init)
 *   rho_init  array of count pointers to N_r initial densities (host or device)
 * Errors: LB_ERR_ARG (count < 1, mixed prec/trace_every/device, FP64, or any
 * lb_init error), LB_ERR_OOM, LB_ERR_CUDA. */
typedef struct lb_batch lb_batch;
lb_status lb_batch_init(lb_batch** out, int count, const lb_params* params,
                        const double* const* rho_init, void* stream);
/* Advance every replica n >= 0 steps (asynchronous). */
lb_status lb_batch_step(lb_batch* b, long n);
/* lb_energy / lb_fields / lb_trace of replica `replica` (0 <= replica < count). */
lb_status lb_batch_energy(lb_batch* b, int replica, double out[4]);
lb_status lb_batch_fields(lb_batch* b, int replica, double* rho, double* ux, double* uy);
lb_status lb_batch_trace(lb_batch* b, int replica, double* buf, int cap, int* count);
/* Tile shape shared by all replicas (block_x in {64, 96, 128, 192, 256},
 * rows_per_cta in [4, 4096]) and whether steps replay from a CUDA graph
 * (use_graph 0 or 1). Defaults: 128, 32, 1. */
lb_status lb_batch_get_launch(const lb_batch* b, int* block_x, int* rows_per_cta, int* use_graph);
lb_status lb_batch_set_launch(lb_batch* b, int block_x, int rows_per_cta, int use_graph);
/* lb_check_guards summed over the replicas. */
lb_status lb_batch_check_guards(lb_batch* b, int* damaged);
/* Number of replicas (-1 for NULL) and steps taken (-1 for NULL). */
int lb_batch_count(const lb_batch* b);
long lb_batch_time(const lb_batch* b);
/* Free the batch and its replicas; NULL is a no-op. */
void lb_batch_destroy(lb_batch* b);

/* Pseudo-energies and mass of caller-provided fields, without any device
 * allocation. The paper has no counterpart to this entry point: it exists
 * for callers that cannot call cudaMalloc, such as code running inside a
 * framework that hands out all device memory from its own pool (an extra
 * cudaMalloc there bypasses the pool's accounting and can fail once the pool
 * holds the memory), or code that must not trigger the implicit device
 * synchronisation of cudaMalloc. The sums are the same as lb_energy's:
 *   out[0] = E_s, out[1] = E_m, out[2] = E_bulk, out[3] = sum rho,
 * computed from
 *   psi, rho  N = nx*ny doubles each, row-major [y][x], in device memory of
 *             the current device (the psi values are used as given); memory
 *             of another device is refused with LB_ERR_ARG before any launch;
 *   nx, ny    >= 5, and nx*ny <= 134,217,728 sites (8192 CTAs of 16,384
 *             sites: the capacity of the scratch array below);
 *   G1, G2    the couplings, as for lb_init;
 *   out       4 doubles, host or device memory. With host memory the call
 *             synchronises the stream and returns LB_ERR_NONFINITE if a sum
 *             is not finite; with device memory it returns without waiting.
 *             A host out while the stream is being captured is refused with
 *             LB_ERR_ARG (the synchronisation would break the capture).
 * Scratch: one static device array of 262,208 bytes inside this library,
 * present on every GPU that loads the library until the process exits. The
 * first call on a device looks up that array's device address with the
 * device current (cudaGetSymbolAddress), so make the first call on each
 * device before any stream capture begins. Every call shares the array and
 * clears its arrival counter first; calls whose kernels overlap on the GPU
 * (different streams, or different host threads on one device) race on it
 * and must be serialised by the caller.
 * Errors: LB_ERR_ARG (NULL, psi/rho not in memory of the current device,
 * sizes out of range, non-finite couplings, host out during capture),
 * LB_ERR_CUDA, LB_ERR_NONFINITE. */
lb_status lb_energy_noalloc(const double* psi, const double* rho, int nx, int ny, double G1,
                            double G2, double* out, void* stream);

/* Current time step t (number of lb_step steps taken since lb_init); -1 for NULL. */
long lb_time(const lb_state* s);

/* Free the state and its device memory; NULL is a no-op. Synchronises the stream. */
void lb_destroy(lb_state* s);

/* Static description of a status code. */
const char* lb_status_str(lb_status st);

#ifdef __cplusplus
}
#endif
#endif

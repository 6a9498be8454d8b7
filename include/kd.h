/*
 * kd.h -- C ABI of the GB300 (sm_103a) FFT split-operator library for the 2D Dirac
 * equation in a Gaussian-beam standing light wave.
 *
 * Paper: Ge, Ahrens & Shen, "Two-dimensional simulation of the spin-flip in the
 * Kapitza-Dirac effect", arXiv 2307.01571.  Every call below names the passage that
 * defines what it computes.
 *
 * Conventions shared by all calls
 *  - All functions return KD_OK (0) or a negative KD_ERR_* code and never abort.
 *    kd_last_error() returns a thread-local message describing the last failure.
 *  - A spinor is an array of complex numbers laid out [ny][nx][4], point-major,
 *    components in the Dirac (standard) representation (psi1..psi4), complex128
 *    (interleaved doubles) for KD_FP64 and KD_DW simulations and complex64 for KD_FP32
 *    and KD_FP32_TC.
 *    Row iy, column ix is the point (x_min + ix dx, y_min + iy dy) of the box at t = 0.
 *  - `where` = KD_HOST for a host pointer (the call copies synchronously) or
 *    KD_DEVICE for a device pointer on the simulation's GPU (the call is ordered on the
 *    simulation's stream; the caller keeps the memory alive until the stream has
 *    passed the call).
 *  - The library owns its device buffers.  The caller owns every pointer it passes
 *    and may free the parameter structs as soon as a call returns.
 *  - Sizes: nx and ny are powers of two in [4, 4096].
 *  - There is no CPU fallback: with no usable CUDA device kd_create fails with
 *    KD_ERR_CUDA.
 *  - A kd_sim is not thread-safe; use one per host thread or serialise calls.
 */
#ifndef KD_H
#define KD_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KD_OK 0
#define KD_ERR_ARG (-1)              /* invalid argument (null pointer, bad value) */
#define KD_ERR_UNSUPPORTED_SIZE (-2) /* grid size not a power of two in [4, 4096] */
#define KD_ERR_CUDA (-3)             /* a CUDA call failed, or no usable device */
#define KD_ERR_NONFINITE (-4)        /* an observed norm was NaN or infinite */
#define KD_ERR_NORM_DRIFT (-5)       /* observed norm left the watchdog tolerance */
#define KD_ERR_TIMEOUT (-6)          /* a bounded device wait ran out */
#define KD_ERR_STATE_MISMATCH (-7)   /* checkpoint does not match this simulation */
#define KD_ERR_NOMEM (-8)            /* device allocation failed */
#define KD_ERR_CANCELLED (-9)        /* kd_step stopped early at a kd_cancel request */

#define KD_FP64 0 /* complex128 spinor, FP64 arithmetic throughout */
#define KD_FP32 1 /* complex64 spinor, FP32 arithmetic; FP64-built phase tables */
/* Precision form: complex64 spinor and tables as KD_FP32, but the full sweeps of axes of
 * 1024 points evaluate their FFTs as 32-point DFT matrix products on the tensor cores
 * (four-step 1024 = 32 x 32 FFT of Sec. II.D's transforms; FP16 operands split hi + lo,
 * three products per term, FP32 accumulation).  The tensor cores' FP32 accumulation
 * truncates, so the norm decays by ~7e-7 per step (1.4e-3 over a 2000-step run; KD_FP32:
 * below 1e-6) and the error against FP64 grows with it (~1e-4 after 200 steps).  The half
 * sweeps at run ends and axes of other lengths run the KD_FP32 kernels.  State and
 * checkpoints are those of KD_FP32 (interchangeable). */
#define KD_FP32_TC 2
/* Double-word form, FP64-accurate on the FP32 pipe: every real of the spinor, the phase
 * tables and the arithmetic of the step is an unevaluated sum of two floats (48
 * significand bits; error-free transformations of Knuth, Dekker and Joldes-Muller-Popescu),
 * the field's exp and sin/cos evaluated to ~1e-14; the FP64 pipe of GB300 runs at 1/64 of
 * the FP32 pipe.  The step is the same Strang step as KD_FP64 (Sec. II.D); results agree
 * with FP64 to ~1e-11 relative over thousands of steps.  The ABI's spinors are complex128
 * as for KD_FP64; read-outs (observables, densities) are computed in FP64 from an FP64
 * copy of the state.  Device memory as KD_FP64 plus one spinor-sized buffer. */
#define KD_DW 3

#define KD_HOST 0
#define KD_DEVICE 1

#define KD_FIELD_NONE 0     /* free particle */
#define KD_FIELD_PLANE 1    /* plane-wave standing wave, A = -2 A0 sin(wt) cos(k x) e_y */
#define KD_FIELD_GAUSS 2    /* Gaussian-beam standing wave, Sec. II.A */

/* Unit system: electron mass, speed of light, reduced Planck constant, charge.
 * Atomic units are {1, 137.035999, 1, -1}; natural units {1, 1, 1, -1}. */
typedef struct { double m, c, hbar, q; } kd_units;

/* Periodic box at t = 0 (Sec. II.D: 2048 x 128 points over 80 x 40 wavelengths). */
typedef struct {
    int32_t nx, ny;
    double x_min, x_max, y_min, y_max;
} kd_grid;

/* Laser field, Eqs. (Equation_of_Gaussian_beam), (Phase_of_Gaussian_beam),
 * (Equation_of_vector_potential), scalar potential zero.
 *  a0        q A0 / (m c^2), dimensionless (the paper's A0 = 0.1 mc/q is a0 = 0.1)
 *  k_L       wave number, omega = c k_L
 *  epsilon   beam divergence, waist w0 = 1/(k_L epsilon), Rayleigh length k_L w0^2 / 2
 *  env_T     length of a sin^2(pi t / env_T) envelope; 0 = continuous wave
 *  phase0    added to omega t
 *  p_shift_* constant-gauge offset: kinetic = canonical + p_shift (the paper's
 *            A_m = 1.0 mc/q along y is p_shift_y = m c)
 *  box_vy    speed of the co-moving box along y (rows sit at y + box_vy t); the frame
 *            translation adds the phase exp(+i box_vy p_y dt / hbar) to each kinetic step */
typedef struct {
    int32_t kind;
    int32_t longitudinal;
    double a0, k_L, epsilon, env_T, phase0, p_shift_x, p_shift_y, box_vy;
} kd_field;

/* Gaussian wave packet, Eq. (Density_distribution_of_Gaussian_wave_packet):
 * p0 kinetic centre momentum, r0 centre position (absolute, t = 0), sigma_p width,
 * spin +1/-1 along x (basis 0, chi = (1, +-1)/sqrt 2) or along z (basis 1). */
typedef struct {
    double p0x, p0y, r0x, r0y, sigma_p;
    int32_t spin, basis;
} kd_packet;

/* Momentum-space read-out windows (Sec. III.B, Tables I and II): the incoming and the
 * diffracted peak, each the cells within half_width (infinity norm) of the grid point
 * nearest to the given kinetic momentum, plus a single-cell read-out at target. */
typedef struct {
    double p_in_x, p_in_y, p_diff_x, p_diff_y, target_x, target_y;
    double half_width;
    int32_t basis; /* spin basis of c^+- : 0 = x-polarised (the paper's), 1 = z */
    int32_t pad_;
} kd_obs_spec;

/* Observables of one position-space state (Sec. III).  Momentum-space values are
 * discrete cell probabilities |DFT psi|^2 dx dy / P (they sum to the norm);
 * c^+- = u^+-(pi)^dagger phi with normalised bispinors, Eq. (Equation_of_spin_projection). */
typedef struct {
    double t;
    double norm;                       /* sum |psi|^2 dx dy, Eq. (probability_density) */
    double pop_in, pop_diff;           /* window sums of |phi|^2 */
    double cp_in, cm_in, cp_diff, cm_diff; /* window sums of |c+|^2, |c-|^2 */
    double max_diff, cp_max_diff, cm_max_diff; /* maxima over the diffracted window */
    double p_target, cp_target, cm_target;     /* values at the target cell */
} kd_obs;

typedef struct kd_sim kd_sim;

/* Creates a simulation on the current CUDA device.  precision is KD_FP64, KD_FP32,
 * KD_FP32_TC or KD_DW.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream) on which every
 * device operation of this simulation is ordered.  The spinor starts at zero, t = 0.
 * Errors: KD_ERR_ARG, KD_ERR_UNSUPPORTED_SIZE, KD_ERR_CUDA, KD_ERR_NOMEM. */
int kd_create(const kd_units* units, const kd_grid* grid, const kd_field* field,
              int32_t precision, void* cuda_stream, kd_sim** out);

/* Sets psi to the packet: phi(p, 0) = u^s(p) rho(p) on the momentum grid
 * (Sec. II.C), an inverse 2D FFT, and normalisation to sum |psi|^2 dx dy = 1.  Resets
 * t to 0 and sets the default observation spec (windows around p0 and p0 + 2 hbar
 * k_L e_x, half width hbar k_L / 2, target p0 + 2 hbar k_L e_x). */
int kd_init_packet(kd_sim* sim, const kd_packet* packet);

/* Replaces the observation spec used by kd_step and by kd_observe(sim, NULL, ...). */
int kd_set_obs_spec(kd_sim* sim, const kd_obs_spec* spec);

/* Copies a [ny][nx][4] spinor in (set) or out (get); layout in the header comment. */
int kd_set_spinor(kd_sim* sim, const void* psi, int32_t where);
int kd_get_spinor(kd_sim* sim, void* psi, int32_t where);

/* Sets the time of the current state (and the step counter to 0), or reads them. */
int kd_set_time(kd_sim* sim, double t);
int kd_get_time(kd_sim* sim, double* t, int64_t* steps_done);

/* Advances the state by nsteps Strang steps of length dt (Sec. II.D):
 *   psi <- exp(-i dt V(t_{n+1})/2) F^-1 exp(-i dt K) F exp(-i dt V(t_n)/2) psi,
 * with V = -q alpha.A (Eq. Hamiltonian operator, phi = 0), K = c alpha.pi + beta m c^2 -
 * box_vy p_y evaluated per grid momentum in closed form, F the unnormalised 2D DFT.
 * If obs_every > 0, the observables of the spec are recorded after every obs_every
 * steps; up to obs_cap records go to obs_out (host memory) and *n_obs (may be NULL)
 * receives how many were produced.  Returns KD_ERR_NONFINITE if a recorded norm was not
 * finite and KD_ERR_NORM_DRIFT if one left the watchdog tolerance (the state is then
 * the state after all nsteps).  On return the state is in position space at t + nsteps dt
 * and, when obs_every > 0, the call has synchronised the stream.
 * The steps are enqueued in chunks of obs_every steps (64 without observations), each a
 * CUDA graph launch; unless the stream is being captured, the host keeps at most four
 * chunks in flight (it waits for the chunk four back before enqueuing the next), so the
 * call returns when all but the last few chunks have run.
 * Cancellation (kd_cancel): a request seen before a chunk is enqueued makes that chunk the
 * call's last one, closed at its end, and kd_step returns KD_ERR_CANCELLED with the state
 * a valid position-space state after the steps that ran (kd_get_time reports them, and
 * the observation records of those steps are delivered). */
int kd_step(kd_sim* sim, double dt, int64_t nsteps, int64_t obs_every, kd_obs* obs_out,
            int64_t obs_cap, int64_t* n_obs);

/* Observables of the current state with spec (NULL = the simulation's spec).  Synchronous. */
int kd_observe(kd_sim* sim, const kd_obs_spec* spec, kd_obs* out);

/* Per-cell momentum-space probabilities (Eqs. px_momentum_space_probability_density and
 * Equation_of_spin_projection): out[ny][nx][3] doubles = (|phi|^2, |c+|^2, |c-|^2) in
 * the given spin basis, cells in FFT order (index k -> k < n/2 ? k : k - n). */
int kd_get_momentum_density(kd_sim* sim, int32_t basis, double* out, int32_t where);

/* y-integrated density Phi(x) = sum_y |psi|^2 dy over the box, Eq.
 * (y_integrated_probability_density): out[nx] doubles. */
int kd_get_density_x(kd_sim* sim, double* out, int32_t where);

/* Sets the watchdog of kd_step: a recorded norm that differs from the norm at the start
 * of the call by more than tol times that norm makes kd_step return KD_ERR_NORM_DRIFT.
 * tol <= 0 switches the drift check off (the default); the non-finite check is always
 * on when observations are recorded. */
int kd_set_watchdog(kd_sim* sim, double tol);

/* Checkpoint: *size receives the byte count; with buf non-NULL and *size large enough
 * the state (spinor, time, step counter and a hash of the parameters) is written to
 * buf (host memory).  kd_set_state restores it; KD_ERR_STATE_MISMATCH if it was taken
 * from a simulation with different parameters or precision. */
int kd_get_state(kd_sim* sim, void* buf, size_t* size);
int kd_set_state(kd_sim* sim, const void* buf, size_t size);

/* Batched form: several independent simulations (any grid sizes and precisions, one
 * device) advanced together.  kd_batch_step runs the same Strang-step schedule as kd_step
 * for every simulation, each with its own dt[i], as one CUDA-graph launch per chunk of
 * steps in which each simulation's sweeps form an independent branch, so that the
 * simulations' kernels run concurrently.  Observation records go to
 * obs_out[i * obs_cap + j] (host memory); *n_obs receives the count per simulation.  The
 * batch borrows the simulations: between batch calls they may be used on their own, but
 * not during one (a batch call orders all their work on cuda_stream).  Returns the first
 * error of any simulation (the others are still advanced).  The batch holds no buffers of
 * its own besides its graphs. */
typedef struct kd_batch kd_batch;
int kd_batch_create(kd_sim* const* sims, int32_t n, void* cuda_stream, kd_batch** out);
int kd_batch_step(kd_batch* batch, const double* dt, int64_t nsteps, int64_t obs_every,
                  kd_obs* obs_out, int64_t obs_cap, int64_t* n_obs);
void kd_batch_destroy(kd_batch* batch);
/* Batch-aware FFT autotuner: members advanced together compete for the GPU, so the launch
 * variants that are fastest for a grid alone (kd_autotune) need not be fastest in the
 * batch.  For each axis and each group of members with the same grid and form (FP64
 * members excepted), every variant is timed over `steps` steps of the whole batch (after
 * one untimed run that captures the graphs), and kept when the batch is more than 2 %
 * faster.  The members' states, times and step counts are restored afterwards (each
 * member's work buffer holds its state meanwhile); only the variants change.  variants
 * (may be NULL) receives 2 ints per member (x, y).  steps in [1, 4096]; synchronises;
 * KD_ERR_ARG while the batch's or a member's stream is being captured. */
int kd_batch_autotune(kd_batch* batch, const double* dt, int32_t steps, int32_t* variants);
/* (In the persistent form, kd_batch_set_mode below, the x variants are searched among the two the
 * persistent kernel holds, and the work item size, 1, 2 or 4 CTA-fulls of blocks, is tuned
 * the same way.) */

/* Persistent form of the batch (KD_BATCH_PERSISTENT): each chunk of steps of all members
 * runs as ONE kernel launch whose CTAs pull work items (step, sweep, member, group of
 * blocks) from a device queue in a fixed order; an item waits for its member's previous
 * sweep through per-member completion counters, each wait bounded by a clock64 budget
 * (about a second), after which the launch is abandoned and kd_batch_step returns
 * KD_ERR_TIMEOUT (the members' states are then not valid evolutions).  The observation and
 * opening-half work at chunk ends runs as graph branches beside it, and the whole chunk is
 * one CUDA-graph launch.  Every member must be KD_FP32 with both axes of 16 ... 512 points
 * (else KD_ERR_UNSUPPORTED_SIZE).  The kernel holds launch variants x 0 and 2 and y 3 and
 * 2: a member's x sweep runs its own variant when it is 2 (as kd_autotune picks for small
 * grids), else 0; its y sweep runs 2 when that is its variant and the y axis has at most
 * 256 points, else 3; entering the persistent form (and every persistent step) sets each
 * member's variants to those it runs (kd_get_sweep_variants reports them), so that its
 * sweeps outside the kernel run them too.  A member advanced this way equals the member
 * advanced alone on those variants, bit for bit.  KD_BATCH_GRAPH (the default) restores the graph-branch
 * form.  The persistent form holds device buffers of its own (descriptors and counters,
 * O(n)).  Synchronises. */
#define KD_BATCH_GRAPH 0
#define KD_BATCH_PERSISTENT 1
int kd_batch_set_mode(kd_batch* batch, int32_t mode);

/* Surrogate network (a learned stand-in for the solver's read-outs; the paper has no network): a fully
 * connected MLP, widths[0] inputs -> ... -> widths[nlayers] outputs, exact-erf GELU on the
 * hidden layers, linear output, trained with mean squared error and Adam
 * (beta = 0.9, 0.999, eps = 1e-8) by hand-written kernels (FP32; the matrix products
 * optionally on BF16 tensor cores, kd_mlp_set_precision); every reduction runs in a fixed
 * order (bitwise reproducible).  Parameters are laid out per layer as W_l
 * [widths[l+1]][widths[l]] row-major followed by b_l; the caller initialises them
 * (kd_mlp_set_params, which also resets Adam).  Row-major float batches [batch][width].
 * kd_mlp_train_step takes device pointers and is asynchronous on cuda_stream; loss_dev
 * (device, may be NULL) receives the batch loss before the update. */
typedef struct kd_mlp kd_mlp;
int kd_mlp_create(const int32_t* widths, int32_t nlayers, kd_mlp** out);
int kd_mlp_num_params(kd_mlp* net, int64_t* count);
int kd_mlp_set_params(kd_mlp* net, const float* params, int32_t where);
int kd_mlp_get_params(kd_mlp* net, float* params, int32_t where);
int kd_mlp_forward(kd_mlp* net, const float* x, int32_t batch, float* y, int32_t where,
                   void* cuda_stream);
int kd_mlp_gradients(kd_mlp* net, const float* x, const float* targets, int32_t batch,
                     float* loss, float* grads, int32_t where, void* cuda_stream);
int kd_mlp_train_step(kd_mlp* net, const float* x, const float* targets, int32_t batch,
                      float lr, float* loss_dev, void* cuda_stream);
/* The same training step on a minibatch selected on the device: rows idx[0 .. batch) of
 * x_all [n_all][widths[0]] and targets_all [n_all][widths[nlayers]] (device pointers;
 * idx device int32, indices outside [0, n_all) select rows of zeros) are gathered by the
 * library's own kernel into its staging buffers. */
int kd_mlp_train_step_gather(kd_mlp* net, const float* x_all, const float* targets_all,
                             int64_t n_all, const int32_t* idx, int32_t batch, float lr,
                             float* loss_dev, void* cuda_stream);
/* Arithmetic of the network's matrix products (forward and backward): KD_MLP_FP32 (the
 * default: FP32 tiled GEMM on the CUDA cores) or KD_MLP_BF16 (operands rounded to BF16,
 * products on the tcgen05 tensor cores with FP32 accumulation in tensor memory; the
 * epilogues, GELU, loss and Adam stay FP32).  Each BF16 product waits for the tensor cores
 * with a bounded wait; if one gives up, the next synchronising call (kd_mlp_forward to
 * host memory, kd_mlp_gradients, kd_mlp_get_params) returns KD_ERR_TIMEOUT. */
#define KD_MLP_FP32 0
#define KD_MLP_BF16 1
int kd_mlp_set_precision(kd_mlp* net, int32_t precision);
void kd_mlp_destroy(kd_mlp* net);

/* Benchmark hook: enqueues `reps` back-to-back launches of one fused sweep on the
 * simulation's stream, in place on the current state, and returns without waiting.
 * kind 0 = x sweep (inverse x-FFT, full potential step exp(-i dt V(t)/hbar), forward
 * x-FFT; the row pass of one Strang step, Sec. II.D), kind 1 = y sweep (forward y-FFT,
 * kinetic step, inverse y-FFT; the column pass).  Uses the tables and time of the last
 * kd_step call (KD_ERR_ARG before any kd_step).  The state is left in an unspecified
 * mixed representation: call it on a scratch simulation, or restore a checkpoint after.
 * The launches of one (kind, reps) pair are captured once into a CUDA graph and replayed. */
int kd_bench_sweep(kd_sim* sim, int32_t kind, int32_t reps);

/* FFT autotuner.  The FP32 sweeps are compiled in KD_SWEEP_VARIANTS launch variants
 * per axis, differing in radix schedule (radix-8 or radix-4 Stockham stages of the 2D
 * FFT of Sec. II.D), threads per CTA, column-tile width and spinor components per CTA.
 * Variant 0 is the default.  kd_autotune times every variant of both sweeps on this
 * simulation's grid (reps back-to-back launches each, graph-replayed, reading the state
 * and writing only scratch: the state is unchanged) with the step's pointwise ops for
 * time step dt, keeps variant 0 unless another is faster by more than 2 %, and applies
 * the choice to this simulation.  The choice is remembered for the process per device,
 * grid and field kind, so later simulations of that shape only look it up (flags =
 * KD_TUNE_FORCE times again).  variant_x / variant_y (may be NULL) receive the choice,
 * times_ms (may be NULL, 2 * KD_SWEEP_VARIANTS floats: x then y) the measured ms per
 * launch (the recorded ones when the choice was looked up; -1 for FP64).  FP64
 * simulations have one variant (0).  Synchronises the simulation's stream: KD_ERR_ARG
 * while that stream is being captured (kd_set_sweep_variants likewise, when it changes the
 * variants).  Variants 0 and 1 differ only in threads per CTA and give
 * bitwise identical results; the radix-4 schedule (2) and the components-per-CTA change
 * (3) round differently in the last bits (every variant meets the same accuracy).  A
 * simulation's results are reproducible for fixed variants.  kd_set_sweep_variants selects variants directly
 * (KD_ERR_ARG out of range), kd_get_sweep_variants reads them back.  The variants are
 * not part of a kd_get_state checkpoint. */
#define KD_SWEEP_VARIANTS 4
#define KD_TUNE_FORCE 1
int kd_autotune(kd_sim* sim, double dt, int32_t reps, int32_t flags, int32_t* variant_x,
                int32_t* variant_y, float* times_ms);
int kd_set_sweep_variants(kd_sim* sim, int32_t variant_x, int32_t variant_y);
int kd_get_sweep_variants(kd_sim* sim, int32_t* variant_x, int32_t* variant_y);

/* Test hook for the tensor-core sweeps' bounded waits.  kind KD_FAULT_TC_WAIT: during
 * the next step call (kd_step, or kd_batch_step of a batch holding the simulation) the
 * tensor-core sweeps issue no matrix products, so every wait
 * for them gives up after its iteration limit (about a second); the kernels then skip
 * their remaining work, free their tensor memory and set the simulation's status, and
 * kd_step returns KD_ERR_TIMEOUT with the context intact; the state is then not a valid
 * evolution (restore a checkpoint or set a new spinor).  kind 0 cancels either hook.
 * KD_ERR_ARG for other kinds, or for KD_FAULT_TC_WAIT when the simulation is not
 * KD_FP32_TC. */
#define KD_FAULT_TC_WAIT 1
/* kind KD_FAULT_PERSIST_HOLD: in the next kd_batch_step of a persistent batch holding the
 * simulation, the completion of the simulation's first work item is never signalled, so
 * the items that depend on it wait until their bounded waits give up and the call returns
 * KD_ERR_TIMEOUT (no fault, trap or hang); any precision. */
#define KD_FAULT_PERSIST_HOLD 2
int kd_inject_fault(kd_sim* sim, int32_t kind);

/* Requests that the kd_step running on this simulation (in another host thread), or the
 * next one, stop at its next chunk boundary (see kd_step).  The request is consumed by
 * the kd_step that honours it.  Safe to call from any thread while kd_step runs; not
 * applied by kd_batch_step. */
int kd_cancel(kd_sim* sim);

/* Test hook for out-of-memory handling, process-wide: with after >= 0, the device
 * allocation made after `after` further successful ones fails as if the device were out
 * of memory (the call that needed it returns KD_ERR_NOMEM and releases what it
 * allocated), and the hook turns itself off; -1 turns it off.  KD_ERR_ARG for after < -1. */
int kd_inject_alloc_failure(int32_t after);

/* Number of kernel launches this simulation has enqueued so far (graph replays counted
 * node by node). */
int kd_get_launch_count(kd_sim* sim, int64_t* launches);

/* Allocation-free density read-out.  The paper has no counterpart: this is a service
 * of the library.  It computes the norm sum |psi|^2 dx dy and the y-integrated density
 * Phi(x) = sum_y |psi|^2 dy of a caller's device spinor.
 *
 * For callers that cannot allocate device memory: hosts that hand the library a fixed
 * memory budget (another framework's pool already owns the device memory), real-time
 * loops that must never wait on the allocator (cudaMalloc and cudaFree can synchronise
 * the device), and plug-ins running inside a runtime that forbids them to allocate.  It
 * needs no kd_sim and calls no cudaMalloc/cudaFree: its only scratch is a static device
 * array of KD_NOALLOC_MAX_ROWS doubles (32 KiB) that every GPU which loads the library
 * holds until the process exits.
 *
 *  psi            device pointer, [ny][nx][4] complex spinor in the layout above,
 *                 complex128 (KD_FP64) or complex64 (KD_FP32); caller-owned
 *  dx, dy         grid spacings
 *  norm_out       device pointer to one double: sum |psi|^2 dx dy (may be NULL)
 *  density_x_out  device pointer to nx doubles: Phi(x) = sum_y |psi|^2 dy (may be NULL)
 *  cuda_stream    cudaStream_t the work is ordered on (NULL = legacy default stream)
 * Both sums accumulate in FP64.  Returns KD_ERR_UNSUPPORTED_SIZE if ny >
 * KD_NOALLOC_MAX_ROWS or nx > 4096, KD_ERR_ARG for null pointers, KD_ERR_CUDA on launch
 * failure or without a usable device.  Asynchronous on the stream.
 *
 * The first call on each device looks up the scratch array's device address with that
 * device current, and so does the first call after the device's context was replaced
 * (cudaDeviceReset); such a call made on a stream that is being captured returns
 * KD_ERR_CUDA, so make the first call before any stream capture.  All calls on a device
 * share the one scratch array (each call overwrites every entry it reads, so nothing
 * needs clearing): calls whose kernels can overlap on the GPU (different streams without
 * ordering) race on it and must be serialised by the caller. */
#define KD_NOALLOC_MAX_ROWS 4096
int kd_density_noalloc(const void* psi, int32_t nx, int32_t ny, int32_t precision, double dx,
                       double dy, double* norm_out, double* density_x_out, void* cuda_stream);

/* Frees the simulation's device memory and CUDA graphs.  NULL is a no-op. */
void kd_destroy(kd_sim* sim);

/* Thread-local description of the last error ("" if none). */
const char* kd_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int kd_version(void);

#ifdef __cplusplus
}
#endif
#endif

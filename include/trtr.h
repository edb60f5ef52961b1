/*
 * trtr.h -- C ABI of the GB300 (sm_103a) TRT-R lattice Boltzmann library for the
 * convection-diffusion equation with variable coefficients
 *
 *     d_t phi + d_a(phi u_a) = d_a(kappa d_a phi) + S                    Eq. (1)
 *
 * (Yu, Qin, Yuan, Shu, arXiv 2312.10316).  One call of trtr_step advances every node of an
 * nx x ny periodic D2Q9 grid by the evolution equation of Sec. 2.2,
 *
 *   g_i(x + e_i dt, t + dt) = g_i^eq + (1 - 1/tau1) w_i H_ia B_a^neq / cs^2
 *                           + (1 - 1/tau2) w_i H_iab B_ab^neq / (2 cs^4)
 *                           + dt G_i + dt F_i + dt^2/2 d_t F_i               Eq. (14)
 *
 * with the third-order Hermite equilibrium (Eq. (6)), the first-order discrete-velocity
 * source F_i (Eq. (3)) and the space-derivative auxiliary term
 * G_i = w_i e_ia/cs^2 (1 - 1/(2 tau1)) phi u_b d_b u_a (Eq. (16)).  kappa = D(x) sets
 * tau1 = 1/2 + kappa / (cs^2 dt) (Sec. 2.4); tau2 is free, set either by the magic
 * parameter Lambda = (tau1 - 1/2)(tau2 - 1/2) (Eq. (28)) or given directly.
 *
 * Equation numbers count the paper's displayed equations in order.
 *
 * Conventions shared by every call:
 *  - Fields are row-major [ny][nx] doubles, x fastest; node (i, j) sits at
 *    (x0 + i dx, y0 + j dx).  Populations are [9][ny][nx] doubles in the D2Q9 order
 *    0:(0,0) 1:(1,0) 2:(-1,0) 3:(0,1) 4:(0,-1) 5:(1,1) 6:(-1,-1) 7:(1,-1) 8:(-1,1).
 *  - Physical units: u in length/time, D (= kappa) in length^2/time, S in 1/time.
 *  - `on_device` = 1: the pointer is CUDA device memory of the context's device, read
 *    (or written) on the context's stream during the call only; 0: host memory.  Caller
 *    memory is never retained.  All device buffers of a context are owned by the library.
 *  - Every call returns a trtr_status; nothing throws across the ABI.  TRTR_EINVAL: bad
 *    argument (nothing was changed); TRTR_ESTATE: call out of order (e.g. step before
 *    init); TRTR_ECUDA: a CUDA call failed (trtr_last_error has the text; the context
 *    should be destroyed); TRTR_EUNSTABLE: non-finite populations found by the stability
 *    check.
 *  - trtr_step only enqueues work on the context's stream: an asynchronous device fault
 *    surfaces as TRTR_ECUDA from the next call that synchronises (moments, mass, error,
 *    sample, get, save, sync).
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef TRTR_H
#define TRTR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TRTR_OK = 0,
    TRTR_EINVAL = 1,
    TRTR_ENOMEM = 2,
    TRTR_ECUDA = 3,
    TRTR_EUNSTABLE = 4,
    TRTR_ETIMEOUT = 5,
    TRTR_ESTATE = 6,
    TRTR_EBOUNDS = 7 /* bounds-checked builds only: a kernel access out of bounds was caught */
} trtr_status;

/* Storage / arithmetic of the populations.  F64: stored and computed in double.  F32:
 * stored and computed in float.  F16_OFS / BF16_OFS: stored as the half-precision offset
 * g_i - w_i phi_ref (rounded as trtr_params.rounding says), computed in float. */
typedef enum { TRTR_F64 = 0, TRTR_F32 = 1, TRTR_F16_OFS = 2, TRTR_BF16_OFS = 3 } trtr_precision;

typedef enum { TRTR_TAU2_MAGIC = 0, TRTR_TAU2_FIXED = 1 } trtr_tau2_mode;

/* d_b u_a in G_i: second-order central differences; at the first and last column/row
 * either wrapped periodically or one-sided (two-point), which is exact for a linear u
 * such as a rigid rotation that jumps across the periodic seam. */
typedef enum { TRTR_GRAD_PERIODIC = 0, TRTR_GRAD_ONESIDED_EDGE = 1 } trtr_grad_mode;

/* Source S: none; a field set with trtr_set_source (S^n, the previous step's field kept as
 * S^{n-1}); or the built-in manufactured source of the rotating pulse (trtr_set_pulse).
 * d_t F_i is (F^n - F^{n-1}) / dt.  The built-in source is a closed form of t, so its S^{n-1}
 * is S(t_n - dt) at the first step too; a field source has no predecessor at the first step
 * after init and takes F^{-1} := F^0. */
typedef enum { TRTR_SRC_NONE = 0, TRTR_SRC_FIELD = 1, TRTR_SRC_PULSE = 2 } trtr_src_mode;

/* Boundaries: periodic, or Dirichlet values phi_b held by non-equilibrium extrapolation (the
 * scheme of the paper's Sec. 3 runs).  With TRTR_BC_DIRICHLET_NEE the edge nodes (i = 0,
 * nx - 1; j = 0, ny - 1) are boundary nodes: after each step's streaming every population of
 * edge node b is replaced by g_i^eq(phi_b(b), u(b)) + g_i(f) - g_i^eq(phi(f), u(f)), f the next
 * node inward along the normal (diagonally at corners), g^eq the third-order Hermite
 * equilibrium of Eq. (6).  Needs nx, ny >= 3 and trtr_set_dirichlet before stepping; use
 * TRTR_GRAD_ONESIDED_EDGE for the velocity gradient at the edges. */
typedef enum { TRTR_BC_PERIODIC = 0, TRTR_BC_DIRICHLET_NEE = 1 } trtr_bc_mode;

/* Rounding of the stored F16_OFS / BF16_OFS offsets (not part of the paper's method, which is
 * stated in exact arithmetic).  STOCHASTIC (the default, 0): round up with probability equal
 * to the discarded fraction of the format's unit (the hardware's stochastic-rounding
 * conversion), fed with random bits that are a fixed hash of the node, the step number and the
 * population, so a run is reproducible bit for bit and independent of how its steps are split
 * into calls.  NEAREST: round to nearest even.  Nearest rounding of a smooth field repeats the
 * same error at neighbouring nodes and steps, so the error of phi grows linearly with the step
 * count (FP16: 1.8e-1 relative L2 after 10 000 steps of the 4096^2 pulse); stochastic rounding
 * makes each rounding error zero-mean and independent, the diffusion of the method damps them,
 * and the error stays near its first-step level (FP16: 2.6e-4 on the same run).  Ignored by the
 * F32 and F64 storages. */
typedef enum { TRTR_ROUND_STOCHASTIC = 0, TRTR_ROUND_NEAREST = 1 } trtr_rounding;

typedef struct {
    int nx, ny;         /* nodes, >= 1 each; ny * round_up(nx, 32) < 2^31              */
    double x0, y0;      /* coordinates of node (0, 0)                                  */
    double dx, dt;      /* lattice spacing and time step (> 0); c = dx / dt             */
    int precision;      /* trtr_precision                                               */
    double phi_ref;     /* offset level for the *_OFS storage (ignored otherwise)       */
    int tau2_mode;      /* trtr_tau2_mode                                               */
    double magic;       /* Lambda for TRTR_TAU2_MAGIC (the paper uses 1/12)             */
    double tau2;        /* tau2 for TRTR_TAU2_FIXED (> 1/2)                             */
    double tau1_const;  /* > 0: tau1 everywhere, the D field is ignored; 0: from D(x)   */
    int grad_mode;      /* trtr_grad_mode                                               */
    int src_mode;       /* trtr_src_mode                                                */
    int check_every;    /* > 0: trtr_step checks every k steps that all populations are
                           finite and returns TRTR_EUNSTABLE if not (synchronises)      */
    int bc_mode;        /* trtr_bc_mode                                                 */
    int rounding;       /* trtr_rounding of the 2-byte storages (0: stochastic)          */
} trtr_params;

typedef struct trtr_ctx trtr_ctx; /* opaque, library-owned */

/* Creates a context on the current CUDA device and allocates its device buffers (two
 * population arrays, the coefficient fields, source buffers, reduction scratch).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) that every later call of this
 * context enqueues on.  Validates the parameters (Sec. 2.2 lattice, Sec. 2.4 tau rules).
 * *out receives the context, or NULL on error. */
trtr_status trtr_create(const trtr_params* p, void* cuda_stream, trtr_ctx** out);

/* Frees every device and host buffer of the context after synchronising its stream.
 * NULL is accepted. */
trtr_status trtr_destroy(trtr_ctx* ctx);

/* Copies in the coefficient fields u_x, u_y and D (= kappa(x), Eq. (1)); D may be NULL when
 * tau1_const > 0.  S (may be NULL) sets the source field for TRTR_SRC_FIELD as by
 * trtr_set_source.  tau1 = 1/2 + 3 D dt / dx^2 must exceed 1/2 at every node: D must be
 * finite and > 0 everywhere, else TRTR_EINVAL with the fields unchanged (checked by a reduction
 * over the device copy on the context's stream, so the call synchronises when D is given).
 * Fields persist until set again. */
trtr_status trtr_set_fields(trtr_ctx* ctx, const double* ux, const double* uy, const double* D,
                            const double* S, int on_device);

/* TRTR_SRC_FIELD: sets S^n, the source of the next step (Eq. (3)); the source used by the
 * previous step becomes S^{n-1}.  Before the first step after init, S^{n-1} := S^n unless
 * trtr_set_source_prev gives it. */
trtr_status trtr_set_source(trtr_ctx* ctx, const double* S, int on_device);

/* TRTR_SRC_FIELD: sets S^{n-1} of the next step explicitly, for a source known in closed form
 * at t_n - dt (the d_t F term of Eq. (14) at the first step).  Needs a current source
 * (trtr_set_source) and is undone by trtr_init_equilibrium / trtr_set_populations, so call it
 * after those.  S: [ny][nx], host or device. */
trtr_status trtr_set_source_prev(trtr_ctx* ctx, const double* S, int on_device);

/* TRTR_BC_DIRICHLET_NEE: the boundary values phi_b imposed after each following step's
 * streaming, i.e. phi at t_{n+1} for the step from t_n.  phi_b: [ny][nx] (host or device);
 * only the edge nodes are read (copied, so the caller may reuse the array at once; host input
 * synchronises the stream).  Values stay until set again: call it before every
 * trtr_step(ctx, 1) for time-dependent values. */
trtr_status trtr_set_dirichlet(trtr_ctx* ctx, const double* phi_b, int on_device);

/* Rotating, spreading Gaussian pulse (the benchmark family of Sec. 3 on this periodic box):
 * u = omega (-y, x); D = D0 (1 + D_amp sin(pi x) sin(pi y)); phi_a(x, t) =
 * (s0^2/s^2) exp(-|x - c(t)|^2 / (2 s^2)), s^2 = s0^2 + 2 D0 t, c(t) = R(omega t)(xc, yc).
 * Fills u and D on the device, and makes the manufactured source
 * S = -div((D - D0) grad phi_a) (TRTR_SRC_PULSE), trtr_init_equilibrium(ctx, NULL, 0) and
 * trtr_error_vs_pulse refer to this pulse.  sigma0 > 0, D0 >= 0. */
trtr_status trtr_set_pulse(trtr_ctx* ctx, double omega, double xc, double yc, double sigma0, double D0,
                           double D_amp);

/* Initial condition g_i = g_i^eq(phi_0, u) (Sec. 3) and step counter n = 0.  phi0: [ny][nx];
 * NULL = the pulse's phi_a(x, 0) (needs trtr_set_pulse).  Needs the fields. */
trtr_status trtr_init_equilibrium(trtr_ctx* ctx, const double* phi0, int on_device);

/* Advances n >= 0 time steps of Eq. (14): one fused pull-stream + collide kernel per step on
 * the context's stream (plus the boundary pass with TRTR_BC_DIRICHLET_NEE), ping-pong buffers,
 * no host synchronisation (unless check_every).  With FP32 storage, or FP16 / BF16 offset
 * storage on a grid of even nx, periodic boundaries and src_mode NONE or PULSE, pairs of steps
 * run as one launch of the two-step kernel (the same arithmetic and roundings, the same results
 * bit for bit; populations read and written once per two steps; see
 * trtr_set_steps_per_launch); an odd last step, or a pair whose middle step is a check_every
 * point, runs one step per launch.  Short launches use programmatic dependent launch: each
 * waits for the work before it on the stream before reading its results. */
trtr_status trtr_step(trtr_ctx* ctx, long n);

/* k = 2 (the default): trtr_step uses the two-step kernel where it applies; k = 1: one step per
 * launch always.  TRTR_EINVAL for other k. */
trtr_status trtr_set_steps_per_launch(trtr_ctx* ctx, int k);

/* The steps one launch of trtr_step advances where it can on this context: 2 when the two-step
 * kernel applies (FP32, or FP16 / BF16 with even nx; periodic; src_mode NONE or PULSE; not
 * disabled), else 1. */
trtr_status trtr_get_steps_per_launch(const trtr_ctx* ctx, int* k);

/* phi(x, t_n) = sum_i g_i(x, t_n) of the pre-collision populations (B_0^neq = 0, Sec. 2.2),
 * written as doubles [ny][nx].  Synchronises. */
trtr_status trtr_moments(trtr_ctx* ctx, double* phi_out, int on_device);

/* FP64 sum over nodes of phi(x, t_n) (conserved when S = 0).  Synchronises. */
trtr_status trtr_mass(trtr_ctx* ctx, double* sum_phi);

/* RMS error E_r = sqrt(sum (phi - phi_a)^2 / (nx ny)) (Eq. (33)) and relative L2 error
 * ||phi - phi_a|| / ||phi_a|| against the pulse's closed form at t_n = n dt, accumulated in
 * FP64.  Needs trtr_set_pulse.  Synchronises. */
trtr_status trtr_error_vs_pulse(trtr_ctx* ctx, double* rms, double* rel_l2);

/* As trtr_error_vs_pulse against a given field phi_ref [ny][nx] (rel_l2 falls back to the
 * absolute L2 norm when phi_ref is all zero). */
trtr_status trtr_error_vs(trtr_ctx* ctx, const double* phi_ref, int on_device, double* rms, double* rel_l2);

/* Pre-collision populations g_i(x, t_n) as doubles [9][ny][nx].  Synchronises. */
trtr_status trtr_get_populations(trtr_ctx* ctx, double* g_out, int on_device);

/* Sets the pre-collision populations g_i(x, t_n) from doubles [9][ny][nx] (rounded to the
 * storage precision) and the step counter n = step >= 0; S^{n-1} := S^n for the next step. */
trtr_status trtr_set_populations(trtr_ctx* ctx, const double* g, int on_device, long step);

/* g_i(x, t_n) at `count` node indices k = j * nx + i (host array), written to host
 * out[count][9].  Synchronises. */
trtr_status trtr_sample_populations(trtr_ctx* ctx, const long* nodes, int count, double* out);

/* Step counter n and time t_n = n dt. */
trtr_status trtr_time(const trtr_ctx* ctx, long* step, double* t);

/* Checkpoint of the state (populations in storage precision, step counter, source
 * buffers).  host_buf == NULL: *bytes receives the size needed.  Otherwise *bytes is the
 * buffer size on input and the bytes written on output.  Synchronises. */
trtr_status trtr_save(trtr_ctx* ctx, void* host_buf, size_t* bytes);

/* Restores a checkpoint written by trtr_save from a context with the same nx, ny and
 * precision; fields and pulse are not part of it. */
trtr_status trtr_load(trtr_ctx* ctx, const void* host_buf, size_t bytes);

/* Waits for the context's stream and reports any pending CUDA error, or TRTR_ETIMEOUT if a
 * step kernel gave up one of its bounded waits for its TMA loads (about 2 s of SM clock: the
 * context's flag is then cleared, so the context stays usable). */
trtr_status trtr_sync(trtr_ctx* ctx);

/* Failure-detection check (the paper has no counterpart): launches one block whose bounded
 * wait on a barrier that nothing ever completes gives up after `cycles` SM clock cycles
 * (1 .. 2^31), through the same path as a step kernel's wait on its loads, and synchronises.
 * Returns TRTR_ETIMEOUT when that path works; the flag is cleared as it is reported, so the
 * next calls on the context run normally.  No copy is in flight, so nothing is left behind. */
trtr_status trtr_check_timeout_path(trtr_ctx* ctx, long long cycles);

/* Number of kernels the library enqueued on this context since creation (launch count). */
trtr_status trtr_launch_count(const trtr_ctx* ctx, long* launches);

/* ---- Gradients with respect to the diffusivity field (discrete adjoint) ------------------
 * For J any function of the final phi, dJ/dD(x) through n steps of Eq. (14): the exact
 * derivative of the discrete step (a discrete adjoint), which the paper does not treat.
 * D enters each step through tau1 = 1/2 + 3 D dt/dx^2 (Sec. 2.4) and, with the magic
 * parameter, through tau2 (Eq. (28)).  Scope: S = 0 (src_mode TRTR_SRC_NONE) and periodic
 * boundaries (TRTR_EINVAL otherwise). */

/* Advances n >= 1 steps from the current state, keeping a copy of the state every
 * `interval` steps (0: ceil(sqrt(n))), and remembers the run for trtr_adjoint.  Allocates
 * about (n/interval + interval) population arrays of device memory (freed by the next
 * record or by trtr_destroy). */
trtr_status trtr_forward_record(trtr_ctx* ctx, long steps, int interval);

/* Backward sweep of the recorded run: dJ_dphi = dJ/dphi(x, t_end) [ny][nx] (host or device);
 * grad_D receives dJ/dD(x) [ny][nx] in physical units (host or device).  Each segment between
 * checkpoints is recomputed once from its checkpoint.  The context must still be at the end
 * of the recorded run (TRTR_ESTATE otherwise); its state is not changed.  Synchronises. */
trtr_status trtr_adjoint(trtr_ctx* ctx, const double* dJ_dphi, int on_device, double* grad_D, int grad_on_device);

/* ---- Batched instances ----------------------------------------------------------------
 * Many independent problems of uneven sizes advanced together, each by the same step of
 * Eq. (14).  The paper solves one problem at a time; this is a throughput mode of its step.
 * Persistent kernel launches walk a work-list of (instance, tile) pairs spanning every
 * instance: one time step per launch, or two (the two-step kernel) where every instance has
 * FP32 storage, or 2-byte storage with even nx;
 * trtr_batch_step replays two-launch CUDA graphs of them.
 * Each instance is an ordinary context (trtr_batch_instance gives it out for queries). */
typedef struct {
    trtr_params p;  /* the instance's lattice and options.  precision: the same for every
                       instance, TRTR_F32, TRTR_F16_OFS or TRTR_BF16_OFS; src_mode: NONE or
                       PULSE (the manufactured source of its pulse); bc_mode: PERIODIC;
                       rounding: the same for every instance                             */
    double omega, xc, yc, sigma0, D0, D_amp; /* its pulse, as for trtr_set_pulse          */
} trtr_instance;

typedef struct trtr_batch trtr_batch; /* opaque, library-owned */

/* Creates one context per instance on cuda_stream (NULL: the batch creates its own stream;
 * graphs cannot be captured on the legacy default stream), fills each with its pulse's
 * fields and initial condition g = g^eq(phi_a(x, 0), u), and builds the work-list of the
 * default configuration.  On error nothing is left allocated. */
trtr_status trtr_batch_create(const trtr_instance* inst, int count, void* cuda_stream, trtr_batch** out);

/* Frees the batch and its instance contexts.  NULL is accepted. */
trtr_status trtr_batch_destroy(trtr_batch* b);

/* Number of launch configurations (tile shape x CTA-to-tile schedule) and their names. */
int trtr_batch_config_count(void);
const char* trtr_batch_config_name(int config);

/* Autotuner: times every configuration (of the one-step kernel, one step per launch) over
 * trial_steps (>= 2) steps with CUDA events and keeps the fastest; *config_out (may be NULL) receives it and ms_out (may be NULL, else
 * trtr_batch_config_count() floats) the milliseconds per step of each.  A batch tuned at
 * step 0 gets its step-0 state back afterwards, whatever set it (the pulse, a phi0 or the
 * caller's populations): the tuner keeps a temporary device copy of every instance's
 * populations for the trials (TRTR_ENOMEM if that copy cannot be allocated, nothing changed).
 * At a later step the trial steps advance every instance.  Synchronises. */
trtr_status trtr_batch_tune(trtr_batch* b, int trial_steps, int* config_out, float* ms_out);

/* Selects a configuration explicitly. */
trtr_status trtr_batch_set_config(trtr_batch* b, int config);

/* Advances every instance by n >= 0 steps (asynchronous on the batch's stream).  Where the
 * two-step kernel applies (every instance FP32, or 2-byte with even nx), pairs of steps run as
 * launches of it over a work-list of its tiles (the same results bit for bit; see
 * trtr_batch_set_steps_per_launch), the other steps
 * with the configured one-step kernel.  Instances must not be stepped through their own
 * contexts in between (TRTR_ESTATE). */
trtr_status trtr_batch_step(trtr_batch* b, long n);

/* k = 2 (the default): trtr_batch_step runs pairs of steps with the two-step kernel where it
 * applies (FP32 instances, or 2-byte instances of even nx); k = 1: every step with the
 * configured one-step kernel.
 * TRTR_EINVAL for other k. */
trtr_status trtr_batch_set_steps_per_launch(trtr_batch* b, int k);

/* The steps one launch of trtr_batch_step advances where it can: 2 when the two-step kernel
 * applies to the batch and is not disabled, else 1.  TRTR_EINVAL for NULL arguments. */
trtr_status trtr_batch_get_steps_per_launch(const trtr_batch* b, int* k);

/* Waits for the batch's stream; TRTR_ETIMEOUT if a step kernel gave up a bounded wait
 * (TRTR_EBOUNDS in the bounds-checked build if a kernel access out of bounds was caught). */
trtr_status trtr_batch_sync(trtr_batch* b);

/* The context of instance k (owned by the batch): moments, mass, error, populations. */
trtr_status trtr_batch_instance(trtr_batch* b, int k, trtr_ctx** ctx);

/* Instance count, total nodes, step counter and current configuration (any may be NULL). */
trtr_status trtr_batch_info(const trtr_batch* b, int* count, long long* nodes, long* step, int* config);

/* Largest grid height (rows) that trtr_phi_sums_noalloc accepts. */
#define TRTR_NOALLOC_MAX_ROWS 16384

/* The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory: code whose device memory is owned by another allocator (for
 * example a framework's caching allocator that has reserved nearly all of HBM, so a
 * cudaMalloc would fail or fragment it), latency-critical loops where the implicit
 * synchronisation of cudaMalloc/cudaFree is not acceptable, and plug-in hosts whose policy
 * forbids libraries from allocating.  It allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library call.
 *
 * Computes, in FP64, out[0] = sum over nodes of phi = sum_i g_i, and, when phi_ref is not
 * NULL, out[1] = sum (phi - phi_ref)^2 and out[2] = sum phi_ref^2 (else both 0), from which
 * the caller forms the mass, the RMS error sqrt(out[1] / (nx ny)) and the relative L2 error
 * sqrt(out[1] / out[2]).
 *   g       device memory, [9][ny][nx] doubles: pre-collision populations (the layout that
 *           trtr_get_populations writes);
 *   phi_ref device memory, [ny][nx] doubles, or NULL;
 *   out     device memory, 3 doubles, written by the last kernel of the call;
 *   cuda_stream  a cudaStream_t (NULL = legacy default stream) the two kernels run on; the
 *           call returns once they are enqueued.
 * Its scratch is a fixed array of TRTR_NOALLOC_MAX_ROWS x 3 doubles (384 KiB) in static
 * device memory, which every device that loads the library holds until the process exits.
 * ny > TRTR_NOALLOC_MAX_ROWS, nx < 1, ny < 1 or a NULL g / out return TRTR_EINVAL with
 * nothing enqueued.  The first call on a device (with that device current) looks up the
 * array's device address and keeps it for the life of the process; make that first call
 * before any stream capture, and make no call on a device after resetting it
 * (cudaDeviceReset frees the array and leaves the kept address stale).  An error already
 * pending in the CUDA runtime when the call starts is returned as TRTR_ECUDA, left pending,
 * with nothing enqueued.  Every call
 * shares the array and it keeps the last call's contents (each call overwrites rows
 * [0, ny) before reading them, so nothing needs clearing); calls that overlap on the GPU --
 * on different streams, or from several host threads -- race on it and must be serialised
 * by the caller.  TRTR_ECUDA: the address lookup or a launch failed. */
trtr_status trtr_phi_sums_noalloc(const double* g, int nx, int ny, const double* phi_ref, double* out,
                                  void* cuda_stream);

/* Static text of a status code. */
const char* trtr_status_str(trtr_status s);

/* Last error message of the context ("" if none); valid until the next call on it. */
const char* trtr_last_error(const trtr_ctx* ctx);

/* The library's D2Q9 table: ex[9], ey[9] (integers) and w[9]. */
void trtr_d2q9(int* ex, int* ey, double* w);

/* ABI version (incremented on incompatible change). */
int trtr_abi_version(void);

/* ---- Bounds-checked debug build ---------------------------------------------------------
 * The library built with TRTR_BOUNDS_CHECK=1 (libtrtr_checked.so) checks its kernels' memory
 * accesses against the ghosted plane layout: every plane index, the two-node stores, the bulk
 * row copies (inside the interior row, 16-byte aligned addresses and size) and the TMA load
 * coordinates (x times the element size a multiple of 16 bytes, 128-byte aligned destination).
 * A bad access is recorded and skipped (or kept inside the ghost frame); nothing traps.  The
 * next call that synchronises a context's stream (or trtr_batch_sync) then returns
 * TRTR_EBOUNDS with the first access in trtr_last_error.  The default build compiles none of
 * these checks. */

/* 1 in the bounds-checked build, 0 in the default build. */
int trtr_bounds_checked(void);

/* Synchronises the current device, then returns the record of every kernel since the last
 * report and clears it: out[0] = accesses caught, out[1] = kind of the first (1 plane index,
 * 2 two-node store, 3 bulk row copy, 4 TMA load), out[2] = its column i | row j << 32 (for a
 * TMA load, x | y << 32).  The default build writes zeros.  TRTR_EINVAL: out is NULL;
 * TRTR_ECUDA: a CUDA call failed. */
trtr_status trtr_bounds_report(unsigned long long out[3]);

/* Checks the recording path of the bounds-checked build without a bad access: one thread gives
 * the checks four bad arguments (a plane index one column past the ghost frame, a TMA x
 * coordinate of 12 bytes, a TMA destination off its 128-byte boundary, a bulk row copy past
 * the row end) and accesses nothing with them.  Returns TRTR_EBOUNDS in the checked build
 * (trtr_last_error: 4 accesses, the first of kind 1 at (nx + 2, 0), the population planes
 * having two ghost columns), TRTR_OK in the default
 * build; the record is cleared either way.  Needs a created context (any state). */
trtr_status trtr_check_bounds_path(trtr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TRTR_H */

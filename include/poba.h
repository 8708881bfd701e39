/*
 * poba.h -- C ABI of the GB300 Power Bundle Adjustment library (libpoba.so).
 *
 * The library solves bundle-adjustment problems in the BAL camera model (Sec. 4: d_p = 9
 * camera parameters [w0 w1 w2 t0 t1 t2 f k1 k2], 3 landmark coordinates) with
 * Levenberg-Marquardt, where each damped normal equation (Sec. 4.1, eq. `normal`) is reduced to
 * the camera system S dx_p = -b~ (Sec. 4.2, eqs. `Sx`, `Schur`) and solved matrix-free by the
 * truncated power series x(m) = -sum_{i<=m} (U^-1 W V^-1 W^T)^i U^-1 b~ (Sec. 4.3, eqs.
 * `S_approx`, `x_approx`) with the stop rule (i+1)||x(i)-x(i-1)|| / ||x(i)|| < eps (eq.
 * `qcriterion`).  Every step runs in CUDA kernels for sm_103a on one GPU.
 *
 * Conventions shared by all entry points
 *  - Status: every call returns a ba_status; nothing throws across the ABI.  On an error the
 *    handle stays usable unless the status is BA_ERR_CUDA (a CUDA runtime error other than an
 *    allocation failure, after which the handle should be destroyed).  ba_last_error() gives a
 *    one-line description of the most recent failure on the calling thread.
 *  - Ownership: ba_create copies every input; the library owns all device memory of a handle
 *    and frees it in ba_destroy.  Output pointers belong to the caller.
 *  - Pointer kinds: ptr_kind 0 = host memory, 1 = device memory of the handle's GPU.
 *  - Streams: all GPU work of a handle is ordered on the handle's CUDA stream (the stream given
 *    at creation, or a stream the library creates when NULL).  Calls that return host scalars
 *    synchronise that stream before returning; others do not.
 *  - Threading: a handle must not be used from two threads at once; handles are independent.
 *  - Layout: cams [n_cams][9], lms [n_lms][3], obs [n_obs][2], row-major float64; index arrays
 *    int32.  Observations may be given in any order; the library reorders them internally and
 *    every per-observation output is returned in the caller's original order.
 */
#ifndef POBA_H
#define POBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_handle ba_handle; /* opaque, owned by the library */

typedef enum {
  BA_OK = 0,
  BA_ERR_INVALID_ARG = 1,    /* bad size, pointer, index, option, or unsupported shape */
  BA_ERR_CUDA = 2,           /* CUDA runtime failure (message in ba_last_error) */
  BA_ERR_OOM = 3,            /* device allocation failed */
  BA_ERR_NOT_SPD = 4,        /* a damped U or V block had a non-positive Cholesky pivot */
  BA_ERR_NONFINITE = 5,      /* non-finite input, residual, cost or step */
  BA_ERR_NOT_LINEARIZED = 6, /* a solve was requested before ba_linearize */
  BA_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up (a grid barrier of the
                                persistent series kernel waited longer than its limit) */
  BA_ERR_CHECK = 8           /* debug builds (libpoba_checks.so): a device-side index check or
                                a buffer guard failed (message in ba_last_error) */
} ba_status;

typedef enum {
  BA_FP64 = 0,      /* residuals, Jacobians and series matvecs in float64 */
  BA_FP32_BULK = 1  /* residuals, Jacobians and series matvecs in float32 with float32 sums
                       inside a landmark / camera-tile segment and float64 across segments;
                       block inverses, cost, model decrease and gain ratio stay float64 */
} ba_precision;

typedef struct {
  int32_t n_cams, n_lms, n_obs; /* n_cams >= 1, n_lms >= 1, n_obs >= 0 */
  const double* cams;           /* [n_cams][9] initial cameras */
  const double* lms;            /* [n_lms][3] initial landmarks */
  const double* obs;            /* [n_obs][2] pixel observations */
  const int32_t* cam_idx;       /* [n_obs] camera of each observation, 0 <= . < n_cams */
  const int32_t* lm_idx;        /* [n_obs] landmark of each observation, 0 <= . < n_lms */
  const double* weights;        /* [n_obs] observation weights > 0, or NULL for all ones;
                                   F = 1/2 sum_o w_o ||r_o||^2 */
  int32_t ptr_kind;             /* 0: all arrays above are host memory, 1: device memory */
  int32_t precision;            /* ba_precision */
  void* cuda_stream;            /* cudaStream_t to order work on, or NULL */
} ba_problem_desc;

typedef struct {
  double lambda0;       /* initial damping, Sec. 5.1: 1e-4 */
  double func_tol;      /* relative function tolerance, Sec. 5.1: 1e-6 */
  double eps;           /* series stop threshold of eq. `qcriterion`, Sec. 5.1: 0.01 */
  int32_t max_lm;       /* LM iteration cap, Sec. 5.1: 50 */
  int32_t max_inner;    /* cap on series terms beyond x(0), Sec. 5.1: 20 */
  int32_t damping_mode; /* 0: D^T D = diag(J^T J) clamped to [1e-6, 1e32]; 1: D = I */
  int32_t series_exec;  /* how the series loop runs: 0 one launch per kernel, 1 the same launches
                           replayed as a captured CUDA graph, 3 one persistent cooperative kernel
                           for all terms with bounded grid barriers, 4 (BA_FP32_BULK; else as 3)
                           the persistent kernel with each chunk's inputs staged in shared
                           memory by bulk asynchronous copies issued one chunk ahead, 5 one
                           persistent cooperative kernel without grid barriers: blocks take
                           (term, group) tickets, a group starts once the previous term's
                           update of its cameras is published, and the block that completes a
                           camera's rows of a term runs that camera's update (and the block
                           that completes a problem's cameras its stop rule), so blocks run
                           ahead into the next term instead of waiting for the slowest group, 2
                           (default) the handle's schedule (ba_set_schedule / ba_autotune; at
                           creation 3 at the largest residency, 4 blocks per SM in BA_FP32_BULK,
                           3 in BA_FP64).  A device that cannot run a persistent form falls back
                           (4 and 5 to 3, 3 to 1: all blocks must be co-resident), and so do
                           forms 4 and 5 on a problem with tracks of more than 256 observations
                           (or, in BA_FP64, a landmark seen by more than 96 cameras).
                           All forms give bitwise-equal results for the handle's series
                           schedule. */
} ba_options;

typedef struct {
  int32_t inner_iters; /* m: number of applications of U^-1 W V^-1 W^T performed */
  int32_t stopped;     /* 1 if eq. `qcriterion` fired (or ||x|| = 0), 0 if m hit max_inner */
  double stop_value;   /* (m+1) ||x(m)-x(m-1)|| / ||x(m)|| at the last term (inf if m = 0) */
  double x_norm;       /* ||x(m)||_2 */
  double lambda;       /* damping the blocks were built with */
} ba_series_info;

typedef struct {
  double cost_before;     /* F(x) before the step */
  double cost_after;      /* F(x + dx) of the trial step */
  double lambda;          /* damping used for this step */
  double gain_ratio;      /* (F(x) - F(x+dx)) / (L(0) - L(dx)) */
  double model_decrease;  /* L(0) - L(dx) = 1/2||r||^2 - 1/2||r + J dx||^2 */
  double stop_value;      /* series stop value (see ba_series_info) */
  int32_t accepted;       /* 1 if the step was applied */
  int32_t inner_iters;    /* series terms used */
  int32_t converged;      /* 1 if accepted with relative decrease < func_tol */
  int32_t iteration;      /* LM iteration index of this step (0-based) */
  int32_t not_spd;        /* 1 if a damped block failed its Cholesky factorisation: the
                             iteration had no step and was rejected (cost_after is NaN) */
} ba_step_info;

/* Fill *opts with the defaults of Sec. 5.1 (lambda0 1e-4, func_tol 1e-6, eps 0.01, max_lm 50,
 * max_inner 20, damping_mode 0, series_exec 2).  Returns BA_ERR_INVALID_ARG if opts is NULL. */
ba_status ba_default_options(ba_options* opts);

/* Create a problem handle (Sec. 4: state x = (x_p, x_l), residuals r(x)).  Copies and
 * validates the inputs (sizes, index ranges, finiteness, weights > 0), sorts observations by
 * landmark, orders landmarks for camera locality and builds the tile schedule, then allocates
 * all device memory once.  A landmark with more than 256 observations (a long track) is split
 * into near-equal pieces of at most 256 observations, which the kernels treat as landmarks
 * holding copies of its state; the landmark-side sums (V, b_l, the series' J_l^T J_p t and the
 * back-substitution's) are added over the pieces in piece order, so the results are those of
 * the unsplit problem.  opts may be NULL for the defaults.  Errors: BA_ERR_INVALID_ARG (bad
 * sizes, NULL pointers, out-of-range index),
 * BA_ERR_NONFINITE (non-finite input), BA_ERR_OOM, BA_ERR_CUDA.  *out is NULL on error. */
ba_status ba_create(const ba_problem_desc* desc, const ba_options* opts, ba_handle** out);

/* Replace the options of a handle (takes effect at the next call). */
ba_status ba_set_options(ba_handle* h, const ba_options* opts);

/* Linearise at the current state (Sec. 4.1): residuals r, Jacobians J_p (2x9) and J_l (2x3)
 * per observation, and the undamped blocks U = J_p^T J_p, V = J_l^T J_l, b_p = J_p^T r,
 * b_l = J_l^T r (eq. `normal`).  *cost_out (may be NULL) receives 1/2||r||^2 computed from the
 * linearisation residuals (in the handle's precision); synchronises only if cost_out != NULL.
 * Errors: BA_ERR_CUDA. */
ba_status ba_linearize(ba_handle* h, double* cost_out);

/* Solve the damped normal equation at the current linearisation with damping `lambda`:
 * U_lambda, V_lambda and their Cholesky inverses (Sec. 4.1), b~ (Sec. 4.2), the power series
 * x(m) (Sec. 4.3) with the handle's eps / max_inner, and the back-substitution
 * dx_l = -V_lambda^-1 (b_l + W^T dx_p) (Sec. 4.2; sign derived from eq. `normal`).  The step
 * stays on the device (read it with ba_get_step).  info may be NULL (then nothing is
 * synchronised).  Errors: BA_ERR_NOT_LINEARIZED, BA_ERR_INVALID_ARG (lambda <= 0 or not
 * finite), BA_ERR_NOT_SPD and BA_ERR_TIMEOUT (reported when info != NULL), BA_ERR_CUDA. */
ba_status ba_solve_schur_power(ba_handle* h, double lambda, ba_series_info* info);

/* One Levenberg-Marquardt iteration (Sec. 5.1 "LM loop"): linearise if the state changed,
 * damp with the handle's current lambda, solve with the power series, back-substitute,
 * evaluate F(x + dx) and the model decrease, accept iff F decreased and the model decrease is
 * positive, update lambda (accept: lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2; reject:
 * lambda *= nu, nu *= 2; clamp to [1e-10, 1e32]) and apply an accepted step.  Sec. 4.1 takes
 * the damped blocks to be positive definite; when one still fails its Cholesky factorisation
 * in floating point (damping that underflows, a nearly singular block), the iteration has no
 * step: it is rejected like a step that did not decrease F, lambda grows, and info->not_spd = 1
 * -- this is not an error.  Synchronises once.  info may be NULL.  Errors: BA_ERR_NONFINITE
 * (non-finite cost at the current state), BA_ERR_TIMEOUT, BA_ERR_CUDA. */
ba_status ba_lm_step(ba_handle* h, ba_step_info* info);

/* LM steps as one CUDA graph (no counterpart in the paper).  With step graphs on (the default)
 * the first LM step captures the device part of a step -- the linearisation, gated on a device
 * flag that the previous step's decision raises when a step was accepted; damping and
 * inversion; b~, x(0), the series in the handle's form (the persistent kernel included) and the
 * back-substitution; the trial cost, the decision and the update; the copies of the step's
 * records to pinned host memory -- and every step replays it: one graph launch, then one
 * synchronisation to read the records.  The capture is redone when the options, the schedule,
 * the timing switch or the barrier limit change.  Results equal the step-by-step launches bit
 * for bit.  If the device cannot capture a form, the handle turns graphs off and launches the
 * kernels one by one.  ba_get_step_graph: *enabled (may be NULL) the switch,
 * *kernels_per_step (may be NULL) the kernel launches one replay makes (0: nothing captured
 * yet). */
ba_status ba_set_step_graph(ba_handle* h, int32_t enable);
ba_status ba_get_step_graph(ba_handle* h, int32_t* enabled, int32_t* kernels_per_step);

/* Run ba_lm_step until convergence (func_tol) or max_lm iterations.  trace may be NULL or
 * hold max_lm entries; *n_steps (may be NULL) receives the number of iterations run. */
ba_status ba_lm_solve(ba_handle* h, ba_step_info* trace, int32_t* n_steps);

/* F(x) = 1/2 sum_o w_o ||r_o(x)||^2 at the current state (Sec. 4), always in float64 with a
 * fixed-order reduction.  Synchronises.  Errors: BA_ERR_INVALID_ARG (cost_out NULL), CUDA. */
ba_status ba_cost(ba_handle* h, double* cost_out);

/* Copy the current cameras [n_cams][9] and landmarks [n_lms][3] (caller's landmark order) to
 * host (ptr_kind 0) or device (1) memory.  Either pointer may be NULL.  Synchronises. */
ba_status ba_get_params(ba_handle* h, double* cams, double* lms, int32_t ptr_kind);

/* Overwrite the current state (same layout as ba_get_params); marks the linearisation stale
 * and leaves lambda unchanged.  A state equal to the current one in every bit (for instance the
 * state a rejected LM step left, read back with ba_get_params) changes nothing: the
 * linearisation and the cost at that state stay in place.  Synchronises (the finiteness check).
 * Errors: BA_ERR_NONFINITE, BA_ERR_INVALID_ARG. */
ba_status ba_set_params(ba_handle* h, const double* cams, const double* lms, int32_t ptr_kind);

/* Copy the last solve's step dx_p [n_cams][9] and dx_l [n_lms][3] (caller's order).
 * Synchronises. */
ba_status ba_get_step(ba_handle* h, double* dx_p, double* dx_l, int32_t ptr_kind);

/* Copy the last linearisation in the caller's observation order, converted to float64:
 * r [n_obs][2], J_p [n_obs][2][9], J_l [n_obs][2][3] (weights applied as sqrt(w)).  Any pointer
 * may be NULL.  Errors: BA_ERR_NOT_LINEARIZED. */
ba_status ba_get_linearization(ba_handle* h, double* r, double* Jp, double* Jl, int32_t ptr_kind);

/* Copy the last linearisation's undamped blocks: U [n_cams][9][9], V [n_lms][3][3] (caller's
 * landmark order), b_p [n_cams][9], b_l [n_lms][3].  Any pointer may be NULL. */
ba_status ba_get_blocks(ba_handle* h, double* U, double* V, double* b_p, double* b_l, int32_t ptr_kind);

/* LM state for checkpoint / resume: damping lambda, its growth factor nu, the iteration
 * counter and the current cost.  ba_set_lm_state marks nothing stale. */
ba_status ba_get_lm_state(ba_handle* h, double* lambda, double* nu, int32_t* iteration, double* cost);
ba_status ba_set_lm_state(ba_handle* h, double lambda, double nu, int32_t iteration);

/* Device bytes held by the handle (all buffers of the arena). */
ba_status ba_memory_footprint(ba_handle* h, uint64_t* bytes);

/* Number of kernel launches the handle has issued since creation (each graph replay counts
 * its kernel nodes). */
ba_status ba_kernel_launches(ba_handle* h, uint64_t* count);

/* Kernel timing (CUDA events recorded on the handle's stream around each kernel class, also
 * inside the replayed series graph).  Classes: 0 linearise (camera prep, residual/Jacobian/
 * block kernel, camera block reduce), 1 damp and invert, 2 reduced RHS and x(0) (tile + camera
 * kernel), 3 series tile kernel (one per executed term), 4 series camera kernel (one per
 * executed term), 5 back-substitution with model decrease, 6 LM evaluation (trial camera prep,
 * cost, decision, apply).  Times are collected by the calls that synchronise (ba_lm_step,
 * ba_solve_schur_power with info); series terms skipped after the stop rule fired are not
 * counted.  Enabling resets the totals; timing adds a few event records per kernel. */
#define BA_TIMING_CLASSES 7
typedef struct {
  double ms[BA_TIMING_CLASSES];      /* summed device time per class */
  uint64_t count[BA_TIMING_CLASSES]; /* timed launches (or launch groups) per class */
} ba_timing;
ba_status ba_set_timing(ba_handle* h, int32_t enable);
ba_status ba_get_timing(ba_handle* h, ba_timing* out);

/* Allocation-free cost evaluation.  The paper has no counterpart: this entry point exists for
 * callers that must not let a library allocate device memory -- cudaMalloc and cudaFree
 * synchronise the whole device, which latency-bound loops cannot afford, and processes whose
 * device memory is owned by another allocator (a framework's caching allocator, or a budget
 * fixed up front) must not take memory behind its back.
 *
 * Computes *cost_out = F(x) = 1/2 sum_o w_o ||r_o(x)||^2 in float64, like ba_cost, but without a
 * handle: every pointer is device memory of the current device (cams [n_cams][9], lms
 * [n_lms][3], obs [n_obs][2] 16-byte aligned, cam_idx / lm_idx [n_obs], weights [n_obs] or
 * NULL, cost_out one double).  Work is queued on cuda_stream (NULL: the legacy default stream)
 * and the call returns without synchronising.  It calls no cudaMalloc / cudaFree: its scratch
 * (camera rotation records and per-block sums) is one fixed device array of
 * BA_NOALLOC_MAX_CAMS * 25 + 2048 doubles (about 816 KiB) that every GPU using the library
 * holds until the process exits.  n_cams above BA_NOALLOC_MAX_CAMS is rejected with
 * BA_ERR_INVALID_ARG.  Each call looks up the array's address in the current device's context
 * (the first call on a device loads the module, so make it outside any stream capture); a
 * context that was reset between calls is therefore safe.  All calls
 * share the one array and it keeps the last call's contents; every entry a call reads is
 * written earlier in the same call.  Calls that overlap on the GPU (other streams, other host
 * threads) race on the array: order them.  An out-of-range index makes *cost_out NaN. */
#define BA_NOALLOC_MAX_CAMS 4096
ba_status ba_cost_noalloc(int32_t n_cams, int32_t n_lms, int32_t n_obs, const double* cams,
                          const double* lms, const double* obs, const int32_t* cam_idx,
                          const int32_t* lm_idx, const double* weights, double* cost_out,
                          void* cuda_stream);

/* ---- Batches of independent problems ---------------------------------------------------
 * Sec. 5.3 (Power Stochastic BA, PoST) solves many small, independent sub-problems -- camera clusters
 * of at most 100 cameras -- each with the power-series solver and the Sec. 5.1 settings.  A
 * batch handle holds P such problems in one arena; every kernel of a step covers all P at once
 * (one persistent series launch for the whole batch), while each problem keeps its own LM
 * record (lambda, nu, cost, gain ratio, accept), its own series stop rule and its own
 * convergence test.  Results per problem equal those of a handle created for that problem
 * alone, bit for bit.
 *
 * ba_create_batch: descs[0 .. n_problems-1] as for ba_create, each problem's indices local to
 * that problem (0 <= cam_idx < its n_cams).  All problems need the same precision; weights may
 * be NULL for some problems (ones) and not others; descs[0].cuda_stream orders the batch.
 * The batch behaves as one problem whose cameras, landmarks and observations are the
 * problems' concatenated in order: ba_get_params / ba_set_params / ba_get_step /
 * ba_get_linearization / ba_get_blocks use that concatenation, ba_get_batch_layout gives its
 * offsets, ba_cost and ba_linearize's cost return the sum over problems, and
 * ba_solve_schur_power solves every problem with the one lambda given (its info then holds the
 * largest m and stop value, stopped = 1 iff every problem stopped, and the norm of the whole
 * camera step; ba_get_series_state gives each problem's).  ba_lm_step, ba_lm_solve and
 * ba_get_lm_state reject a handle with more than one problem (BA_ERR_INVALID_ARG);
 * ba_set_lm_state sets every problem's state and makes every problem active again.
 * Errors of ba_create_batch: those of ba_create, prefixed "problem p:" in ba_last_error, and
 * BA_ERR_INVALID_ARG for n_problems < 1 or mixed precisions. */
ba_status ba_create_batch(const ba_problem_desc* descs, int32_t n_problems, const ba_options* opts,
                          ba_handle** out);

/* *n_problems = P; cam_off / lm_off (each [P+1], either may be NULL): problem p owns cameras
 * [cam_off[p], cam_off[p+1]) and landmarks [lm_off[p], lm_off[p+1]) of the concatenation.
 * A handle from ba_create reports P = 1. */
ba_status ba_get_batch_layout(ba_handle* h, int32_t* n_problems, int32_t* cam_off, int32_t* lm_off);

/* Series state of the last solve per problem: infos[P] (m, stopped, stop value, ||x(m)|| and
 * the lambda that problem was damped with).  Synchronises. */
ba_status ba_get_series_state(ba_handle* h, ba_series_info* infos);

/* One LM iteration (as ba_lm_step) of every active problem of the handle.  A problem that
 * converges (accepted with relative decrease < func_tol) becomes inactive: later steps leave it
 * unchanged, its series is skipped, and its info keeps converged = 1 and its own iteration
 * count with accepted = 0.  infos (may be NULL) receives P entries; *n_active (may be NULL) the
 * problems still active afterwards.  Synchronises once.  Errors as ba_lm_step (any problem). */
ba_status ba_lm_step_batch(ba_handle* h, ba_step_info* infos, int32_t* n_active);

/* ba_lm_step_batch until no problem is active or max_lm steps ran; infos (may be NULL, P
 * entries) receives each problem's last step, *n_steps the steps run. */
ba_status ba_lm_solve_batch(ba_handle* h, ba_step_info* infos, int32_t* n_steps);

/* F(x) of each problem at the current state: costs[P] (host), float64, fixed order. */
ba_status ba_cost_batch(ba_handle* h, double* costs);

/* Preconditioned conjugate gradients on the reduced camera system S dx_p = -b~ (Sec. 4.2,
 * eqs. `Sx`, `Schur`): the comparison solvers of the paper, built from the same kernels.  S is
 * applied matrix-free (S p = U_lam p - W V_lam^-1 W^T p, the series tile kernel plus a camera
 * kernel).  precond 0: Schur-Jacobi -- the inverses of the 9x9 diagonal blocks of S, the
 * preconditioner of Ceres-explicit / Ceres-implicit (Sec. 5); precond 1: the order-m_precond
 * power series sum_{i<=m} (U^-1 W V^-1 W^T)^i U^-1 (eq. `S_approx`) as M^-1, the Neumann-series
 * preconditioner of Fig. 2 ("PoCG"; each application is a series solve of m_precond terms in
 * the handle's series_exec form).  Hestenes-Stiefel CG from dx_p = 0 until ||r|| <= rtol ||b~||
 * or max_iter iterations; then dx_l by back-substitution.  The step is read with ba_get_step.
 * Vector reductions have a fixed order.  Synchronises once per iteration.  Errors:
 * BA_ERR_NOT_LINEARIZED, BA_ERR_INVALID_ARG, BA_ERR_NOT_SPD, BA_ERR_NONFINITE, BA_ERR_CUDA,
 * BA_ERR_OOM (the PCG vectors are allocated on the first call). */
typedef struct {
  int32_t iterations;  /* CG iterations performed */
  int32_t converged;   /* 1 if the relative residual reached rtol */
  double rel_residual; /* ||r|| / ||b~|| at the end */
  double lambda;       /* damping the blocks were built with */
} ba_pcg_info;
ba_status ba_solve_schur_pcg(ba_handle* h, double lambda, int32_t precond, int32_t m_precond,
                             double rtol, int32_t max_iter, ba_pcg_info* info);

/* Series schedule (no counterpart in the paper; the GPU form of the paper's per-landmark memory
 * blocks, Sec. 5 "Efficient storage").  The power-series kernels cut each problem's observed
 * landmarks into groups of consecutive landmarks of about group_obs observations (boundaries
 * at whole landmarks, balanced by observation count, at most 256 distinct cameras per group in
 * BA_FP32_BULK and 96 in BA_FP64, whose group body also keeps a chunk's J_p in shared memory; a
 * landmark seen by more cameras than that, like a long track, is a group of its own), and each
 * group into chunks of at most 256 observations.  One thread block runs one group and
 * keeps one camera-keyed accumulator per distinct camera of the group, written once per group:
 * larger groups mean fewer partial rows for the camera step, smaller ones finer load balance.
 * The sums of a step depend on the group boundaries, so two handles give bitwise-equal results
 * when their group sizes agree (a batch and handles made for its problems alone included).
 *   group_obs      observations per group; 0: automatic, n_obs / (the blocks of the
 *                  persistent kernel at its largest residency that run groups: SMs x residency
 *                  - 1), i.e. one group per block (two per block for a batch, whose problems
 *                  stop at different terms and steps; at least 256);
 *   tail_parts     each group of at least 512 observations gives its last eighth to
 *                  tail_parts smaller groups, which blocks take after the large ones (groups go
 *                  out largest first), so that the blocks that finish early even out the end of
 *                  the phase; 0: no split (the default at creation);
 *   series_exec    the form series_exec 2 runs: 1 (graph of per-term launches), 3 (persistent
 *                  kernel), 4 (persistent kernel with staged chunks, BA_FP32_BULK) or 5
 *                  (dataflow persistent kernel);
 *   blocks_per_sm  the persistent kernel's residency (1 .. its occupancy limit on the device:
 *                  on GB300 4 for forms 3 and 5 in BA_FP32_BULK, 3 in BA_FP64, 3 for form 4);
 *   n_groups, n_chunks, n_group_slots (ba_get_schedule only): the resulting schedule; the
 *                  camera step sums n_group_slots partial rows of 9 values per term.
 * ba_set_schedule rebuilds the schedule on the host when the group size changes (it waits for
 * the handle's stream and replaces the schedule's device allocation).  Errors:
 * BA_ERR_INVALID_ARG (negative group_obs, tail_parts outside [0, 64], a form other than 1, 3, 4
 * or 5, form 4 in BA_FP64, a residency out of range),
 * BA_ERR_OOM, BA_ERR_CUDA. */
typedef struct {
  int32_t group_obs;
  int32_t tail_parts;
  int32_t series_exec;
  int32_t blocks_per_sm;
  int32_t n_groups, n_chunks, n_group_slots;
} ba_schedule;
ba_status ba_get_schedule(ba_handle* h, ba_schedule* out);
ba_status ba_set_schedule(ba_handle* h, const ba_schedule* in);

/* Autotuner of the series schedule (no counterpart in the paper; the schedule choice of the
 * batched form).  On the handle's current linearisation (linearising first if needed) it times
 * `trials` series solves (damp, invert, max_inner terms, back-substitution; after one warm-up)
 * at lambda0 for: each persistent form (3, 5, and 4 in BA_FP32_BULK) at each residency the
 * device allows with one group per block (group_obs = n_obs / (the blocks that run groups);
 * two per block for a batch) and no tail split; at the fastest of those, tail splits of 0 and 4 and half the group size;
 * and the replayed CUDA graph of per-term launches on the fastest schedule.  The fastest
 * becomes the handle's schedule (ba_get_schedule reports it) and the form series_exec 2 runs.
 * Overwrites the last step (as ba_solve_schur_power does).  *exec_out (may be NULL) receives
 * the chosen form (1, 3, 4 or 5),
 * *blocks_per_sm_out (may be NULL) its blocks per SM (0 for the graph).  Synchronises.
 * Errors: BA_ERR_INVALID_ARG (trials < 1), and those of ba_solve_schur_power. */
ba_status ba_autotune(ba_handle* h, int32_t trials, int32_t* exec_out, int32_t* blocks_per_sm_out);

/* Implicit-differentiation adjoint (no counterpart in the paper; the differentiable form built
 * around its solver).  At the current state x (normally a converged solution, where
 * g = sum_o w_o J_o^T r_o = 0), and for a scalar L(x) whose gradient the caller passes as
 * g_cams = dL/dx_p [n_cams][9] and g_lms = dL/dx_l [n_lms][3] (caller's landmark order), it
 * solves the adjoint system H_lam a = (g_cams; g_lms) with the damped Gauss-Newton matrix of eq.
 * `normal` (Sec. 4.1) -- the same damping as an LM step at `lambda`, which also removes the
 * gauge freedom -- through the Schur complement and the power series of Sec. 4.3 (the
 * handle's eps, max_inner and series_exec; the reduced right-hand side is g_p - W V^-1 g_l),
 * then writes per observation (caller's order)
 *   d_obs [n_obs][2]   = dL/dobs_o = w_o J_o a_o,
 *   d_weights [n_obs]  = dL/dw_o   = -r_o^T J_o a_o   (may be NULL),
 * i.e. the implicit-function-theorem gradients with H_lam in place of dg/dx (exact for a
 * Gauss-Newton step at a fixed point, and at zero residuals for the minimiser of F plus the
 * prior lambda/2 ||D (x - x*)||^2).  The series converges more slowly as lambda decreases
 * (its ratio approaches 1 along the gauge directions): pass a larger max_inner or a larger
 * lambda where the LM's final lambda is tiny.  Linearises first if the state changed;
 * overwrites the last step (the step buffers hold a).  All four arrays are host (ptr_kind 0)
 * or device (1) memory.  info (may be NULL) receives the series state as for
 * ba_solve_schur_power.  Synchronises.  Errors: BA_ERR_INVALID_ARG, BA_ERR_NOT_SPD,
 * BA_ERR_TIMEOUT, BA_ERR_CUDA, BA_ERR_OOM. */
ba_status ba_adjoint(ba_handle* h, double lambda, const double* g_cams, const double* g_lms,
                     double* d_obs, double* d_weights, int32_t ptr_kind, ba_series_info* info);

/* Free all device memory of the handle (and its own stream, if it created one). NULL is OK. */
ba_status ba_destroy(ba_handle* h);

/* Phase timeline of the last persistent series solve: for each executed term (at most 64),
 * five %globaltimer readings in ns taken by the grid's first block.  Forms 3 and 4 (a block
 * that always has group and camera work): term start, end of its group phase, release of the
 * first grid barrier, end of its camera phase, release of the second barrier.  Form 5 (block 0's
 * first group of the term; 0 where block 0 ran no group of that term): its claim, the end of
 * its group body, the end of its row counting, the end of its camera updates, the end of its
 * step (stop rule included).  Copies min(capacity, 5 * terms) values; *n_terms receives the
 * terms. */
ba_status ba_get_series_trace(ba_handle* h, int64_t* ns, int32_t capacity, int32_t* n_terms);

/* Test hook for the bounded grid barriers: the limit, in GPU clock cycles, that a block of the
 * persistent series kernel waits at a barrier before it gives up (default 2^33, several
 * seconds).  Values < 1 restore the default. */
ba_status ba_set_barrier_timeout(ba_handle* h, int64_t cycles);

/* Device rate probe (diagnostics; the paper has no counterpart).  Measures the FP64 fused
 * multiply-add rate of the current device, the ceiling of the float64 series and
 * linearisation kernels: one launch of blocks_per_sm x (number of SMs) blocks of 256 threads,
 * each thread running 8 independent FMA chains for `iters` iterations, after one shorter
 * untimed launch, timed with CUDA events on cuda_stream (NULL: the legacy default stream).
 * *flops_per_s = 2 x FMAs / time; *ms_out (may be NULL) the timed launch in ms.  Synchronises
 * the stream.  Errors: BA_ERR_INVALID_ARG (blocks_per_sm outside [1, 8], iters < 1, NULL
 * flops_per_s), BA_ERR_CUDA. */
ba_status ba_probe_fp64_fma(int32_t blocks_per_sm, int32_t iters, void* cuda_stream,
                            double* flops_per_s, double* ms_out);

/* Debug checks.  The library built with -DPOBA_CHECKS (libpoba_checks.so) checks every camera,
 * landmark, slot, position and segment index its kernels read from the schedule before using
 * it (a bad index is recorded and replaced by an in-range one, so the kernel completes; no
 * trap), and guards every sub-buffer of a handle's device allocations with 256 bytes of 0xA5.
 * Each call that synchronises the handle's stream verifies both and returns BA_ERR_CHECK on a
 * failure.  ba_debug_checks verifies them now: *enabled = 1 in that build (0 in the release
 * build, where the other outputs are 0); *site = the first failed check (0: none; 100 + i: the
 * guard of sub-buffer i of the main allocation, 1100 + i: of the series schedule's), *count =
 * failed checks, *index = the offending index (or byte offset).  The record is then cleared.
 * Any output may be NULL.  Synchronises. */
ba_status ba_debug_checks(ba_handle* h, int32_t* enabled, uint32_t* site, uint32_t* count,
                          int64_t* index);

/* Static string for a status code. */
const char* ba_status_string(ba_status s);

/* Description of the most recent error on the calling thread ("" if none). */
const char* ba_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* POBA_H */

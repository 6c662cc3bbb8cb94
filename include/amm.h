/*
 * amm.h -- C-ABI of the batched A-MMMSE / WMMSE precoding solver for GB300.
 *
 * The library solves many independent multi-cell MU-MIMO weighted-sum-rate
 * problems (problem (1) of arXiv 2510.20507, Sec. II) at once, one thread
 * block per instance, with hand-written sm_103a CUDA kernels.
 *
 * Notation (the paper's letters in brackets): an instance has C cells /
 * base stations (K), K users per cell (I), Nt BS antennas (M), Nr receive
 * antennas per user (N) and d streams per user; user r = k*K + i is user
 * i of cell k (i_k).  m = C*K*Nr is the number of receive rows, n = K*d the
 * number of streams of one cell.
 *
 * Data layouts (device memory, complex values as interleaved float pairs
 * (re, im) = CUDA float2, row-major, instances packed back to back in
 * instance order, no padding):
 *   H      per instance C blocks of (m x Nt): block j row r*Nr + a is row a
 *          of H_{r j}, the channel from BS j to user r.
 *   V, V0  per instance C blocks of (Nt x n): block k columns i*d..i*d+d-1
 *          are the precoder V_{i_k}.
 *   alpha, sigma2  one float per user (C*K per instance);  P  one float per
 *          cell (C per instance).
 *
 * Conventions.  Every call is asynchronous on the stream given at
 * amm_create (a cudaStream_t passed as void*, NULL = legacy default stream)
 * unless it says otherwise, and returns an amm_status; nothing is thrown
 * across the ABI.  The caller owns every buffer it passes; the context owns
 * its workspace (channel copy, iterate history, per-instance scalars),
 * allocated in amm_create and freed in amm_destroy.  Numeric trouble inside
 * an instance (non-finite input, a non-positive Cholesky pivot) is recorded
 * in that instance's status word (amm_status_dev) and the instance stops
 * iterating; other instances are unaffected.  A context must be used from
 * one host thread at a time.
 */
#ifndef AMM_H_
#define AMM_H_

#include <stdint.h>

#if defined(__GNUC__)
#define AMM_API __attribute__((visibility("default")))
#else
#define AMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMM_OK = 0,
  AMM_EINVAL = 1,      /* bad argument: null pointer, size out of range, d > Nr, ... */
  AMM_ENOMEM = 2,      /* device workspace allocation failed */
  AMM_ECUDA = 3,       /* a CUDA call or kernel launch failed */
  AMM_ENUMERIC = 4,    /* per-instance: non-finite input or non-PD matrix */
  AMM_ETIMEOUT = 5,    /* per-instance: a bounded device wait ran out */
  AMM_ENOTCONV = 6,    /* per-instance: tolerance not reached in max_iter */
  AMM_EUNSUPPORTED = 7 /* valid request this build does not implement */
} amm_status;

/* Arithmetic of the two complex GEMMs of each iteration (Z = H V and the
 * gradient H^H Y).  The small Hermitian solves are chosen by fp64_solves. */
typedef enum {
  AMM_FP32 = 0,    /* CUDA-core FP32 FFMA GEMMs (the plain path) */
  AMM_BF16 = 1,    /* tcgen05 BF16 products, FP32 accumulation */
  AMM_BF16X3 = 2,  /* tcgen05 split BF16: hi*hi + hi*lo + lo*hi, FP32 accumulation */
  AMM_BF16X6 = 3   /* tcgen05 three-term split (hi + mid + lo), six products, about
                      FP32 accuracy */
} amm_precision;

/* Sizes of one instance.  1 <= cells <= 16, users >= 1, d <= nr <= 4. */
typedef struct {
  int cells;   /* C  (paper: K cells)          */
  int users;   /* K  (paper: I users per cell) */
  int nt;      /* Nt (paper: M)                */
  int nr;      /* Nr (paper: N)                */
  int d;       /* streams per user             */
} amm_dims;

/* Solver options; amm_default_opts fills the paper's settings. */
typedef struct {
  double eps1;          /* stage-switch tolerance of Algorithm 3; Sec. VII-A: 0.1 */
  double eps2;          /* stopping tolerance of Algorithm 3; Sec. VII-D: 1e-3 */
  int tc;               /* Tc of eq. (16): spectral steps per stage; Sec. V-A: 3 */
  double gamma_c;       /* > 0: the fixed step of eq. (16); <= 0: keep the last
                           spectral step of the stage (step_rule 0) */
  int extrapolate;      /* 1: eqs. (17)-(18); 0: omega = 0 ("w/o extrap.") */
  int switch_iter;      /* -1: automatic stage switch (relative WSR change <= eps1,
                           latched); s >= 1: stage II from iteration s on
                           (1 = A-WMMSE) */
  int step_rule;        /* 0: 1/||F_k||_2 for the first tc iterations of each stage,
                              then gamma_c;  1: 1/||F_k||_2 every iteration;
                           2: gamma_c every iteration (needs gamma_c > 0) */
  int precision;        /* amm_precision */
  int u_at_extrapolated;/* 0: U^t at V^{t-1};  1: U^t at the extrapolated point */
  int lanczos_steps;    /* most Lanczos steps for ||F_k||_2 (capped at Nt and 64);
                           the iteration stops earlier once its largest Ritz
                           value, tested at step 12 and every third step after,
                           moves by less than 1e-6 relative between tests; 64 */
  long long spin_budget;/* SM clock cycles any device-side wait may spin before
                           the instance gets AMM_ETIMEOUT; 2e9 (about 1 s) */
  int smem_budget;      /* bytes of shared memory per block the solver may use;
                           0 = automatic */
  int fp64_solves;      /* arithmetic of the per-user Nr x Nr / d x d Cholesky
                           solves of the U and W updates (eqs. (9), (10)):
                           1: FP64 (default); 2: float-float (pairs of FP32,
                           about 48 significant bits, on the FP32 pipe: a
                           cheaper stand-in for FP64, rates from FP32 log1p);
                           0: FP32.  The WSR evaluation of amm_wsr is FP64
                           whatever this says.  Other values: AMM_EINVAL. */
  int gemm_tile;        /* register tile of the FP32-path block GEMMs: 0 automatic
                           (per GEMM shape, the tile whose slowest thread does
                           the least work), 1: 4x4, 2: 2x2, 3: 4x2, 4: 4x3,
                           5: 2x5 (set by the autotuner); 0 */
  int cluster_cells;    /* multi-cell instances (2 <= cells <= 8) whose channel does
                           not fit one block's shared memory, on the FP32 GEMM path:
                           1 = one thread-block cluster per instance, one block per
                           cell, each keeping its cell's channel block resident and
                           exchanging the per-user covariance parts and U, W over
                           distributed shared memory (default, when such a cluster
                           fits the GPU); 0 = one block per instance, one cell's
                           channel block staged per cell and iteration */
  int schedule;         /* blocks of the one-block-per-instance kernel: 0 = one block
                           per instance, launched longest first for uneven batches
                           (default); 1 = persistent blocks, as many as fit the GPU,
                           each taking the next instance of that order from a device
                           counter (zeroed by a memset before every launch) */
} amm_opts;

typedef struct amm_ctx amm_ctx;

/* Fill *opts with the defaults: eps1 0.1, eps2 1e-3, tc 3, gamma_c 0,
 * extrapolate 1, switch_iter -1, step_rule 0, AMM_FP32, u_at_extrapolated 0,
 * lanczos_steps 64, spin_budget 2e9, smem_budget 0, fp64_solves 1, gemm_tile 0,
 * cluster_cells 1, schedule 0. */
AMM_API void amm_default_opts(amm_opts* opts);

/* Create a solver for `batch` instances.  `dims` points to `n_dims` entries:
 * n_dims == 1 gives every instance the same sizes, n_dims == batch gives
 * instance b the sizes dims[b] (an uneven batch; all instances must then
 * have the same number of cells).  `opts` may be NULL for the defaults.
 * Allocates all device workspace.  Synchronous.  Errors: AMM_EINVAL for
 * sizes out of range (see amm_dims) or a null out pointer, AMM_ENOMEM,
 * AMM_ECUDA.  On error *out is NULL. */
AMM_API amm_status amm_create(amm_ctx** out, int batch, const amm_dims* dims, int n_dims,
                      const amm_opts* opts, void* stream);

/* Total element counts of the packed layouts, for sizing caller buffers:
 * complex elements of H and of V, users (alpha, sigma2), cells (P). */
AMM_API amm_status amm_sizes(const amm_ctx* ctx, int64_t* h_elems, int64_t* v_elems,
                     int64_t* n_users, int64_t* n_cells);

/* Load the problem data of problem (1): channels H (complex64 device,
 * layout above), priority weights alpha, noise powers sigma2 and power
 * budgets P (float device arrays).  The context keeps its own copy of H
 * scaled per user by 1/sigma (the iteration only sees H V V^H H^H/sigma^2,
 * so this is exact) and sets every instance's status word to AMM_OK, or to
 * AMM_ENUMERIC where an input is not finite or sigma2 <= 0. */
AMM_API amm_status amm_set_problem(amm_ctx* ctx, const void* H, const float* alpha,
                           const float* sigma2, const float* P);

/* Initialise the iterate (Algorithm 3, "Initialize"): V^0 is the caller's
 * draw V0 (complex64 device, V layout; Sec. VII-A uses CN(0,1) entries)
 * projected onto each cell's power ball by eq. (15); V^{-1} = V^0; t = 1;
 * stage I (W = I) unless switch_iter == 1.  This starts the two-stage warm
 * start of Sec. V-B; the stage switch itself happens inside amm_step /
 * amm_solve. */
AMM_API amm_status amm_warmstart(amm_ctx* ctx, const void* V0);

/* Run n_iters iterations of Algorithm 3 on every instance: omega by eq. (18),
 * extrapolation eq. (17), U by eq. (9), the stage test and W by eq. (10) or
 * W = I, the step size by eq. (16), and the projected gradient step of
 * eqs. (13)-(15).  One kernel launch; no host synchronisation. */
AMM_API amm_status amm_step(amm_ctx* ctx, int n_iters);

/* Iterate each instance until Algorithm 3's test |R^t - R^{t-1}|/R^{t-1}
 * <= eps2 holds after a stage-II iteration, or max_iter iterations.
 * iters (device int per instance, may be NULL) receives the iterations run
 * by this call; instances that stop at max_iter get status AMM_ENOTCONV. */
AMM_API amm_status amm_solve(amm_ctx* ctx, int max_iter, int* iters);

/* Weighted sum rate of the current iterate per instance, in bits per channel
 * use: sum_r alpha_r log2 det(I + H_rr V_r V_r^H H_rr^H Q_r^{-1}), Q_r the
 * interference-plus-noise covariance (rate definition of Sec. II), with the
 * Cholesky factorisations and the log-det in FP64.  wsr: device double per
 * instance. */
AMM_API amm_status amm_wsr(amm_ctx* ctx, double* wsr);

/* Run n_iters iterations of plain WMMSE (Algorithm 2): U by eq. (9), W by
 * eq. (10), V by eq. (12) with the multiplier lambda_k found by bisection
 * on [0, ||B_k||_F/sqrt(P_k)] until the interval is narrower than
 * bisect_tol or after bisect_max halvings (Sec. VII-A: 1e-4 and 100).  A
 * reference on the GPU, not the fast path. */
AMM_API amm_status amm_wmmse_step(amm_ctx* ctx, int n_iters, double bisect_tol, int bisect_max);

/* The same WMMSE iteration (Algorithm 2, eq. (12) with the same bisection and
 * arguments) with A_k = Q diag(l) Q^H decomposed once per cell and iteration
 * by cyclic Jacobi rotations (FP32, at most 12 sweeps, until the
 * off-diagonal mass is below 1e-5 of ||A_k||_F): each bisection point then
 * costs O(Nt K d) instead of a Cholesky factorisation, and
 * V_k = Q diag(1 / (l + lambda)) Q^H B_k.  Same sizes, errors and status
 * words as amm_wmmse_step. */
AMM_API amm_status amm_wmmse_step_eig(amm_ctx* ctx, int n_iters, double bisect_tol, int bisect_max);

/* Copy the current iterate V (complex64, V layout) to a device buffer. */
AMM_API amm_status amm_get_V(const amm_ctx* ctx, void* V);

/* Iteration state for checkpoint / resume and step-by-step comparison.
 * All pointers are device buffers sized by amm_sizes: V and Vprev hold
 * V^{t-1} and V^{t-2} (complex64, V layout); t, stage (1 or 2) and
 * stage_iter (iterations run in the current stage) are ints per instance;
 * rho_prev (double per instance) is R^{t-1} in nats (NaN before the first
 * iteration); gamma_c (float per cell) is the frozen step of eq. (16). */
typedef struct {
  void* V;
  void* Vprev;
  int* t;
  int* stage;
  int* stage_iter;
  double* rho_prev;
  float* gamma_c;
} amm_state;

AMM_API amm_status amm_get_state(const amm_ctx* ctx, const amm_state* st);
AMM_API amm_status amm_set_state(amm_ctx* ctx, const amm_state* st);

/* Copy the per-instance status words (amm_status values) to a device int
 * buffer. */
AMM_API amm_status amm_status_dev(const amm_ctx* ctx, int* status);

/* End-to-end solve from HOST buffers: copy H, alpha, sigma2, P and V0 to the
 * device, run amm_set_problem, amm_warmstart, amm_step(n_iters) and amm_wsr,
 * and copy the WSR per instance (double, bits) and, if V_out is not NULL,
 * the final precoders (complex64) back.  Host buffers are in the layouts
 * above; pinned host memory makes the copies asynchronous.  Synchronises
 * the context's stream before returning. */
AMM_API amm_status amm_solve_host(amm_ctx* ctx, const void* H, const float* alpha,
                          const float* sigma2, const float* P, const void* V0,
                          int n_iters, double* wsr_out, void* V_out);

/* A whole solve without any device allocation, for callers that must not
 * allocate device memory while they run: a base-station scheduler computing
 * precoders inside a per-slot deadline, where cudaMalloc / cudaFree can
 * synchronise the device and stall far longer than the slot lasts, or a
 * process whose own pool owns all device memory.  (The paper has no
 * counterpart: this is a deployment entry point.)
 *
 * Runs, on a uniform batch of `batch` instances of sizes *dims, what
 * amm_set_problem + amm_warmstart(V0) + amm_step(n_iters) + amm_wsr do on the
 * FP32 GEMM path, with the same kernels and results.  Inputs H, alpha, sigma2,
 * P, V0 and outputs V_out (final precoders, complex64, V layout) and wsr_out
 * (double per instance, bits; NaN for an instance with non-finite input or a
 * failed factorisation) are caller-owned device buffers.  The workspace lives
 * in one static device array of 32 MiB that every GPU loading the library
 * holds until the process exits; batches needing more get AMM_EINVAL with
 * the byte count in `err` (a caller buffer of err_len bytes, may be NULL).
 * opts may be NULL; it is checked as amm_create checks it (AMM_EINVAL /
 * AMM_EUNSUPPORTED), and its precision must be AMM_FP32 (AMM_EUNSUPPORTED
 * otherwise).
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not call
 * this entry point on a device after cudaDeviceReset (the reset destroys the
 * context holding the array, so the kept address is stale).  Every call reuses the array and overwrites or clears what it
 * reads, so consecutive calls are independent; calls whose GPU work overlaps
 * (two host threads, or two streams) race on the array and must not be
 * issued.  Asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 * stream). */
AMM_API amm_status amm_solve_noalloc(int batch, const amm_dims* dims, const amm_opts* opts, const void* H,
                                     const float* alpha, const float* sigma2, const float* P, const void* V0,
                                     int n_iters, void* V_out, double* wsr_out, void* stream, char* err,
                                     int err_len);

/* Fault injection for tests, on the host: the nth device allocation that
 * amm_create or amm_solve_host makes from now on (nth = 1: the next one)
 * fails as if the device were out of memory, without calling cudaMalloc, so
 * the AMM_ENOMEM paths and their clean-up can be exercised with no GPU
 * fault.  nth <= 0 disarms it.  Process-wide; not for production use.
 * (No counterpart in the paper.) */
AMM_API void amm_test_fail_alloc(int nth);

/* Release the context and its workspace (synchronises its stream). */
AMM_API void amm_destroy(amm_ctx* ctx);

/* Message of the last error on this context (or of the last failed
 * amm_create when ctx is NULL).  Valid until the next call. */
AMM_API const char* amm_last_error(const amm_ctx* ctx);

/* Number of kernel launches this context has issued, for launch accounting. */
AMM_API int64_t amm_launch_count(const amm_ctx* ctx);

/* Which iteration kernel the context runs (chosen in amm_create from the
 * sizes and options): 0 one block per instance with CUDA-core FP32 GEMMs,
 * 1 one block per instance with tcgen05 GEMMs, 2 one thread-block cluster per
 * multi-cell instance (see cluster_cells); -1 for a NULL context.  (No
 * counterpart in the paper.) */
AMM_API int amm_path(const amm_ctx* ctx);

/* ---------------------------------------------------------------------
 * CUDA graph of a whole solve.
 *
 * amm_graph_create records, on a private capture stream, what
 * amm_set_problem(H, alpha, sigma2, P) + amm_warmstart(V0) +
 * amm_step(n_iters) + amm_wsr(wsr) enqueue (the normalisation, the warm
 * start, one persistent launch that runs all n_iters iterations of
 * Algorithm 3, and the FP64 WSR), and instantiates it.  amm_graph_launch
 * replays it on the context's stream: one graph launch per solve, reading
 * the inputs from the same caller buffers each time, so a caller refills
 * H / alpha / sigma2 / P / V0 in place between replays (stream-ordered) and
 * replays.  The graph belongs to ctx and uses its workspace: do not destroy
 * ctx before the graph, and do not interleave other ctx calls with a replay
 * in flight.  (The paper has no counterpart: a serving entry point.)
 * ------------------------------------------------------------------- */
typedef struct amm_graph amm_graph;

AMM_API amm_status amm_graph_create(amm_ctx* ctx, const void* H, const float* alpha, const float* sigma2,
                                    const float* P, const void* V0, int n_iters, double* wsr,
                                    amm_graph** out);

/* Replay the recorded solve on the context's stream (asynchronous). */
AMM_API amm_status amm_graph_launch(amm_graph* g);

/* Release the graph (its context stays). */
AMM_API void amm_graph_destroy(amm_graph* g);

/* ---------------------------------------------------------------------
 * Differentiable unrolled A-MMMSE.
 *
 * T iterations of Algorithm 3 (Sec. V, eqs. (9), (10), (13)-(18)) in which
 * the step of iteration t is a parameter gamma_t (eq. (16) replaced by a
 * learnable schedule shared by the batch) and the stage schedule is fixed:
 * stage I (W = I) before iteration switch_iter, stage II (W = E^{-1}, eq.
 * (10)) from it on (switch_iter < 1: stage I throughout).  U^t is taken at
 * V^{t-1}, the gradient at the extrapolated point with omega^t of eq. (18)
 * (extrapolate = 0: omega = 0), and V^t is projected onto the power ball
 * (eq. (15)).  The output is WSR(V^T) in bits.  A hand-written adjoint
 * returns its gradient with respect to every gamma_t and to H.  The paper
 * unrolls nothing; this is the differentiable variant of its iteration.
 *
 * One cell per instance (dims.cells = 1), a uniform batch, every instance's
 * working set in shared memory (AMM_EUNSUPPORTED otherwise).  The forward
 * pass keeps (V^{c-1}, V^c) every ckpt_every iterations; the backward pass
 * recomputes each segment from its checkpoint.
 * ------------------------------------------------------------------- */
typedef struct amm_unrolled amm_unrolled;

/* Create an unrolled solver for `batch` instances of sizes *dims, T
 * iterations, checkpoints every ckpt_every iterations; work is queued on
 * `stream` (a cudaStream_t; NULL = legacy default stream).  Allocates the
 * checkpoint and recomputation workspace. */
AMM_API amm_status amm_unrolled_create(amm_unrolled** out, int batch, const amm_dims* dims, int T, int ckpt_every,
                                       int switch_iter, int extrapolate, void* stream);

/* Forward pass.  Device inputs, caller-owned, read again by the backward
 * pass (keep them alive and unchanged until it has run): H (complex64, batch
 * x K Nr x Nt, the amm_set_problem layout for one cell), alpha and sigma2
 * (float, batch x K), P (float, batch), V0 (complex64, batch x Nt x K d; a
 * feasible start, e.g. the projected warm start of eq. (15)), gamma (float,
 * T).  Output wsr (double, batch, bits).  Channels are normalised by sigma
 * inside, as in amm_set_problem.  Asynchronous. */
AMM_API amm_status amm_unrolled_forward(amm_unrolled* u, const void* H, const float* alpha, const float* sigma2,
                                        const float* P, const void* V0, const float* gamma, double* wsr);

/* Backward pass for the last forward pass: wsr_bar (double, batch) holds
 * dL/dWSR per instance; outputs gamma_bar (float, batch x T: instance b's
 * dL/dgamma_t, summed over b by the caller) and H_bar (complex64, the layout
 * of H: dL/dRe(H) + i dL/dIm(H)).  Asynchronous. */
AMM_API amm_status amm_unrolled_backward(amm_unrolled* u, const double* wsr_bar, float* gamma_bar, void* H_bar);

/* Per-instance status of the last pass (AMM_OK or AMM_ENUMERIC) into a
 * device int array of batch entries. */
AMM_API amm_status amm_unrolled_status(amm_unrolled* u, int* status_dev);

/* Message of the last error on u (or of the last failed create when u is NULL). */
AMM_API const char* amm_unrolled_last_error(amm_unrolled* u);

/* Release u and its workspace. */
AMM_API void amm_unrolled_destroy(amm_unrolled* u);

#ifdef __cplusplus
}
#endif

#endif /* AMM_H_ */

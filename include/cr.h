/*
 * cr.h -- C ABI of the GB300 (sm_103a) library for the dual smoothing method of
 * Aybat & Wang, "A Parallelizable Dual Smoothing Method for Large Scale Convex
 * Regression Problems" (arXiv 1608.02227).
 *
 * Problem (Eq. (regularize), Section 2.1): given points x_l in R^n and observations
 * ybar_l, l = 0..N-1, find
 *     min  1/2 ||y - ybar||^2 + gamma/2 ||xi||^2
 *     s.t. (C eta)_ij = y_j - y_i + xi_i . (x_i - x_j) >= 0   for all i != j
 * (Eq. (original): the first-order convexity conditions of a fitted convex function
 * with values y_l and subgradients xi_l).  Every one of the N(N-1) constraints is
 * dualised (the K = N case of the partition of Section 2.1), so the multipliers form
 * an N x N matrix Lambda (lambda_ij of pair (i, j), diagonal unused) and Step 1 of
 * P-APG (Figure "papg") is the closed form
 *     y = ybar + a,  xi = b / gamma,  (a, b) = C^T lambda,
 *     a_l = sum_i lambda_il - sum_j lambda_lj,   b_l = sum_j lambda_lj (x_l - x_j).
 * One iteration k is then (Steps 2-4 of Figure "papg", Eq. (dual gradient)):
 *     lambda~ = lambda^{k-1} + beta_k (lambda^{k-1} - lambda^{k-2}),
 *     rho_ij  = -(C eta(lambda~))_ij = y_i - y_j + xi_i . (x_j - x_i),
 *     lambda^k_ij = max(0, lambda~_ij + rho_ij / L),
 *     t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  beta_{k+1} = (t_k - 1) / t_{k+1},
 * with L an upper bound on the Lipschitz constant of grad g_gamma (Eq. (lischitz)).
 *
 * Conventions of every entry point:
 *   - Pointers may be host or device memory of the context's device (copies use
 *     unified addressing, cudaMemcpyDefault).  Arrays are dense and row-major: X is N x n
 *     (X[l*n + k]), xi is N x n, Lambda is N x N with leading dimension ld.
 *   - The library copies its inputs; the caller owns every buffer it passes.
 *   - Errors are returned as cr_status; nothing throws across the ABI.  The text
 *     of the last failure on the calling thread is returned by cr_last_error().
 *   - A context is bound to the CUDA device that was current at cr_create and to
 *     one stream; it is not thread-safe (one thread at a time per context).
 */
#ifndef CR_H
#define CR_H

#ifdef __cplusplus
extern "C" {
#endif

#define CR_API __attribute__((visibility("default")))

typedef struct cr_ctx cr_ctx;

typedef enum {
    CR_OK = 0,
    CR_EINVAL = 1,       /* bad argument: N < 2, n < 1, n > CR_MAX_N, gamma <= 0, non-finite data */
    CR_ENOMEM = 2,       /* a device or host allocation failed */
    CR_ECUDA = 3,        /* a CUDA call failed (message in cr_last_error) */
    CR_ENOTCONV = 4,     /* cr_solve reached max_iter before rel_gap_tol */
    CR_ETIMEOUT = 5,     /* a bounded device-side wait ran out */
    CR_ENUMERIC = 6,     /* a non-finite objective or gap was produced */
    CR_EUNSUPPORTED = 7  /* the requested mode is not available on this device */
} cr_status;

typedef enum {
    CR_FP64 = 0,         /* Lambda, residuals and reductions in FP64 (parity mode) */
    CR_FP32 = 1,         /* Lambda FP32 in HBM, FP32 residuals with hi+lo y and u, FP64 recovery */
    CR_MIXED_TF32 = 2    /* Lambda FP32, xi.x and Lambda.X on tcgen05 (TF32, hi+lo split) */
} cr_precision;

typedef enum {
    CR_L_HESSIAN = 0,    /* L = 2N + sigma_max(A2)^2 / gamma >= lambda_max(C G^-1 C^T) */
    CR_L_PAPER = 1       /* L = (2N + sigma_max(A2)^2) / gamma >= sigma_max(C)^2 / gamma, Eq. (lischitz) */
} cr_lipschitz_rule;

#define CR_MAX_N 128     /* largest point dimension n supported by the kernels (FP64, FP32) */
#define CR_MAX_N_TF32 31 /* CR_MIXED_TF32 (the tensor-core sweep) */
#define CR_MAX_N_BATCH 32 /* cr_batch_* and cr_server_* instances */

/* Step size of Step 2 of Figure "papg".
 *   CR_STEP_CONSTANT: 1/L every iteration.
 *   CR_STEP_ADAPTIVE: the adaptive rule of Section 4 ("Adaptive Step Size Strategy"): iteration k
 *     tries s_k = s_{k-1} upsilon^(l-1) for l = 0, 1, ... and keeps the first step 1/s_k that
 *     satisfies Eq. (adaptive-check); s_0 = L.  Every candidate is one sweep over all pairs; the
 *     decision is taken on the device (three multiplier buffers instead of two), so cr_dual_step
 *     counts candidates (sweeps) and cr_gap_info.k counts accepted iterations.  All precisions,
 *     single instances, batches and the server. */
typedef enum cr_step_rule { CR_STEP_CONSTANT = 0, CR_STEP_ADAPTIVE = 1 } cr_step_rule;

typedef struct cr_options {
    double gamma;        /* Tikhonov parameter gamma > 0 (Section 5 uses 1e-4) */
    double lipschitz;    /* 0: computed on the device at cr_create; > 0: used as L */
    int lipschitz_rule;  /* cr_lipschitz_rule, used when lipschitz == 0 */
    int precision;       /* cr_precision */
    int accelerate;      /* 1: P-APG momentum (Step 4); 0: projected dual gradient ascent */
    int check_every;     /* iterations between convergence checks in cr_solve (>= 1) */
    int graph_iters;     /* iterations per captured CUDA graph in cr_dual_step (even; 0: no graphs) */
    int tile_cols;       /* columns of Lambda per work item (multiple of 128; 0: chosen by the library;
                            with 0 the tensor-core sweep gives every CTA an equal range of
                            32-column chunks instead of whole items) */
    int deterministic;   /* kept for ABI stability: every reduction is already in a fixed order */
    int step_rule;       /* cr_step_rule: CR_STEP_CONSTANT (1/L, Figure "papg") or CR_STEP_ADAPTIVE */
    double upsilon;      /* CR_STEP_ADAPTIVE: the factor upsilon > 1 of the step rule (default 2) */
    int restart;         /* 1: reset the momentum (t = 1) when g_gamma(lambda^k) < g_gamma(lambda^{k-1}),
                            function-value restart of the accelerated iteration (not in the paper) */
    int refresh_every;   /* CR_FP32 / CR_MIXED_TF32 with n <= 32: > 0 reduces each sweep's change of the
                            multipliers, (a,b)^k = (a,b)^{k-1} + C^T (lambda^k - lambda^{k-1}) in FP64, and
                            re-evaluates C^T lambda^k exactly in FP64 from the stored multipliers at
                            k = 2 refresh_every, 3 refresh_every, ...; 0 forms C^T lambda^k from FP32
                            partials every iteration (default 64) */
} cr_options;

/* Convergence record for eta(lambda^k), the primal of Theorem "rate". */
typedef struct cr_gap_info {
    long long k;         /* iterations taken */
    double dual_g;       /* g_gamma(lambda^k) = -1/2||a||^2 - a.ybar - ||b||^2/(2 gamma) */
    double primal_r;     /* r_gamma(eta(lambda^k)) = 1/2||a||^2 + ||b||^2/(2 gamma) */
    double lagr_gap;     /* <lambda^k, C eta(lambda^k)> = primal_r - dual_g (Section 5.1 duality gap) */
    double infeas_norm;  /* ||(C eta(lambda^k))_-||_2 / sqrt(N^2 - N) (Section 5.1 infeasibility) */
    double rel_gap;      /* max(|lagr_gap| / primal_r, infeas_norm / rms(ybar)) */
    double cert_primal;  /* r_gamma of the feasible max-affine repair of eta(lambda^k): >= p*_gamma */
    double cert_gap_rel; /* (cert_primal - dual_g) / cert_primal: a certified bound on (p* - g)/p* */
    double step;         /* 1/s of the next candidate step (1/L with CR_STEP_CONSTANT) */
    long long sweeps;    /* sweeps over all pairs so far (= k with CR_STEP_CONSTANT) */
} cr_gap_info;

/* Fills *opt with the defaults: gamma 1e-4, lipschitz 0 (computed), CR_L_HESSIAN,
 * CR_FP32, accelerate 1, check_every 100, graph_iters 32, tile_cols 0, CR_STEP_CONSTANT,
 * upsilon 2, restart 0, refresh_every 64. */
CR_API void cr_default_options(cr_options *opt);

/* Creates a solver for one instance (Eq. (regularize)).
 *   X: N x n points (host or device, FP64); ybar: N observations (FP64);
 *   opt: NULL for the defaults; stream: a cudaStream_t other than the legacy default
 *   stream, or NULL (or the legacy stream) for a stream the context creates and owns.  Copies X and ybar to the device, computes L (Section
 *   3's "Preprocess", on the device) unless opt->lipschitz > 0, allocates the two
 *   N x N multiplier buffers and sets lambda^0 = 0 (theta^0 = 0, t_1 = 1).
 *   Errors: CR_EINVAL (N < 2, n < 1 or > CR_MAX_N, gamma <= 0, non-finite inputs),
 *   CR_ENOMEM, CR_ECUDA.  On error *out is NULL. */
CR_API cr_status cr_create(const double *X, const double *ybar, long long N, int n,
                           const cr_options *opt, void *stream, cr_ctx **out);

/* Enqueues `iters` P-APG iterations (Figure "papg", K = N) on the context's stream and
 * returns without waiting.  Each iteration is the fused Lambda sweep (Steps 2 and 4 and
 * the reductions of C^T) followed by the recovery of Step 1 for the next iteration. */
CR_API cr_status cr_dual_step(cr_ctx *ctx, int iters);

/* Runs iterations until rel_gap <= rel_gap_tol (CR_OK) or max_iter iterations in total
 * have been taken (CR_ENOTCONV); checks every opt->check_every iterations.  *out (may
 * be NULL) receives the last record.  Blocks the calling thread. */
CR_API cr_status cr_solve(cr_ctx *ctx, double rel_gap_tol, long long max_iter, cr_gap_info *out);

/* Copies eta(lambda^k) = (y, xi) (FP64; y: N, xi: N x n) into caller buffers (host or
 * device).  Synchronises the stream. */
CR_API cr_status cr_primal(const cr_ctx *ctx, double *y, double *xi);

/* Computes the convergence record at the current iterate, including the pass over all
 * pairs that gives infeas_norm and the certified repair (cert_primal).  Synchronises. */
CR_API cr_status cr_gap(cr_ctx *ctx, cr_gap_info *out);

/* Copies rows [row0, row0 + rows) of lambda^k as FP64 into out (rows x N, leading
 * dimension ld >= N; host or device).  Synchronises.  For parity checks and checkpoints. */
CR_API cr_status cr_lambda(const cr_ctx *ctx, long long row0, long long rows, double *out,
                           long long ld);

/* Enqueues `iters` iterations like cr_dual_step, without graphs, with CUDA events around
 * every launch of the Lambda sweep; returns after the stream drains with *sweep_ms = the
 * summed device time of the sweeps and *total_ms = the device time of all iterations. */
CR_API cr_status cr_dual_step_timed(cr_ctx *ctx, int iters, float *sweep_ms, float *total_ms);

/* Writes a one-line JSON description of the context (sizes, tile shape, grid, bytes per
 * iteration, L) into buf (always NUL-terminated). */
CR_API cr_status cr_describe(const cr_ctx *ctx, char *buf, int len);

/* Returns the step constant L in use. */
CR_API cr_status cr_lipschitz(const cr_ctx *ctx, double *L);

/* Allocation-free computation of the step constant L that cr_create computes (the paper
 * has no counterpart: this is an interface for callers that must not allocate device
 * memory at the moment they need L -- e.g. an admission controller that budgets HBM before
 * reserving it, a framework whose caching allocator owns all of HBM, or a latency-critical
 * loop where cudaMalloc/cudaFree would synchronise the device).
 *   X: N x n points, FP64, row-major, DEVICE memory of the current device only (host
 *   pointers and memory of another device are rejected with CR_EINVAL); rule: CR_L_HESSIAN or
 *   CR_L_PAPER; stream: cudaStream_t or NULL; *L receives the same value cr_create computes
 *   for these inputs.  Errors as cr_create: CR_EINVAL for bad sizes or a non-finite entry of
 *   X, CR_ENUMERIC when L comes out non-finite or <= 0, CR_ECUDA for a failed CUDA call.
 * Limit: 1 <= n <= CR_MAX_N (128); the scratch is a fixed 264 KB array in device memory that
 * every GPU which loads the library holds until the process exits.  No cudaMalloc, cudaFree
 * or other allocating call is made.  The first call on a device (with that device current)
 * looks up the array's device address.  Every call copies the result to the host and
 * synchronises the stream, so it cannot be made while that stream is being captured.
 * Every call shares the array: calls whose work overlaps on the GPU (two streams or threads
 * at once) race and must be serialised by the caller. */
CR_API cr_status cr_lipschitz_noalloc(const double *X, long long N, int n, double gamma, int rule, void *stream,
                                      double *L);

/* Failure-path hook (the paper has no counterpart): bounds every wait of the FP32 TMA sweep's
 * consumer warps for data to land (default 2 s) by consumer_wait_ns nanoseconds (0 restores
 * the default).  The producer's waits keep their normal bound, so every copy it issued lands
 * before a CTA exits.  A wait that runs out makes the sweep abort cleanly; the next cr_gap or
 * cr_solve on the context returns CR_ETIMEOUT and the context's iterate is no longer valid
 * (destroy it; other contexts are unaffected).  For tests of the timeout path; CR_EUNSUPPORTED
 * when the context does not run the TMA sweep. */
CR_API cr_status cr_set_wait_limit(cr_ctx *ctx, long long consumer_wait_ns);

/* Iterations taken so far (sweeps with CR_STEP_ADAPTIVE). */
CR_API long long cr_iterations(const cr_ctx *ctx);

/* Continuation in gamma (Section 6): changes gamma of Eq. (regularize) in place, keeping
 * lambda^k as the warm start theta^0 of the new problem.  Recomputes L by the context's rule from
 * the cached sigma_max(A2)^2 and the step (1/L, or upsilon/L for the adaptive rule), restarts the
 * momentum (t = 1, as Iteration 0 of Figure "papg"), rebuilds eta(lambda^k) for the new gamma
 * and recomputes the record's g, r and lambda^T C eta of lambda^k at the new gamma.
 * CR_EINVAL when gamma is not finite and > 0 or when the context was created with a caller-given
 * L (opt.lipschitz > 0), which cannot follow gamma. */
CR_API cr_status cr_set_gamma(cr_ctx *ctx, double gamma);

/* The continuation path of Section 6: for t = 0 .. stages-1, gamma_t = gammas[t] (cr_set_gamma,
 * warm start from the previous stage) and cr_solve to rel_gap <= tols[t] with at most max_sweeps
 * sweeps in the stage.  *out (nullable) is the record of the last stage run; CR_ENOTCONV when a
 * stage reaches its cap (the path stops there). */
CR_API cr_status cr_solve_path(cr_ctx *ctx, const double *gammas, const double *tols, int stages,
                               long long max_sweeps, cr_gap_info *out);

/* The continuation schedule of Section 6: for t = 1 .. stages, eps_t = eps0 / beta^t,
 * gamma_t = kappa_gamma * eps_t and delta_t = kappa_delta * eps_t; stage t warm-starts from
 * stage t-1 (cr_set_gamma) and iterates (checks every opt.check_every sweeps) until lambda^k
 * passes either test of delta_t-optimality for Eq. (dual-problem):
 *   certified:  cert_primal - dual_g <= delta_t  (a bound on max g_gamma - g_gamma(lambda^k),
 *               since cert_primal >= p*_gamma; rigorous but loose),
 *   practical:  |lagr_gap| <= delta_t and infeas_norm <= infeas_tol  (the duality gap
 *               |lambda^T C eta| and normalised infeasibility of Section 5's stopping rule;
 *               infeas_tol < 0 disables it).
 * At most max_sweeps iterations per stage (CR_ENOTCONV, the path stops there).  Requires
 * beta > 1 and eps0, kappa_gamma, kappa_delta > 0 (else CR_EINVAL).  *out (nullable) is the
 * record of the last check. */
CR_API cr_status cr_solve_continuation(cr_ctx *ctx, double eps0, double beta, double kappa_gamma,
                                       double kappa_delta, double infeas_tol, int stages,
                                       long long max_sweeps, cr_gap_info *out);

/* Checkpoint / resume of the iteration state: the multiplier buffers, the C^T history, the
 * vectors of eta the next sweep reads and the device scalars, as one block of
 * cr_checkpoint_bytes(ctx) bytes in caller-owned memory (host or device).  cr_restore loads a
 * block into a context created for the same instance and options (CR_EINVAL when its shape,
 * precision or step rule differ, or when X or ybar differ: the block carries a fingerprint
 * of both); the next iterations are bitwise those of the saved run. */
CR_API long long cr_checkpoint_bytes(const cr_ctx *ctx);
CR_API cr_status cr_checkpoint(cr_ctx *ctx, void *buf, long long bytes);
CR_API cr_status cr_restore(cr_ctx *ctx, const void *buf, long long bytes);

/* Releases every resource of the context (NULL is ignored). */
CR_API void cr_destroy(cr_ctx *ctx);

/* ------------------------------------------------------------------------------------
 * Row sharding over several GPUs.  The per-iteration work of the method is the pass over the
 * constraints that applies C and C^T (Section 3), and it splits over disjoint sets of
 * constraints: a shard holds the multipliers of the pairs (i, j) with i in [row0, row0 + rows)
 * and every j.  Each rank (one GPU) creates one shard; an iteration is
 *     cr_shard_sweep   -> the caller sums the N + 1 exchange values over all shards ->
 *     cr_shard_finish,
 * and afterwards every shard holds the same a = C_y^T lambda^k, y, g_gamma, r_gamma and
 * <lambda, C eta>, and xi of its own rows.  The constant step of Figure "papg" (the adaptive
 * check would need a second exchange), C^T formed from the partials every iteration (no
 * exact refresh across shards), no CUDA graphs, n <= CR_MAX_N_BATCH.  The entry points of a
 * whole instance (cr_dual_step, cr_solve, cr_gap, cr_primal, ...) return CR_EINVAL on a shard.
 * ------------------------------------------------------------------------------------ */

/* X: all N x n points, ybar: all N observations (host or device, copied); the shard holds rows
 * [row0, row0 + rows): row0 a multiple of 128, row0 + rows <= N.  opt as in cr_create (the
 * step rule must be CR_STEP_CONSTANT: CR_EUNSUPPORTED otherwise).  stream: the stream on which
 * the caller's exchange runs, or NULL. */
CR_API cr_status cr_shard_create(const double *X, const double *ybar, long long N, int n, long long row0,
                                 long long rows, const cr_options *opt, void *stream, cr_ctx **out);

/* Enqueues the next iteration's sweep over the shard's rows and writes into exchange (DEVICE
 * memory of the context's device, N + 1 FP64) the shard's share of the sums every shard needs:
 * exchange[l] = sum over the held rows i of lambda_il - [l held] sum_j lambda_lj (summed over all
 * shards: a_l = c_l - r_l of Definition 1), exchange[N] = sum over the held rows of ||b_l||^2. */
CR_API cr_status cr_shard_sweep(cr_ctx *ctx, double *exchange);

/* Completes the iteration from exchange summed over all shards (device memory, N + 1 FP64):
 * C^T lambda^k, the objective values, t and beta, and eta of the next extrapolated point. */
CR_API cr_status cr_shard_finish(cr_ctx *ctx, const double *exchange);

/* eta(lambda^k) as the shard holds it: y (N, every point) and xi of the held rows (rows x n;
 * either pointer may be NULL; host or device), and *out (nullable): k, g_gamma, r_gamma,
 * <lambda, C eta> and |<lambda, C eta>| / r_gamma as rel_gap (the infeasibility term needs a pass
 * over all constraints and is left at 0).  Synchronises. */
CR_API cr_status cr_shard_state(cr_ctx *ctx, double *y, double *xi, cr_gap_info *out);

/* ------------------------------------------------------------------------------------
 * Batched solving: many independent instances (uneven N and n) iterate together.  Every
 * iteration is one persistent sweep launch per bucket over a device work-list of (instance,
 * row block, column split) items -- one bucket per padded point dimension for the FP32 TMA
 * sweep (32-row blocks), one bucket for all tensor-core instances (128-row blocks); the
 * buckets run as parallel branches of a captured CUDA graph -- followed by one finalize
 * launch over all instances.
 * Each instance keeps its own multipliers, step constant, t_k and iteration count, and is
 * retired at its own convergence check (the K = N method of Figure "papg" per instance).
 * A batch is bound to one stream and is not thread-safe.
 * ------------------------------------------------------------------------------------ */
typedef struct cr_batch cr_batch;

/* opt: NULL for the defaults (precision CR_FP32 or CR_MIXED_TF32; graph_iters is the number
 * of iterations per captured graph; check_every the iterations between checks in
 * cr_batch_run).  With CR_MIXED_TF32 every instance with n <= CR_MAX_N_TF32 runs the
 * tensor-core sweep (all of them in one persistent launch over a work-list of 128-row items)
 * and an n = 32 instance runs the FP32 sweep.  stream: as in cr_create. */
CR_API cr_status cr_batch_create(const cr_options *opt, void *stream, cr_batch **out);

/* Adds one instance (X: N x n with n <= CR_MAX_N_BATCH, ybar: N; host or device; copied).  It is retired once a
 * check finds rel_gap <= rel_gap_tol (status CR_OK) or after max_iter iterations
 * (status CR_ENOTCONV).  *id receives its handle (>= 0). */
CR_API cr_status cr_batch_add(cr_batch *b, const double *X, const double *ybar, long long N, int n,
                              double rel_gap_tol, long long max_iter, int *id);

/* Runs `iters` iterations of every active instance, then checks every active instance
 * and retires the converged ones.  *active (may be NULL) receives how many remain. */
CR_API cr_status cr_batch_step(cr_batch *b, int iters, int *active);

/* Repeats cr_batch_step(opt.check_every) until no instance is active. */
CR_API cr_status cr_batch_run(cr_batch *b);

/* Retirement state of instance id: *done = 1 once retired; *status = CR_OK (converged),
 * CR_ENOTCONV (max_iter) or an error; *info = its last convergence record. */
CR_API cr_status cr_batch_poll(cr_batch *b, int id, int *done, int *status, cr_gap_info *info);

/* eta(lambda^k) of instance id, as cr_primal. */
CR_API cr_status cr_batch_primal(cr_batch *b, int id, double *y, double *xi);

/* Releases the device memory of instance id (active or retired); the id stays invalid. */
CR_API cr_status cr_batch_remove(cr_batch *b, int id);

/* Device bytes that an instance of N points in n dimensions takes at most in a batch with the
 * constant step, in either precision (the adaptive step adds a third multiplier buffer,
 * 4 N ceil32(N) bytes, and O(N n)). */
CR_API long long cr_batch_instance_bytes(long long N, int n);

/* Times `iters` iterations of the active instances for each column-split width in
 * {512, 1024, 2048, 4096, whole rows} and keeps the fastest (the iterations count as
 * real iterations).  *tile_cols (may be NULL) receives the chosen width. */
CR_API cr_status cr_batch_autotune(cr_batch *b, int iters, int *tile_cols);

CR_API void cr_batch_destroy(cr_batch *b);

/* ------------------------------------------------------------------------------------
 * Serving: a request queue in front of one batch, driven by a server thread.  Requests
 * (one instance each) are admitted in arrival order while their device memory
 * (cr_batch_instance_bytes) fits under mem_cap and fewer than max_active run; admitted
 * instances join the running ones at the next block of opt->check_every iterations, share
 * their launches, and retire at their own tolerance, which frees their memory for the queue.
 * Submit/poll/wait/result may be called from any thread.
 * ------------------------------------------------------------------------------------ */
typedef struct cr_server cr_server;

typedef struct cr_serve_stats {
    long long completed;  /* requests finished (converged, capped or failed) */
    long long converged;  /* finished with CR_OK */
    long long queued;     /* waiting for admission */
    long long running;    /* on the GPU */
    long long mem_used;   /* device bytes reserved by running requests */
    long long mem_cap;
    double p50_s, p99_s;  /* submit-to-finish latency percentiles of finished requests */
    double elapsed_s;     /* since cr_server_create */
    double busy_s;        /* time spent in iteration blocks */
} cr_serve_stats;

/* opt as in cr_batch_create; mem_cap_bytes > 0; max_active >= 1; stream as in cr_create. */
CR_API cr_status cr_server_create(const cr_options *opt, long long mem_cap_bytes, int max_active, void *stream,
                                  cr_server **out);

/* Queues one solve of Eq. (regularize) (inputs copied before returning; host or device;
 * n <= CR_MAX_N_BATCH).  CR_ENOMEM if the instance alone exceeds the memory cap. */
CR_API cr_status cr_server_submit(cr_server *s, const double *X, const double *ybar, long long N, int n,
                                  double rel_gap_tol, long long max_iter, long long *req_id);

/* *state: 0 queued, 1 running, 2 finished; *status: CR_OK, CR_ENOTCONV or an error (when
 * finished); *info: last convergence record; *latency_s: submit-to-finish, or -1. */
CR_API cr_status cr_server_poll(cr_server *s, long long req_id, int *state, int *status, cr_gap_info *info,
                                double *latency_s);

/* Blocks until the request is finished (CR_OK) or timeout_s passes (CR_ETIMEOUT). */
CR_API cr_status cr_server_wait(cr_server *s, long long req_id, double timeout_s);

/* Copies eta(lambda^k) of a finished request (y: N, xi: N x n; host or device). */
CR_API cr_status cr_server_result(cr_server *s, long long req_id, double *y, double *xi);

/* Forgets a finished request (its host result buffers are freed). */
CR_API cr_status cr_server_release(cr_server *s, long long req_id);

CR_API cr_status cr_server_stats(cr_server *s, cr_serve_stats *out);

/* Stops the server thread after the current block and frees everything. */
CR_API void cr_server_destroy(cr_server *s);

CR_API const char *cr_strerror(cr_status s);
CR_API const char *cr_last_error(void);
CR_API int cr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CR_H */

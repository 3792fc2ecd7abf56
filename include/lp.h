/*
 * lp.h -- C ABI of the GB300 restarted-PDHG linear-programming solver.
 *
 * Problem (the paper's Section 2.2 primal form):
 *
 *     min  c^T x   s.t.  G x >= h,  A x = b,  l <= x <= u,
 *
 * given as one CSR matrix K = (G; A) whose rows may come in any order, with a
 * per-row sense flag: sense[i] = 1 marks a row of G (K_i x >= q_i), sense[i] = 0
 * a row of A (K_i x == q_i); q stacks h and b the same way.  A <= row is passed
 * negated.  Bounds may be -INFINITY / +INFINITY (IEEE).  The dual (Section 2.2)
 * is  max q^T y + l^T lambda^+ + u^T lambda^-  with lambda = c - K^T y in Lambda
 * and y >= 0 on the rows of G.
 *
 * Conventions for every entry point:
 *   - Every call returns lp_status.  Negative values are API or device failures;
 *     non-negative values are solver outcomes.  Nothing aborts, prints or traps.
 *   - Pointers are host or device memory as the accompanying memory_space field
 *     says (LP_MEM_HOST / LP_MEM_DEVICE).  Device pointers must belong to the
 *     current CUDA device.
 *   - lp_create deep-copies its inputs; the handle owns all device memory it
 *     allocates and releases it in lp_destroy.  The caller owns every input and
 *     every result buffer.
 *   - All work of a handle runs on the CUDA stream given to lp_create (or a
 *     private stream if that is NULL).  lp_solve / lp_solve_batch / lp_grad
 *     return after that stream has finished the call's work.
 *   - A handle is not thread-safe: one call at a time per handle.
 */
#ifndef GB300_PDHG_LP_H
#define GB300_PDHG_LP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LP_ABI_VERSION 5

typedef struct lp_problem_s* lp_handle;

typedef enum {
    LP_OK = 0,
    LP_OPTIMAL = 1,              /* all three relative errors of Section 2.3.2 <= tol */
    LP_PRIMAL_INFEASIBLE = 2,    /* Algorithm 6 found a primal infeasibility certificate (Section 2.4.5) */
    LP_DUAL_INFEASIBLE = 3,      /* Algorithm 6 found a dual infeasibility certificate (Section 2.4.5) */
    LP_ITERATION_LIMIT = 4,
    LP_TIME_LIMIT = 5,
    LP_NUMERICAL_ERROR = 6,      /* NaN / Inf met in an iterate or a reduction */
    LP_INVALID_ARGUMENT = -1,
    LP_CUDA_ERROR = -2,
    LP_OUT_OF_MEMORY = -3,
    LP_DEVICE_TIMEOUT = -4,
    LP_NOT_SUPPORTED = -5
} lp_status;

enum { LP_MEM_HOST = 0, LP_MEM_DEVICE = 1 };

/* Arithmetic of the PDHG iterations.
 * LP_PREC_FP64: matrix, iterates and reductions in FP64.
 * LP_PREC_MIXED: matrix, iterates and SpMV accumulation in FP32, every
 *   reduction (KKT terms, step-size terms) in FP64; once the FP32 phase reaches
 *   max(tol, polish_switch_tol) its candidate moves to the FP64 engine, whose
 *   check re-evaluates the three relative errors of Section 2.3.2 with FP64
 *   products and FP64 element terms.  LP_OPTIMAL is returned only when they hold
 *   there; otherwise (and whenever tol < polish_switch_tol) FP64 iterations
 *   continue from the candidate to tol (FP64 polish).  lp_result.precision_used
 *   is LP_PREC_FP64 when FP64 iterations ran. */
enum { LP_PREC_FP64 = 0, LP_PREC_MIXED = 1 };

/* The LP.  Arrays: row_ptr[m+1] (row_ptr[0] = 0, non-decreasing,
 * row_ptr[m] = nnz), col_idx[nnz] in [0, n) (any order inside a row; duplicates
 * are summed), vals[nnz], sense[m], c[n], q[m], l[n], u[n] with l <= u and no
 * NaN anywhere.  Requirements: m >= 1, n >= 1, nnz < 2^31 - 64. */
typedef struct {
    int64_t m, n, nnz;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const double* vals;
    const uint8_t* sense;
    const double* c;
    const double* q;
    const double* l;
    const double* u;
    int32_t memory_space;     /* LP_MEM_HOST or LP_MEM_DEVICE, for all arrays above */
    int32_t reserved;
} lp_desc;

/* Solver options.  Fill with lp_opts_default, then change fields. */
typedef struct {
    double tol;                  /* epsilon of Section 2.3.2 (default 1e-4) */
    int64_t max_iters;           /* accepted PDHG iterations (default 1e6) */
    double time_limit_s;         /* wall-clock limit checked on the device (default 3600) */
    int32_t precision;           /* LP_PREC_FP64 (default) or LP_PREC_MIXED */
    int32_t check_every;         /* accepted iterations between KKT checks (default 64) */
    int32_t ruiz_iters;          /* passes of Algorithm 3 (default 10; 0 disables) */
    int32_t pock_chambolle;      /* 0 (default): no Pock-Chambolle pass; 1: one pass with
                                    pc_alpha after Ruiz (rows by 1/sqrt(sum_j |K~_ij|^(2-alpha)),
                                    columns by 1/sqrt(sum_i |K~_ij|^alpha)); 2 (lp_solve only):
                                    alpha chosen from {0, 1/2, 1, 2} by trial solves of
                                    pc_trial_iters iterations each, the one with the smallest
                                    relative KKT error (Section 2.3.2) at its end wins (ties: the
                                    earlier); lp_fishnet treats 2 as 1 */
    int32_t adaptive_step;       /* 1: Algorithm 5 (default 1); 0: fixed eta */
    int32_t primal_weight_update;/* 1: Algorithm 4 at restarts (default 1) */
    int32_t restarts;            /* 1: adaptive restarts of Section 2.4.2 (default 1) */
    int32_t power_iters;         /* iterations of Algorithm 2 (default 100) */
    double ruiz_tol;             /* Algorithm 3 stops when all norms are within this of 1 (1e-4) */
    double eta_scale;            /* initial eta = eta_scale / ||K~||_2 (default 0.9) */
    double beta_sufficient;      /* 0.2 */
    double beta_necessary;       /* 0.8 */
    double beta_artificial;      /* 0.36 */
    double eps_zero;             /* 1e-6 */
    double polish_switch_tol;    /* LP_PREC_MIXED: the FP32 phase runs to max(tol, this)
                                    (default 1e-5) */
    const double* x0;            /* optional warm start (unscaled primal, length n) or NULL */
    const double* y0;            /* optional warm start (unscaled dual, length m) or NULL */
    double omega0;               /* > 0: initial primal weight instead of ||c~||/||q~|| */
    double eta0;                 /* > 0: initial step size instead of eta_scale/||K~|| */
    int32_t warm_memory_space;   /* memory space of x0 / y0 */
    int32_t loop_mode;           /* 0 (default): the loop runs inside one CUDA graph with a
                                    device-side while condition; 1: the host launches the loop
                                    body graph and reads the stop flag after each body (for
                                    profilers that cannot see kernels under a conditional node) */
    int32_t infeas_detect;       /* 1 (default): Algorithm 6 (Section 2.4.5) at every KKT check on
                                    the last step's differences; a solve that finds a certificate
                                    stops with LP_PRIMAL_INFEASIBLE or LP_DUAL_INFEASIBLE */
    int32_t reserved_opts;       /* must be 0 */
    double infeas_tol;           /* tolerance of Algorithm 6, applied to the differences
                                    normalised to unit length (default 1e-6) */
    int32_t autotune;            /* 1: at the first solve of each precision, time the candidate
                                    warp-task schedules of K and K^T (nonzeros and rows per task)
                                    on the device and keep the fastest of each (a candidate must
                                    beat the default by 3 %); the summation order, and so the
                                    last bits of the result, then depends on that timing.
                                    0 (default): the largest tasks (the compiled defaults) */
    int32_t halpern;             /* 1: restarted (reflected) Halpern PDHG, the variant the
                                    Conclusion names as future work (Lu and Yang, 2024), in
                                    place of the averaged restarts: every iteration maps
                                    z -> (k+1)/(k+2) ((1+rho) T(z) - rho z) + 1/(k+2) z_anchor,
                                    T one fixed-step PDHG step (eta = eta_scale / ||K~||_2,
                                    adaptive_step ignored), k the iterations since the last
                                    restart; the candidate of a check is T(z) of the last
                                    iteration; restarts (to that candidate) follow the three
                                    criteria of Section 2.4.2 on the fixed-point residual
                                    ||z - T(z)||_P, P = [[I/tau, K~^T], [K~, I/sigma]];
                                    Algorithm 4 at restarts; Algorithm 6 is not run.
                                    lp_solve only: lp_solve_batch and lp_batch_solve return
                                    LP_NOT_SUPPORTED, the other entry points ignore it.
                                    0 (default): off */
    double halpern_reflect;      /* rho in [0, 1] (default 1: Halpern on 2T - I); the FP32
                                    phase of LP_PREC_MIXED uses min(rho, 1/2) */
    double pc_alpha;             /* alpha in [0, 2] of the Pock-Chambolle pass (default 1) */
    int32_t pc_trial_iters;      /* pock_chambolle = 2: accepted iterations of each trial
                                    solve (0, the default: 2 check_every) */
    int32_t reserved_opts2;      /* must be 0 */
    double* attempt_log;         /* optional host buffer of attempt_cap records of 9 doubles, one
                                    per step attempt of lp_solve (all phases, in order):
                                    accepted iterations before the attempt, eta tried, eta_bar
                                    of Algorithm 5 (NaN for a fixed step), eta', accepted (1/0),
                                    omega, ||dx||^2, ||dy||^2, dy^T K dx (scaled problem; NaN
                                    for a fixed step); NULL (default): no log */
    int64_t attempt_cap;         /* records attempt_log holds */
} lp_opts;

/* One record per KKT check (the start, every check_every accepted
 * iterations, and the last iteration). */
typedef struct {
    double k;            /* accepted iterations so far */
    double attempts;     /* step attempts (accepted + rejected by Algorithm 5) */
    double restart;      /* 1 if this check restarted */
    double cand_is_avg;  /* 1 if the restart candidate was the average */
    double omega;        /* primal weight after this check */
    double eta;          /* step size at this check */
    double kkt_cur;      /* KKT_omega of the current iterate (scaled problem) */
    double kkt_avg;      /* KKT_omega of the average (+inf when empty) */
    double rel_gap;      /* Section 2.3.2 relative errors of the candidate, unscaled */
    double rel_pres;
    double rel_dres;
    double kkt_cand;     /* KKT_omega of the candidate */
} lp_trace_rec;

/* Results.  x (length n) and y (length m) are caller-owned buffers in
 * memory_space; either may be NULL.  They receive the unscaled candidate of the
 * last check.  trace (host, trace_cap records) is optional. */
typedef struct {
    lp_status status;
    int32_t precision_used;      /* precision of the last phase */
    int64_t iters;               /* accepted iterations (all phases) */
    int64_t attempts;            /* step attempts (all phases) */
    int64_t restarts;
    int64_t fp64_iters;          /* accepted iterations of the FP64 phase */
    double pobj, dobj;           /* c^T x and q^T y + l^T lambda^+ + u^T lambda^- (unscaled) */
    double rel_gap, rel_pres, rel_dres;
    double omega, eta;           /* final primal weight and step size */
    double norm_K;               /* Algorithm 2 estimate of ||K~||_2 */
    double setup_s;              /* scaling + power iteration + casts (host wall clock) */
    double solve_s;              /* iterations (host wall clock) */
    int64_t kernel_launches;     /* kernels this call launched (graph bodies included) */
    double* x;
    double* y;
    int32_t memory_space;        /* of x and y */
    int32_t split_rows;          /* rows of K and K^T whose products the SpMV schedules of the
                                    first phase's precision (FP32 for LP_PREC_MIXED) cut into
                                    pieces on several warps (long rows of unbalanced
                                    schedules; the results do not depend on it) */
    lp_trace_rec* trace;
    int64_t trace_cap;
    int64_t trace_len;           /* records produced (may exceed trace_cap) */
    double pc_alpha_used;        /* alpha of the Pock-Chambolle pass of the solve (NaN: none) */
    int64_t attempt_len;         /* records written to opts->attempt_log (at most attempt_cap) */
} lp_result;

/* Fills *opts with the defaults listed above.  No CUDA call. */
void lp_opts_default(lp_opts* opts);

/* Copies the LP (Section 2.2) to the current device, validates it on the
 * device (row_ptr monotone and in range, col_idx in [0, n), no NaN, l <= u) and
 * builds the transposed CSR K^T (Section 2.3, products K^T y) and the row-block
 * schedules of both matrices.  cuda_stream: a cudaStream_t or NULL.
 * Errors: LP_INVALID_ARGUMENT (NULL pointers, bad sizes, failed validation),
 * LP_OUT_OF_MEMORY, LP_CUDA_ERROR.  On error *out is NULL. */
lp_status lp_create(const lp_desc* desc, void* cuda_stream, lp_handle* out);

/* Restarted PDHG (Algorithm 1 with theta = 1; Ruiz scaling, Algorithm 3;
 * step size from Algorithm 2; adaptive restarts, Section 2.4.2; primal weight,
 * Algorithm 4; adaptive steps, Algorithm 5; termination, Section 2.3.2, on the
 * unscaled problem; infeasibility detection, Algorithm 6, when
 * opts->infeas_detect).  The iteration loop runs on the device inside a CUDA
 * graph with a device-side while condition; the host waits once at the end.
 * Returns the solver outcome (LP_OPTIMAL, LP_PRIMAL_INFEASIBLE,
 * LP_DUAL_INFEASIBLE, LP_ITERATION_LIMIT, LP_TIME_LIMIT, LP_NUMERICAL_ERROR),
 * also stored in res->status, or a negative error. */
lp_status lp_solve(lp_handle h, const lp_opts* opts, lp_result* res);

/* Solves count independent LPs with the same options; results[i] belongs to
 * hs[i] (lp_batch_create + lp_batch_solve + lp_batch_destroy).  Returns LP_OK
 * when every LP has an outcome (in results[i].status), else a negative error. */
lp_status lp_solve_batch(const lp_handle* hs, int32_t count, const lp_opts* opts,
                         lp_result* results);

/* A batch: the LPs of count handles stacked into one block-diagonal problem on
 * the device (copied from the handles; later changes to them are not seen).
 * Solving it runs every LP's restarted PDHG together: one launch per kernel covers
 * all LPs (warp tasks never span two LPs), while Ruiz stopping, the spectral norm,
 * eta_0, omega_0, step sizes, restarts, primal weights and termination stay per LP
 * exactly as in lp_solve; an LP that finishes stops consuming work.  The loop runs
 * in one CUDA graph (device-side while condition) until every LP is done.
 * LP_PREC_MIXED runs FP32 iterations with FP64 reductions to
 * max(tol, polish_switch_tol); the LPs that phase declares optimal then go to an
 * FP64 phase from their candidates, whose first check re-evaluates the relative
 * errors in FP64: LP_OPTIMAL stands only if they hold there, otherwise (and below
 * the hand-over tolerance) FP64 iterations continue to tol, as in lp_solve.
 * Traces, warm starts and Pock-Chambolle trials (pock_chambolle = 2) are not
 * supported (traces and warm starts are ignored; the trials return
 * LP_NOT_SUPPORTED). */
typedef struct lp_batch_s* lp_batch;
lp_status lp_batch_create(const lp_handle* hs, int32_t count, void* cuda_stream, lp_batch* out);
lp_status lp_batch_solve(lp_batch b, const lp_opts* opts, lp_result* results);
void lp_batch_destroy(lp_batch b);

/* Gradient of a loss L(x_K) through K_iters unrolled fixed-step PDHG
 * iterations (Algorithm 1, theta = 1, unscaled problem, start x = proj_X(0),
 * y = 0) with tau = eta / omega, sigma = eta * omega held constant; eta and
 * omega come from opts->eta0 / opts->omega0 when positive, else
 * eta_scale / ||K||_2 (Algorithm 2 on the unscaled K) and ||c|| / ||q||.
 * opts->precision selects FP64 or FP32 arithmetic.  Iterates are checkpointed
 * every ckpt_every iterations and recomputed segment by segment.
 * dL_dxK[n]: input adjoint.  Outputs (caller-owned, overwritten): dc[n],
 * dq[m], dvals[nnz] in the nonzero order of lp_desc, and x_K[n] if not NULL.
 * All of them live in memory_space.  tau_sigma_out (host, 2 doubles, or NULL)
 * receives the tau and sigma used. */
lp_status lp_grad(lp_handle h, const lp_opts* opts, int32_t K_iters, int32_t ckpt_every,
                  const double* dL_dxK, double* dc, double* dq, double* dvals,
                  double* x_K, int32_t memory_space, double* tau_sigma_out);

/* Forward part of lp_grad: K_iters unrolled fixed-step iterations with the
 * same start, step sizes and precision rules; writes x_K[n] and/or y_K[m]
 * (either may be NULL, not both) in memory_space.  tau_sigma_out as in lp_grad. */
lp_status lp_unroll(lp_handle h, const lp_opts* opts, int32_t K_iters, double* x_K, double* y_K,
                    int32_t memory_space, double* tau_sigma_out);

/* Algorithm 7 (fishnet casting, Section 2.5): a multi-start warm start.  On
 * the scaled problem that lp_solve would build with the same opts (Ruiz per
 * ruiz_iters, eta = eta_scale / ||K~||_2 or eta0, omega = ||c~|| / ||q~|| or
 * omega0): P points x~_p = (||K~||_2 / sqrt(n)) g_p and Y = K~ X; then rounds of
 * k_steps fixed-step PDHG iterations (Algorithm 1) on all points, each round
 * keeping the half with the smallest |duality gap| and, at odd rounds while
 * more than two points entered the round, adding one convex combination of the
 * survivors per survivor (weights |z| / sum |z|), until one point is left.
 *   P        number of points, a power of two in 1..64
 *   G        n*P standard-normal draws, G[j*P + p] for coordinate j of point p
 *   Z        nZ normal draws for the repopulations; lp_fishnet_draws(P) of them
 *            are used, in order (fewer: LP_INVALID_ARGUMENT)
 *   x0, y0   receive the surviving point, unscaled (x0[n], y0[m]); pass them to
 *            lp_solve as opts.x0 / opts.y0 for the warm start
 *   gaps     host array of rounds*P doubles or NULL: the |gap| of each point of a
 *            round before its cull, gaps[round*P + point]
 *   rounds   host int32 or NULL: number of rounds
 * G, Z, x0 and y0 live in memory_space.  opts.precision selects the point
 * blocks and products: LP_PREC_FP64 (the cull decisions then match an FP64
 * evaluation) or LP_PREC_MIXED (FP32 blocks and products, FP64 gap reductions).
 * The blocks (n x P and m x P, about s (3n + 4m) P bytes for s-byte values) are
 * allocated for the call and freed before it returns.  The random draws are
 * inputs, so the result is deterministic. */
lp_status lp_fishnet(lp_handle h, const lp_opts* opts, int32_t P, int32_t k_steps,
                     const double* G, const double* Z, int64_t nZ, double* x0, double* y0,
                     double* gaps, int32_t* rounds, int32_t memory_space);

/* Number of repopulation draws lp_fishnet consumes for P points (-1 for an
 * invalid P).  Host only. */
int64_t lp_fishnet_draws(int32_t P);

/* Replaces values of the LP on its existing sparsity pattern: vals[nnz] (in
 * lp_desc's nonzero order), c[n], q[m], l[n], u[n]; a NULL pointer keeps the old
 * array.  The same validation as lp_create (LP_INVALID_ARGUMENT on NaN, l > u).
 * The next lp_solve / lp_grad / lp_unroll uses the new values. */
lp_status lp_update_values(lp_handle h, const double* vals, const double* c, const double* q,
                           const double* l, const double* u, int32_t memory_space);

/* Measurement hook: runs `reps` PDHG step attempts of the given precision on
 * the state left by the last lp_solve of that precision (the Halpern step
 * kernels when that solve ran lp_opts.halpern = 1), timing each kernel
 * class with CUDA events on the handle's stream.  ms_out (host, 4 doubles)
 * receives the mean milliseconds per launch of: [0] primal update,
 * [1] K x' SpMV + dual update, [2] K^T y' SpMV + step terms, [3] step control.
 * bytes_out (host, 4 doubles, or NULL) receives the algorithmic bytes per launch
 * of the same kernels.  The solver state afterwards is unspecified. */
lp_status lp_profile_step(lp_handle h, int32_t precision, int32_t reps, double* ms_out,
                          double* bytes_out);

/* Measurement hook: the gather ceiling of the two SpMV products on this
 * handle's scaled matrices (the products of Algorithm 1).  A minimal kernel
 * streams the nonzeros of K (then of K^T) with coalesced 16-byte loads of values
 * and column indices, gathers the vector entry of each nonzero (x of the last
 * lp_solve of that precision for K, y for K^T; through L1 when the vector takes
 * at most 96 KB, else with loads that do not allocate in L1, as the SpMV kernels
 * do) and multiply-adds it into a per-thread sum: the same request stream as the
 * SpMV kernels without their row structure and epilogues.  Grid:
 * blocks_per_sm (1..8) x the SM count, 256 threads.  ms_out (host, 2 doubles)
 * receives the mean milliseconds per launch over `reps` launches after one
 * warm-up: [0] K side, [1] K^T side.  Requires an lp_solve of that precision on
 * the handle first and a problem large enough for the per-thread sums to fit
 * the handle's scratch (LP_INVALID_ARGUMENT otherwise).  Solver state is kept. */
lp_status lp_profile_gather(lp_handle h, int32_t precision, int32_t reps, int32_t blocks_per_sm,
                            double* ms_out);

/* Termination quantities of one primal-dual pair (x, y) of the LP in desc,
 * computed on the device WITHOUT allocating any device memory.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc when they check a point: hosts that forbid device allocation after
 * start-up (an allocation can block or synchronise the device), or plugins
 * inside an application that owns all device memory.
 * desc: every array in device memory (memory_space = LP_MEM_DEVICE); it is not
 * copied and not validated beforehand, but every row pointer and column index is
 * range-checked on the device (LP_INVALID_ARGUMENT if one is out of range).
 * x[n], y[m]: device.  omega > 0: weight of KKT_omega.  out (host, 8 doubles):
 * [0] c^T x  [1] q^T y + l^T lambda^+ + u^T lambda^-  [2] primal residual norm
 * [3] dual residual norm  [4] rel_gap  [5] rel_pres  [6] rel_dres  [7] KKT_omega
 * (the quantities of lp_result / lp_trace_rec, unscaled).  cuda_stream: a
 * cudaStream_t or NULL; the call copies `out` to the host and returns after that
 * stream finished its work, so it returns LP_NOT_SUPPORTED, launching nothing,
 * when the stream is being captured.  An error already pending in the CUDA
 * runtime when the call starts is returned as LP_CUDA_ERROR and left pending.
 * Scratch: a fixed device array of LP_KKT_NOALLOC_MAX_DOUBLES doubles (8 MiB)
 * compiled into the library, held by every GPU that loads the library until the
 * process exits; problems with m + n + 1800 > LP_KKT_NOALLOC_MAX_DOUBLES are
 * rejected with LP_INVALID_ARGUMENT.  Each call looks up the array's device
 * address (cudaGetSymbolAddress) on the current device; the first call on a
 * device may also load the library's device code there, so make one call at
 * start-up.  All calls share the array and every call overwrites it (what must
 * start at zero is cleared by each call): calls whose work overlaps on the GPU
 * race and must be serialised by the caller. */
#define LP_KKT_NOALLOC_MAX_DOUBLES 1048576
lp_status lp_kkt_noalloc(const lp_desc* desc, const double* x, const double* y, double omega,
                         double* out, void* cuda_stream);

/* Releases the handle and all its device memory.  NULL is ignored. */
void lp_destroy(lp_handle h);

/* Static, NUL-terminated name of a status. */
const char* lp_status_string(lp_status s);

/* LP_ABI_VERSION of the library. */
int32_t lp_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_PDHG_LP_H */

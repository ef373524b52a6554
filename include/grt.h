/*
 * grt.h -- C ABI of libgrt, the GB300 (sm_103a) point solver for semilinear
 * parabolic PDEs by generalized random trees and Pade resummation
 * (Acebron & Rodriguez-Rozas, arXiv 2402.06491).
 *
 * Problem (Sec. 1, Eq. nonlinear_new, with L = D * Laplacian):
 *     u_t = D Lap(u) + f(u),  x in R^d,  t > 0,     u(x, 0) = u0(x),
 *     f(u) = sum_{k=0}^{deg} b_k u^k.
 * A point solve estimates u(x_i, t_i) from N_i random trees per point:
 *   - each tree is a branching Brownian motion (Sec. 2.1 algorithm, Fig. 1)
 *     generated by Strategy A (exponential clock, Eqs. probexp1-probexp2) or
 *     Strategy B (coin xi + uniform split time, Eqs. totalduhamel_B,
 *     probexpB1, probexpBclosed);
 *   - its weight (the multiplicative functional of Eqs. rep_strategyB /
 *     probexpBclosed) is binned by its number of splitting events Ne into the
 *     coefficient a_Ne of a possibly divergent series, trees with Ne > K being
 *     pruned (Sec. 2.4);
 *   - the series is summed by an [L/M] Pade approximant at eps = 1
 *     (Sec. 2.1 end, Sec. 2.4), in FP64.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *     key = (seed mod 2^32, seed >> 32),
 *     ctr = (lo32(id), hi32(id), tree | sub << 31, point_base + i),
 * where id is the node's path label (root 0, child j of id is 16 id + j + 1).
 * Results therefore depend only on (problem, point_base + i, x_i, t_i, N_i,
 * K, L, M, seed) -- not on batching, scheduling or other points in the call.
 *
 * Conventions for every call:
 *   - return value 0 (GRT_OK) or a negative GRT_E* code; the reason is kept
 *     in the context and returned by grt_last_error();
 *   - the caller owns every array passed in; the library never keeps a
 *     pointer to a caller array after the call returns (grt_plan_execute
 *     excepted: it reads and writes the device arrays asynchronously on the
 *     given stream until that stream reaches the end of the call's work);
 *   - a context and its plans are not thread-safe: use one per host thread;
 *   - arrays are row-major; x holds n rows of dim doubles.
 */
#ifndef GRT_H
#define GRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRT_MAX_DIM 3
#define GRT_MAX_DEG 15
#define GRT_MAX_K 16
#define GRT_MAX_TREES_PER_POINT 2147483647ull

/* Return codes. */
#define GRT_OK 0
#define GRT_EINVAL (-1)   /* an argument is outside its documented range     */
#define GRT_ENOMEM (-2)   /* device or pinned host memory could not be had   */
#define GRT_EDEVICE (-3)  /* a CUDA call failed (no device, launch error...) */
#define GRT_ENOTSUP (-5)  /* valid request the library does not support      */
#define GRT_EAGAIN 1      /* (grt_poll) the request has not finished yet      */

/* Strategy (Sec. 2.1 / Sec. 2.2). */
#define GRT_STRATEGY_A 0
#define GRT_STRATEGY_B 1

/* Branching law over the nonzero terms b_k of F (A) or f (B). */
#define GRT_ARITY_UNIFORM 0  /* p_k uniform: the paper's choice (Sec. 2.1 after Eq. probexp2) */
#define GRT_ARITY_ABS_COEF 1 /* p_k proportional to |b_k|, weight b_k / p_k                 */

/* Arithmetic of the tree walk (the Pade always runs in FP64). */
#define GRT_FP32 0
#define GRT_FP64 1

/* Initial data u0 = g (parameters p[0..7]). */
#define GRT_U0_CONST 0     /* p0                                              */
#define GRT_U0_GAUSS 1     /* p0 + p1 exp(-|x - (p3,p4,p5)|^2 / (2 p2^2))     */
#define GRT_U0_COS_PROD 2  /* p0 + p1 prod_i cos(p[2+i] x_i)                  */
#define GRT_U0_TANH_PROD 3 /* p0 + p1 prod_i tanh(x_i - p[2+i])               */
#define GRT_U0_LOGISTIC 4  /* p0 + p1 / (1 + exp(-(x_0 - p2) / p3))           */
#define GRT_U0_GAUSS_AXES 5 /* p0 + p1 exp(-sum_i p_{2+i} (x_i - p_{5+i})^2)  */
#define GRT_U0_QUADRATIC 6  /* p0 + sum_i (p_{1+i} x_i + p_{4+i} x_i^2)        */

/* Path law of a segment (Eqs. green, SDE: L = a_ij d_i d_j + b_i d_i, sigma^2 = a).
 * GRT_SDE_HEAT: L = D Lap, each segment one exact Gaussian increment of
 * variance 2 D s per axis.  GRT_SDE_AFFINE: per axis
 *   dX_i = (beta_i - kappa_i X_i) dt + (s_i + r_i X_i) dW_i,
 * sde_param = {beta[3], kappa[3], s[3], r[3]}, D unused, by Euler-Maruyama
 * (the Euler scheme of Sec. 2.4) with sde_steps equal steps per segment;
 * the normals come from Philox4x32-10 blocks at the node's counter with the
 * sub bit set, block b under the key (k0 ^ (b+1) 0x2545F491, k1 ^ (b+1)
 * 0x6C8E9CF5), Box-Muller on its word pairs: for d <= 2 block b serves steps
 * 2b ((w0, w1)) and 2b + 1 ((w2, w3)); for d = 3 block b serves step b. */
#define GRT_SDE_HEAT 0
#define GRT_SDE_AFFINE 1

/* Variable coefficients c_k(x, t) = b_k gamma(x, t) of the terms selected by
 * coef_mask (Sec. 1, Eq. nonlinear_new; Example 5 uses -e^{-x^2}/(t + 0.1) u^2).
 * The split weight of a term k with bit k set is multiplied by gamma at the
 * particle's position at the split and at the PDE time left to its children
 * (Sec. 2.1, Eq. probexp1: c_j(beta(S), t - S)).  Parameters coef_param[0..7]: */
#define GRT_COEF_CONST 0        /* gamma = 1 (coef_mask ignored)                           */
#define GRT_COEF_GAUSS_OVER_T 1 /* exp(-sum_i p_i (x_i - p_{3+i})^2) / (t + p6), p6 > 0     */
#define GRT_COEF_GAUSS 2        /* exp(-sum_i p_i (x_i - p_{3+i})^2)                        */

/* Per-point status bits. */
#define GRT_STATUS_PADE_SINGULAR 1  /* a Pade pivot was below 1e-14 of the largest matrix
                                       entry: the type was lowered [L-1/M-1] until solvable */
#define GRT_STATUS_PADE_POLE_NEAR 2 /* |Q(1)| < 1e-8                                   */
#define GRT_STATUS_SERIES_PARTIAL 4 /* fewer trees than requested contributed (grt_cancel) */
#define GRT_STATUS_HIGH_PRUNE 8     /* more than 1% of the trees had Ne > K            */

/* Problem description (copied by grt_create). */
typedef struct grt_problem {
    int32_t dim;                       /* d in {1, 2, 3}                                      */
    double D;                          /* diffusion constant >= 0 (variance 2 D tau per axis) */
    int32_t f_deg;                     /* 0 <= deg <= GRT_MAX_DEG                             */
    double f_coef[GRT_MAX_DEG + 1];    /* b_0 .. b_deg; entries above deg are ignored         */
    int32_t u0_kind;                   /* GRT_U0_*                                            */
    double u0_param[8];
    int32_t strategy;                  /* GRT_STRATEGY_A | GRT_STRATEGY_B                     */
    double lambda;                     /* A: clock rate lambda > 0                            */
    double c_pot;                      /* A: potential c pulled out of f, F(u) = f(u) + c u   */
    double q;                          /* B: leaf probability, 0 < q < 1                      */
    int32_t arity_law;                 /* GRT_ARITY_*                                         */
    int32_t precision;                 /* GRT_FP32 | GRT_FP64 (walk arithmetic)               */
    int32_t coef_kind;                 /* GRT_COEF_*; Strategy A rejects a variable linear    */
    double coef_param[8];              /*   term (mask bit 1) together with c_pot != 0        */
    uint32_t coef_mask;                /* bit k: c_k(x, t) = b_k gamma(x, t), k <= f_deg      */
    int32_t sde_kind;                  /* GRT_SDE_*                                           */
    int32_t sde_steps;                 /* AFFINE: Euler steps per segment, 1..4096            */
    double sde_param[12];              /* AFFINE: beta[3], kappa[3], s[3], r[3]               */
} grt_problem;

typedef struct grt_ctx grt_ctx;
typedef struct grt_plan grt_plan;

/* Create a context for one problem on CUDA device `device`.
 * Validates the problem (dim, deg, D >= 0, lambda > 0 for A, 0 < q < 1 for B,
 * u0 kind, precision), builds the branching-law tables (Sec. 2.1 Eq. probexp2,
 * Sec. 2.2 Eq. probexpB1) and selects the kernels.  On GRT_EINVAL/GRT_EDEVICE
 * *out is set to NULL and no context exists (grt_last_error(NULL) then gives
 * the reason of the last failed create in this thread). */
int grt_create(const grt_problem *pb, int device, grt_ctx **out);

/* Release the context, its cached device buffers and its stream.  Plans made
 * from it must be destroyed first.  NULL is ignored. */
void grt_destroy(grt_ctx *ctx);

/* Text of the last error on this context (or of the last failed grt_create in
 * this thread when ctx is NULL).  Owned by the library; valid until the next
 * call on the same context. */
const char *grt_last_error(const grt_ctx *ctx);

/* Synchronous point solve with HOST arrays (the boundary of Sec. 3's
 * "probabilistic part": interface values at single points).
 *   n          number of points, 0 <= n < 2^31 (n = 0 returns GRT_OK at once)
 *   x          [n][dim] positions; t [n] times >= 0; ntrees [n] trees per point,
 *              0 <= N_i <= GRT_MAX_TREES_PER_POINT
 *   K, L, M    series order 0 <= K <= GRT_MAX_K; Pade type with L, M >= 0, L + M <= K
 *   seed       Philox key; point_base: global index of point 0 (for sharding:
 *              the stream of point i is keyed by point_base + i < 2^32)
 *   u_out      [n] Pade value; coef_out / se_out [n][K+1] coefficients a_n and
 *              their standard errors (either may be NULL); status_out [n] bits
 *              (may be NULL).
 * Copies the inputs to the device, runs the walk and the FP64 finalize, and
 * copies the results back before returning. */
int grt_solve(grt_ctx *ctx, int64_t n, const double *x, const double *t, const uint64_t *ntrees, int K,
              int L, int M, uint64_t seed, uint64_t point_base, double *u_out, double *coef_out,
              double *se_out, int32_t *status_out);

/* The plain FP64 point solve: one kernel launch per point, same arguments and
 * HOST arrays as grt_solve (the FP64 comparison path of the serving figures;
 * the walk runs in FP64 whatever the context's precision).  For each point, in
 * order, one launch of min(ceil(N_i / 128), 8 x SMs) blocks of 128 threads:
 * thread g walks trees g, g + G, ... (G threads) of the point's stream (the
 * algorithm after Sec. 2.1 Eq. recursion / Sec. 2.2), adds each tree's weight
 * to its own FP64 per-order sums, the sums are reduced by warp shuffles and
 * then per block in a fixed order, and the launch's last block adds the block
 * partials in block order, forms a_n and SE_n (Sec. 2.4, Eq.
 * simplecase_discrete) and the FP64 [L/M] Pade (Sec. 2.1 end, Sec. 2.4).
 * Results agree with grt_solve on an FP64 context up to the rounding of the
 * different summation order.  GRT_EINVAL as grt_solve; synchronous. */
int grt_solve_plain(grt_ctx *ctx, int64_t n, const double *x, const double *t, const uint64_t *ntrees, int K,
                    int L, int M, uint64_t seed, uint64_t point_base, double *u_out, double *coef_out,
                    double *se_out, int32_t *status_out);

/* Device-resident form, for callers that keep their points in device memory
 * and launch many solves of the same shape (e.g. under a CUDA graph).
 * grt_plan_create fixes n, the per-point tree budgets (HOST array, copied) and
 * K, L, M, lays out the (point, tree-tile) work items and allocates every
 * device buffer the solve needs; grt_plan_execute then allocates nothing.  A
 * plan whose tree records span 2^32 slots or more (about 4.3e9 trees) is
 * walked as several launches over consecutive point ranges (the results are
 * the same; grt_plan_launches counts them). */
int grt_plan_create(grt_ctx *ctx, int64_t n, const uint64_t *ntrees, int K, int L, int M, grt_plan **out);

/* Enqueue one solve on `stream` (a cudaStream_t; NULL = legacy default stream).
 * d_x [n][dim], d_t [n] are DEVICE arrays (t must be finite and >= 0: it is not
 * checked here); d_u [n], d_coef / d_se [n][K+1] (may be NULL), d_status [n]
 * (may be NULL) are DEVICE outputs.  Returns after enqueueing; launch errors
 * are reported, results are ready when the stream reaches them.  Executions of
 * one plan must not overlap in time (they share the plan's work buffers). */
int grt_plan_execute(grt_plan *plan, const double *d_x, const double *d_t, uint64_t seed, uint64_t point_base,
                     double *d_u, double *d_coef, double *d_se, int32_t *d_status, void *stream);

/* Work counters of the plan's last execution (synchronises with it), summed
 * over all points: nodes visited, splitting events (internal nodes, counting
 * the split that prunes a tree) and trees pruned (Ne > K).  Any output may
 * be NULL. */
int grt_plan_counters(grt_plan *plan, uint64_t *nodes, uint64_t *splits, uint64_t *pruned);

/* Kernel timing: when enabled (on != 0), every grt_plan_execute records CUDA
 * events on its stream around the walk kernel and the finalize kernel.
 * grt_plan_timing waits for the last execution's events and returns the two
 * durations in milliseconds (GRT_EINVAL if timing was off for it). */
int grt_plan_set_timing(grt_plan *plan, int on);
int grt_plan_timing(grt_plan *plan, float *walk_ms, float *finalize_ms);

/* Number of kernel launches one grt_plan_execute enqueues. */
int grt_plan_launches(const grt_plan *plan);

/* Launch shape of the FP32 walk, cfg [4] = {warps per block (4 | 8), stack
 * levels kept in shared memory (0 = all K | 3 = the top three, deeper ones in
 * local memory), resident blocks per SM to launch (0 = all that fit), trees per
 * work-queue chunk (multiple of 32)}.  The shape never changes a result: the
 * same trees are walked and their records are binned in the same order.  The
 * FP64 walk has one shape.  Default {4, 0, 0, 512}. */
int grt_plan_set_config(grt_plan *plan, const int32_t *cfg);
int grt_plan_get_config(const grt_plan *plan, int32_t *cfg);

/* The same launch shape for the context's one-shot grt_solve (for instance the
 * shape grt_plan_autotune found for a plan of that workload).  Results do not
 * change.  GRT_EINVAL for a shape outside the list above.  grt_solve_noalloc and
 * the server keep the default shape. */
int grt_set_solve_config(grt_ctx *ctx, const int32_t *cfg);

/* Autotuner (batching of uneven budgets into one launch): runs the plan on the
 * given device buffers once per candidate shape (a warm run plus two timed runs,
 * CUDA events on `stream`), keeps the fastest walk, and returns it in cfg_out
 * [4] (may be NULL).  Leaves the outputs of a full solve in the buffers. */
int grt_plan_autotune(grt_plan *plan, const double *d_x, const double *d_t, uint64_t seed, uint64_t point_base,
                      double *d_u, double *d_coef, double *d_se, int32_t *d_status, void *stream, int32_t *cfg_out);

/* CUDA graph of one execution of the plan on fixed device buffers (the
 * arguments of grt_plan_execute): capture runs the plan once normally (on the
 * context's own stream) and then records one execution into a graph owned by
 * the plan; launch replays it on `stream`.  A new capture replaces the old. */
int grt_plan_graph_capture(grt_plan *plan, const double *d_x, const double *d_t, uint64_t seed, uint64_t point_base,
                           double *d_u, double *d_coef, double *d_se, int32_t *d_status);
int grt_plan_graph_launch(grt_plan *plan, void *stream);

/* Release a plan.  NULL is ignored. */
void grt_plan_destroy(grt_plan *plan);

/* Cancellation factor kappa_n = SA_n / |S1_n| (sum of |W| over the sum of W of the
 * trees of order n; Sec. 2.4, Eq. simplecase_discrete: a_n is the sample mean of
 * those weights) of every point of the plan's last execution, from its
 * resident per-chunk sums: a kappa far above 1 says that order's mean is a
 * small difference of large weights (its relative statistical error grows
 * with kappa).  d_kappa: DEVICE [n][K+1]; 0 where no tree has that order, +inf
 * where S1 = 0 < SA.  Enqueued on `stream` (NULL = legacy default stream),
 * after the execution it reads (same stream, or ordered by the caller).
 * GRT_EINVAL if d_kappa is NULL (n > 0) or the plan has never been executed. */
int grt_plan_kappa(grt_plan *plan, double *d_kappa, void *stream);

/* Per-result statistical error of the Pade value (Sec. 2.4: the Pade value is
 * Lipschitz in the coefficients, Wuytack bound): err_i = sqrt(sum_j (du/da_j
 * SE_j)^2) over j = 0..L+M, the derivatives by central differences of the FP64
 * approximant with steps h_j = 1e-6 max(|a_j|, 1e-12 max_i |a_i|) -- a
 * first-order estimate of the spread of u over independent tree samples.
 * d_coef, d_se: DEVICE [n][K+1] (as written by the solves); d_err: DEVICE [n];
 * +inf where an evaluation is not finite.  Enqueued on `stream` (NULL =
 * legacy default stream).  GRT_EINVAL for bad sizes or NULL arrays. */
int grt_pade_error(grt_ctx *ctx, int64_t n, int K, int L, int M, const double *d_coef, const double *d_se,
                   double *d_err, void *stream);

/* The FP64 [L/M] Pade stage alone (Sec. 2.1 end, Sec. 2.4), on the GPU, for
 * n series given on the HOST as coef [n][K+1] (K >= L + M).  Writes u_out [n]
 * and status_out [n] (may be NULL; only the PADE_* bits are set). */
int grt_pade(grt_ctx *ctx, int64_t n, int K, int L, int M, const double *coef, double *u_out,
             int32_t *status_out);

/* Per-tree records for trees [first_tree, first_tree + ntrees) of one point,
 * generated on the GPU with the context's walk arithmetic (HOST arrays):
 * order [ntrees] (Ne, or K+1 when pruned), w [ntrees] tree weight (0 when
 * pruned), nodes [ntrees] nodes visited, hash [ntrees] FNV-1a-64 over the node
 * codes (0 leaf, term index + 1 split) in preorder.  Any output may be NULL.
 * A diagnostic of the same streams the point solve uses (Sec. 2.2, Fig. 2). */
int grt_trees(grt_ctx *ctx, const double *x, double t, uint64_t point_index, uint64_t first_tree, uint64_t ntrees,
              int K, uint64_t seed, int32_t *order, double *w, uint32_t *nodes, uint64_t *hash);

/* ---- Serving: continuous batching of point-solve requests (the serving form
 * of the probabilistic part of the PDD, Sec. 3). ----------------------------
 * A server owns a scheduler thread and a device-memory budget on one device.
 * Requests (a problem context, points, per-point tree budgets, K, L, M, seed)
 * may be submitted at any time from any thread; each is admitted when its
 * resident state fits the budget, first come first admitted: per point one
 * accumulator (for every order and statistic, the compensated sum of the
 * point's per-8192-tree chunk sums so far) and its result row.  The scheduler
 * runs the GPU in steps of at most `step_trees` trees taken from all admitted
 * requests, smallest remaining work first, in ranges that start on a point's
 * 8192-tree boundaries; requests of one problem, K, L, M and seed share one
 * walk and one binning launch per step; the groups of one step run
 * concurrently on several streams.  A point's result is identical, bit for
 * bit, to grt_solve of the same point (same point_base + index and seed),
 * alone or in any mix.  Batching happens at step boundaries: a request that
 * arrives while others run joins the next step (steps of at most step_trees
 * trees, a few milliseconds at full load).  Contexts passed to grt_submit must
 * outlive their requests. */
typedef struct grt_server grt_server;

/* Memory of a server with steps of step_trees trees (0: 2^27): *step_bytes for
 * its step buffers, *point_bytes per admitted point (either may be NULL).  A
 * server with budget B admits floor((B - step_bytes) / point_bytes) points at a
 * time.  GRT_EINVAL for step_trees outside [8192, 2^31]. */
int grt_server_sizes(uint64_t step_trees, uint64_t *step_bytes, uint64_t *point_bytes);

/* mem_budget_bytes: device memory for step buffers and resident state, at
 * least step_bytes (grt_server_sizes) + 1 MiB; step_trees: trees per step
 * (0: 2^27).  GRT_EINVAL if the budget is too small, GRT_ENOMEM / GRT_EDEVICE
 * on failure. */
int grt_server_create(int device, uint64_t mem_budget_bytes, uint64_t step_trees, grt_server **out);

/* Stop the scheduler (after its current step) and free the server and any
 * requests not yet polled.  NULL is ignored. */
void grt_server_destroy(grt_server *s);

const char *grt_server_last_error(const grt_server *s);

/* Copy a request's inputs (HOST arrays, grt_solve's layout) and queue it;
 * returns at once with *request_id.  GRT_ENOMEM if the request alone exceeds
 * the budget. */
int grt_submit(grt_server *s, grt_ctx *ctx, int64_t n, const double *x, const double *t, const uint64_t *ntrees, int K,
               int L, int M, uint64_t seed, uint64_t point_base, uint64_t *request_id);

/* Wait up to timeout_ms (0: do not wait, < 0: wait until done) for a request.
 * Done: writes u_out [n], coef_out / se_out [n][K+1], status_out [n] (any may be
 * NULL) and *latency_s (submit to completion), releases the request and returns
 * GRT_OK (or the request's error).  Not done: GRT_EAGAIN. */
int grt_poll(grt_server *s, uint64_t request_id, int timeout_ms, double *u_out, double *coef_out, double *se_out,
             int32_t *status_out, double *latency_s);

/* Per-request figures returned by grt_poll_ex. */
typedef struct grt_request_info {
    double latency_s;          /* submit to completion                                    */
    uint64_t shared_launches;  /* walk launches that also walked another request's trees  */
    uint64_t shared_steps;     /* scheduler steps that also ran another request's trees   */
    int32_t cancelled;         /* grt_cancel was called before the request finished       */
} grt_request_info;

/* grt_poll with the number of trees each point's estimate used: ntrees_done [n]
 * (may be NULL; N_i unless the request was cancelled) and *info (may be NULL). */
int grt_poll_ex(grt_server *s, uint64_t request_id, int timeout_ms, double *u_out, double *coef_out, double *se_out,
                int32_t *status_out, uint64_t *ntrees_done, grt_request_info *info);

/* Stop a request early (a caller's deadline: grt_poll with a timeout, then
 * grt_cancel).  The request takes no more trees after the step in progress;
 * each point that has not received all its trees is then completed from the
 * trees already binned -- N_done of them, the first N_done trees of the point's
 * stream, a multiple of 8192 -- and gets GRT_STATUS_SERIES_PARTIAL: its a_n,
 * SE_n and Pade value are those of grt_solve with N_i = N_done, bit for bit
 * (the trees are independent samples, Sec. 3, so the estimate stays unbiased,
 * with the larger error of N_done trees).  A request still waiting for
 * admission ends with N_done = 0 (u = 0, a_n = 0).  Poll it as usual.  GRT_OK
 * also for a request that has already finished; GRT_EINVAL for an unknown id. */
int grt_cancel(grt_server *s, uint64_t request_id);

/* Steps run, trees walked, kernel launches, resident bytes, pending and active
 * requests, walk launches that batched trees of several requests, requests
 * cancelled before they finished (any output may be NULL). */
int grt_server_stats(grt_server *s, uint64_t *steps, uint64_t *trees, uint64_t *launches, uint64_t *resident_bytes,
                     uint64_t *pending_requests, uint64_t *active_requests, uint64_t *shared_launches,
                     uint64_t *cancelled_requests);

/* Limits of grt_solve_noalloc. */
#define GRT_NOALLOC_MAX_POINTS 4096
#define GRT_NOALLOC_MAX_TREES 524288ull /* summed over the call's points */

/* Point solve that allocates no memory (the paper has no counterpart: this is
 * a service for callers that cannot allocate device memory when they solve:
 * an application whose own pool allocator has reserved the device memory, or
 * code on a latency-critical path where a cudaMalloc, which may synchronise
 * the device, is not acceptable).
 * Same arguments and results as grt_plan_execute, without a plan: d_x [n][dim],
 * d_t [n], d_u [n], d_coef / d_se [n][K+1] (may be NULL), d_status [n] (may be
 * NULL) are DEVICE arrays owned by the caller; ntrees [n] is a HOST array.  The
 * work area of the solve is one fixed array of about 7 MB of device memory
 * that the library holds on every GPU that loads it until the process exits.
 * Limits: n <= GRT_NOALLOC_MAX_POINTS and sum(ntrees) <= GRT_NOALLOC_MAX_TREES,
 * else GRT_EINVAL with a message.  The first call on a device looks up the
 * work area's device address; make that first call before any stream capture.
 * Enqueued on `stream` (NULL = legacy default stream); returns after enqueueing.
 * All calls share the one work area, which keeps the last call's contents
 * (each call clears what must start at zero): calls whose GPU work can overlap
 * in time (different streams, or different host threads) race and must be
 * serialised by the caller.  The host-side part of concurrent calls is
 * serialised by the library. */
int grt_solve_noalloc(grt_ctx *ctx, int64_t n, const double *d_x, const double *d_t, const uint64_t *ntrees, int K,
                      int L, int M, uint64_t seed, uint64_t point_base, double *d_u, double *d_coef, double *d_se,
                      int32_t *d_status, void *stream);

/* ======================================================================== */
/* Probabilistic domain decomposition (Sec. 3): interfaces -> spline ->     */
/* independent subdomain solves.                                            */
/* ======================================================================== */

/* Tensor-product not-a-knot cubic spline on a uniform grid (Sec. 3,
 * "Interpolation": nodal points uniformly distributed, not-a-knot condition).
 * ndim in [1, 4] axes; axis a has n_nodes[a] in [4, GRT_SPLINE_MAX_NODES]
 * nodes lo[a] + j (hi[a] - lo[a]) / (n_nodes[a] - 1), hi[a] > lo[a], and
 * n_targets[a] >= 1 target coordinates, given back to back in the HOST array
 * `targets` (axis 0 first; targets outside [lo, hi] use the end cubics).
 * d_values: DEVICE [batch][n_nodes[0]]...[n_nodes[ndim-1]] row-major FP64;
 * d_out: DEVICE [batch][n_targets[0]]...[n_targets[ndim-1]].  The weights and
 * the axis-by-axis contractions run on the GPU; work memory is held by the
 * context.  Enqueued on `stream` (NULL = legacy default stream); returns after
 * enqueueing.  GRT_EINVAL for bad sizes. */
#define GRT_SPLINE_MAX_NODES 256
int grt_spline_grid(grt_ctx *ctx, int ndim, const int32_t *n_nodes, const double *lo, const double *hi,
                    const int32_t *n_targets, const double *targets, int64_t batch, const double *d_values,
                    double *d_out, void *stream);

/* PDD geometry.  The box prod_a [lo[a], hi[a]] is cut into sub[a] equal
 * subdomains along axis a; each has cells[a] in [2, 65] finite-difference
 * cells per axis, so the global grid has N[a] = sub[a] cells[a] + 1 nodes.
 * The planes are the grid planes bounding a subdomain, outer faces included
 * (the outer faces carry probabilistic artificial Dirichlet data, the use the
 * text after Example 4 describes).  On every plane of axis a the nodal points
 * are the tensor grid of nodes[b] >= 4 uniform points over [lo[b], hi[b]]
 * (both ends included) along each other axis b, at the t_nodes >= 3 time
 * levels t_j = T j / t_nodes, j = 1..t_nodes (t = 0 is the initial data
 * itself).  Crank-Nicolson takes nsteps >= 1 steps of T / nsteps. */
typedef struct grt_pdd_grid {
    int32_t dim;        /* 1..3, the context's dimension */
    double lo[3], hi[3];
    int32_t sub[3];
    int32_t cells[3];
    int32_t nodes[3];   /* entry a unused by the planes of axis a */
    int32_t t_nodes;
    double T;
    int32_t nsteps;
} grt_pdd_grid;

/* Subdomain limit: prod_a (cells[a] - 1) interior unknowns per subdomain. */
#define GRT_PDD_MAX_LOCAL 65536

/* The probabilistic nodal points of a PDD grid (HOST only, no GPU work), in
 * the order grt_pdd_solve reads their values: planes axis-major (axis 0 planes
 * k = 0..sub[0], then axis 1, ...), then time level j = 1..t_nodes, then the
 * in-plane nodes row-major over the other axes in ascending order.  x [n][dim]
 * and t [n] are HOST arrays of `capacity` points (x and t NULL with capacity
 * 0 to query the count); *n_out receives the count.  GRT_EINVAL for a bad
 * grid or a capacity below the count. */
int grt_pdd_points(const grt_pdd_grid *g, int64_t capacity, double *x, double *t, int64_t *n_out);

/* The PDD solution at t = T on the global grid.  d_u_nodes: DEVICE values at
 * the points of grt_pdd_points (e.g. the u of grt_solve / grt_plan_execute);
 * d_u_out: DEVICE [N[0]]..[N[dim-1]] row-major.  Steps, all on the GPU:
 *   1. spline (as grt_spline_grid) of every plane in time and in its
 *      coordinates to the finite-difference nodes at t_n = n T / nsteps,
 *      n = 1..nsteps, with the initial data as the t = 0 level;
 *   2. one thread block per subdomain runs all nsteps steps of the linearly
 *      implicit Crank-Nicolson scheme (Sec. 3, "Local solver")
 *        (I - dt/2 D Lap_h) u^{n+1} = (I + dt/2 D Lap_h) u^n + dt f(u*, x, t_{n+1/2}),
 *        u* = (3 u^n - u^{n-1}) / 2  (u^0 on the first step),
 *      Dirichlet data from step 1 (the initial data at t_0), f the context's
 *      f with its variable coefficients; each step's linear system is solved
 *      exactly by fast diagonalisation (sine transforms along each axis);
 *   3. plane nodes of d_u_out take the spline at T (an edge node takes the
 *      plane of its lowest axis), subdomain interiors the solves.
 * Work memory is held by the context: calls on one context must not overlap
 * in time.  Enqueued on `stream` (NULL = legacy default stream); returns after
 * enqueueing.  GRT_EINVAL for a bad grid, a dimension other than the
 * context's, or a subdomain above GRT_PDD_MAX_LOCAL unknowns. */
int grt_pdd_solve(grt_ctx *ctx, const grt_pdd_grid *g, const double *d_u_nodes, double *d_u_out, void *stream);

/* The same for the subdomains [sub_begin, sub_end) of the row-major subdomain
 * numbering (axis 0 slowest) only: the spline stages run in full, every plane
 * node of d_u_out is written, and only these subdomains' interior nodes; the
 * other interiors are left as they are.  The subdomains are independent (Sec.
 * 3: the decoupled sub-problems), so disjoint ranges on different GPUs -- each
 * with all nodal values -- together give grt_pdd_solve's result bit for bit.
 * GRT_EINVAL unless 0 <= sub_begin <= sub_end <= prod_a sub[a]. */
int grt_pdd_solve_range(grt_ctx *ctx, const grt_pdd_grid *g, int64_t sub_begin, int64_t sub_end,
                        const double *d_u_nodes, double *d_u_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GRT_H */

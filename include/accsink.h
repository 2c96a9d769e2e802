/*
 * accsink.h -- C-ABI of the GB300 (sm_103a) Acc-Sinkhorn solver.
 *
 * Solves the entropy-regularised optimal transport problem of the paper
 * "Accelerating Sinkhorn for Entropy-Regularized Optimal Transport"
 * (Xu & Chen), Sec. 1 eq. (EOT):
 *
 *     min_{P in Pi(a,b)}  <C, P> + eps * sum_ij P_ij (log P_ij - 1),
 *
 * through its dual potentials (f, g) in cost units, P_ij = exp((f_i + g_j -
 * C_ij) / eps) (Sec. 2, eq. P-from-dual with the cost divided by eps). Two
 * methods share one data path:
 *   ACCSINK_PLAIN  log-domain Sinkhorn, x_{k+1} = S(x_k) (Sec. 3, eq.
 *                  normalized-sinkhorn), x = g / eps;
 *   ACCSINK_ACC    Acc-Sinkhorn: Algorithm 1 inside the homotopy of
 *                  Algorithm 2 (Sec. 4).
 * One S evaluation is a row log-sum-exp pass and a column log-sum-exp pass
 * over the cost (Sec. 2, u- and v-updates); everything else is O(n + m).
 *
 * Conventions for every entry point
 *   - All functions return an accsink_status; no C++ exception crosses the
 *     ABI. On failure accsink_last_error(ctx) describes the first problem.
 *   - "device" pointers are CUDA device (or managed) memory on the context's
 *     device; "host" pointers are ordinary host memory. Pointers are borrowed:
 *     the library never frees caller memory and keeps no pointer after the
 *     call returns (except inside the cached CUDA graph, which is rebuilt
 *     whenever a call passes different pointers or sizes).
 *   - Work is enqueued on the caller's `stream` (cudaStream_t passed as
 *     void*; NULL = legacy default stream). Solve calls synchronise that
 *     stream before they return, because they return results on the host.
 *   - A context is not thread-safe; use one per host thread.
 *   - Matrices are row-major FP32 with a row stride `ldc` (elements, >= m).
 *     The vectorised kernels need ldc % 4 == 0 and a 16-byte aligned C;
 *     other layouts take a scalar path with identical results.
 */
#ifndef ACCSINK_H
#define ACCSINK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. ACCSINK_ERR_MAXITER is a soft outcome: the potentials are
 * valid, the marginal error is just still above tol. */
typedef enum {
    ACCSINK_OK = 0,
    ACCSINK_ERR_INVALID_ARG = 1,          /* bad size, pointer, eps, tol, ... */
    ACCSINK_ERR_NONPOSITIVE_MARGINAL = 2, /* some a_i or b_j <= 0 (log a, log b are needed) */
    ACCSINK_ERR_NONFINITE = 3,            /* NaN/Inf in C, a, b, or in the iterates */
    ACCSINK_ERR_OOM = 4,                  /* device allocation failed */
    ACCSINK_ERR_BUDGET = 5,               /* workspace would exceed the context's budget */
    ACCSINK_ERR_TIMEOUT = 6,              /* a bounded device wait gave up */
    ACCSINK_ERR_MAXITER = 7,              /* not converged within max_sinkhorn_steps */
    ACCSINK_ERR_CUDA = 8,                 /* a CUDA runtime call failed */
    ACCSINK_ERR_UNSUPPORTED = 9           /* valid request this build does not serve */
} accsink_status;

enum { ACCSINK_COST_DENSE = 0, ACCSINK_COST_SQEUCLID = 1, ACCSINK_COST_COSINE = 2 };
enum { ACCSINK_SCALE_NONE = 0, ACCSINK_SCALE_MAX_TO_ONE = 1 };
enum { ACCSINK_PLAIN = 0, ACCSINK_ACC = 1 };
enum { ACCSINK_STAB_OFF = 0, ACCSINK_STAB_REPORT = 1, ACCSINK_STAB_GATE = 2,
       ACCSINK_STAB_BACKTRACK = 3 };
enum { ACCSINK_CARRY_Y = 0, ACCSINK_CARRY_W = 1 };
enum { ACCSINK_PRECISION_AUTO = 0, ACCSINK_PRECISION_FP32 = 1, ACCSINK_PRECISION_DF32 = 2 };

typedef struct accsink_ctx accsink_ctx;

/* The problem (Sec. 1, eq. EOT). a and b must be positive; they are
 * renormalised to unit mass in FP64 (Sec. 2 assumes 1'a = 1'b = 1).
 * cost_scale = MAX_TO_ONE divides C by its largest entry first (Sec. 5,
 * colour transfer); the returned potentials are then in units of the scaled
 * cost. For ACCSINK_COST_DENSE only C is read; X and Y are for the point-
 * cloud costs C_ij = ||x_i - y_j||^2 and C_ij = 1 - <x_i, y_j> (Sec. 5). */
typedef struct {
    int32_t n;           /* rows (support of a), >= 1                        */
    int32_t m;           /* columns (support of b), >= 1                     */
    int32_t d;           /* point dimension (point-cloud costs only)         */
    int32_t cost_kind;   /* ACCSINK_COST_*                                   */
    int64_t ldc;         /* row stride of C in elements; 0 means m           */
    const float *C;      /* n x m cost, row-major, FP32                      */
    const float *X;      /* n x d points, row-major, FP32                    */
    const float *Y;      /* m x d points, row-major, FP32                    */
    const double *a;     /* n row marginal, FP64                             */
    const double *b;     /* m column marginal, FP64                          */
    int32_t cost_scale;  /* ACCSINK_SCALE_*                                  */
    int32_t reserved;
} accsink_problem;

/* Solver parameters. accsink_params_default() fills:
 *   method ACC, eps 1e-2, tol 1e-6, mu0 0.25, m0 4, max_sinkhorn_steps
 *   100000, stability REPORT, carry Y, evaluate 1, use_graph 1, history 0,
 *   col_transpose 1.
 * mu0 in (0, 1), m0 >= 1 (Algorithm 2). tol is the l1 marginal tolerance of
 * Sec. 5 eq. (l1tol), ||P1 - a||_1 + ||P'1 - b||_1 < tol. The solve tests it
 * after every S evaluation on the FP64 sum of the column errors that its
 * FP32 passes give (the row error is zero up to rounding after a row pass)
 * and stops once that sum is below tol - 2^-22 (2^-22 = 2.4e-7): the guard
 * covers the FP32 floor of the row marginal and the column sums' own error,
 * so the FP64 truth of the whole sum at the returned potentials is below
 * tol. A tol at or below 2^-22 cannot be met; such a solve runs to
 * max_sinkhorn_steps (ACCSINK_ERR_MAXITER). res.marginal_l1 is the estimate
 * the test used. carry selects how a homotopy stage hands w to the next
 * one: CARRY_Y keeps y = w / alpha (the state Theorem 1 follows), CARRY_W
 * hands w over unchanged as Algorithm 2 is printed. stability: OFF skips the
 * Theorem 4 test, REPORT counts failures, GATE also restarts the momentum
 * (w <- alpha x) after a failed step, BACKTRACK instead ends the homotopy
 * stage at once (mu <- mu / 2, so the next step uses a smaller alpha).
 * precision: the arithmetic of the exponent arguments. DF32 forms every
 * argument in FP32 double-float (exact splits; the results sit ~1e-7 from
 * the FP64 truth, which tol = 1e-6 at eps = 1e-3 needs). FP32 drops the low
 * parts where that is cheaper: point-cloud solves with d <= 4 then form x.y
 * in plain FP32 (about twice as fast per pass), with argument errors of
 * ~2^-22 of the terms' size |C| / eps, so only loose tolerances converge
 * (e.g. 1e-5 at eps = 0.1 for costs scaled to max 1). Stored costs are read
 * at the memory bound either way and always use DF32, as do point clouds
 * with d > 4 and batched solves. AUTO (the default) is DF32. */
typedef struct {
    int32_t method;
    int32_t m0;
    double eps;
    double tol;
    double mu0;
    int32_t max_sinkhorn_steps;
    int32_t stability;
    int32_t carry;
    int32_t evaluate;    /* 1: one extra pass computes <C, P> at the end     */
    int32_t use_graph;   /* 1: device-side loop in a CUDA graph; 0: host loop */
    int32_t history;     /* keep per-step history for this many steps (0: no) */
    int32_t col_transpose; /* 1: the context keeps a transposed copy of C
                              (another 4 n m bytes, made once per solve) so
                              the column pass streams rows too, when the
                              budget and the device allow; 0: never */
    int32_t precision;   /* ACCSINK_PRECISION_*                              */
} accsink_params;

/* Result of a solve (host struct, filled by the library). */
typedef struct {
    int32_t status;              /* accsink_status of the solve              */
    int32_t sinkhorn_steps;      /* S evaluations = row+column pass pairs    */
    int32_t outer_stages;        /* completed homotopy stages (Algorithm 2)  */
    int32_t stability_failures;  /* steps where Theorem 4's test failed      */
    double marginal_l1;          /* sum_j |c_j - b_j| at the returned iterate
                                    (row error is zero by construction)      */
    double transport_cost;       /* <C, P> (NaN unless params.evaluate)      */
    double dual_objective;       /* <f,a> + <g,b> - eps (after the row pass) */
    double cost_max;             /* max_ij C_ij of the input                 */
    double gpu_ms;               /* device time of the solve (CUDA events)   */
    int32_t loop_mode;           /* 1: CUDA-graph device loop ran; 0: host loop
                                    (requested, or the graph could not be built);
                                    2: batched persistent launch */
    int32_t reserved;
} accsink_result;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device`. mem_budget_bytes caps the
 * workspace the context may allocate (0 = no cap). */
int accsink_create(accsink_ctx **out, int device, size_t mem_budget_bytes);
void accsink_destroy(accsink_ctx *ctx);
/* Message for the last failed call on this context ("" if none). The string
 * is owned by the context and valid until its next call. */
const char *accsink_last_error(const accsink_ctx *ctx);
void accsink_params_default(accsink_params *p);
/* Library version string, e.g. "accsink 1.0 sm_103a". */
const char *accsink_version(void);

/* ---- whole solves ------------------------------------------------------- */

/* Solves the problem. All problem pointers are device pointers. f_out (n)
 * and g_out (m) are caller-allocated device arrays that receive the
 * potentials in cost units at the returned iterate; f is the row pass at
 * that g, so the row marginal is exact up to rounding. res (host) receives
 * the summary. Returns res->status (ACCSINK_ERR_MAXITER if not converged).
 * Every cost kind is served: DENSE reads C; SQEUCLID and COSINE form each
 * C_ij from X and Y inside the passes (1 <= d <= 64), never storing an
 * n x m matrix, with the device workspace O((n + m) d). Non-finite points
 * give ACCSINK_ERR_NONFINITE. */
int accsink_solve(accsink_ctx *ctx, const accsink_problem *prob,
                  const accsink_params *params, void *stream,
                  double *f_out, double *g_out, accsink_result *res);

/* Same solve (any cost kind) with every problem pointer and f_out/g_out in
 * HOST memory:
 * the library copies the inputs to its workspace, solves, and copies the
 * potentials back, ordered on `stream`. A dense C with rows of a multiple of
 * 4 floats is copied in row chunks on a stream of the context, each chunk
 * transposed as soon as it has landed (the results are those of
 * accsink_solve bit for bit). Host buffers may be pageable or pinned (pinned
 * copies are faster and overlap with the device work). The call returns when
 * the potentials are in f_out/g_out. */
int accsink_solve_host(accsink_ctx *ctx, const accsink_problem *prob_host,
                       const accsink_params *params, void *stream,
                       double *f_out_host, double *g_out_host,
                       accsink_result *res);

/* ---- warm starts and resumed solves ------------------------------------- */

/* State of Algorithm 1-2 (Sec. 4) at the end of a solve: the point the
 * iteration would continue from. x is the iterate (g = eps x in cost units),
 * w the momentum of Algorithm 1 after that step's update (gate and stage
 * hand-over applied), and the homotopy position of Algorithm 2. x and w are
 * caller-owned DEVICE arrays of m doubles. The shift fields are the solver's
 * operand offsets and the cost statistics they were derived for; a resume at
 * the same eps on a cost with the same statistics reuses them, which makes
 * the resumed steps identical to the bit to an uninterrupted run. */
typedef struct accsink_state {
    int32_t m;            /* length of x and w */
    int32_t method;       /* ACCSINK_ACC or ACCSINK_PLAIN */
    int32_t m_stage;      /* Algorithm 2: inner steps of the current stage */
    int32_t j_in_stage;   /* inner steps taken in the current stage */
    int32_t stages;       /* stages completed (mu = mu0 / 2^stages) */
    int32_t carry;        /* carry mode of the solve (ACCSINK_CARRY_*) */
    double eps;           /* regulariser the vectors refer to */
    double mu0, mu;       /* homotopy: initial and current mu */
    double shift_g, shift_f, cost_abs, cost_min, eps_c;   /* internal, see above */
    double *x;            /* device, m doubles */
    double *w;            /* device, m doubles */
} accsink_state;

/* Copies the state of the most recent accsink_solve / accsink_solve_from /
 * accsink_warm_start on this context into *state (x and w on `stream`; the
 * call returns after the copies complete). state->m, state->x and state->w
 * must be set by the caller; m must equal that solve's m. Any other call on
 * the context that runs kernels (single passes, another solve) replaces the
 * state: then, or before any solve, ACCSINK_ERR_INVALID_ARG. */
int accsink_export_state(accsink_ctx *ctx, accsink_state *state, void *stream);

/* Continues the iteration from `state` (Algorithm 1-2 resumed at its
 * homotopy position; plain Sinkhorn from x). The first S evaluation is at
 * state->x again, so a resume repeats one evaluation of the run that made
 * the state and then takes exactly its next steps. params->eps may differ
 * from state->eps: x and w keep their potentials, i.e. are scaled by
 * state->eps / params->eps (eps continuation). params->mu0 and m0 are not
 * used (the state's are); params->method must equal state->method. res and
 * the return value are as for accsink_solve, with res->sinkhorn_steps the
 * evaluations of this call and res->outer_stages the stage count including
 * the state's. */
int accsink_solve_from(accsink_ctx *ctx, const accsink_problem *prob,
                       const accsink_params *params, const accsink_state *state,
                       void *stream, double *f_out, double *g_out, accsink_result *res);

/* Solves from the potential g0 (device, m doubles, cost units) instead of
 * zero: x0 = g0 / eps and, for Algorithm 1, w0 = alpha0 x0 with
 * alpha0 = sqrt(2 mu0) (y0 = x0, the momentum a fixed point has). A g0 that
 * already meets tol stops after one S evaluation. */
int accsink_warm_start(accsink_ctx *ctx, const accsink_problem *prob,
                       const accsink_params *params, const double *g0, void *stream,
                       double *f_out, double *g_out, accsink_result *res);

/* Per-step history of the last solve on this context, if params.history > 0:
 * for evaluation e (0 = x_0) err[e] = marginal L1, dual[e] = dual objective,
 * mu[e] = mu used to form that iterate (0 for x_0 and for PLAIN), stab[e] =
 * bit0 Cond 1 failed, bit1 Cond 2 failed (Theorem 4), for the step that
 * produced e. cond (4 per step, may be NULL) = Cond1 lhs, Cond1 rhs, Cond2
 * lhs, Cond2 rhs. count = min(steps, capacity). Host arrays, caller-owned. */
int accsink_get_history(accsink_ctx *ctx, int32_t capacity, double *err,
                        double *dual, double *mu, int32_t *stab, double *cond,
                        int32_t *count);

/* ---- batches: many independent problems in one persistent launch -------- */

/* Work split of a batch (zero fields take the defaults):
 *   small_max_nm   problems with n*m at most this are solved whole by one
 *                  CTA (default 65536);
 *   row_tile_elems cost entries per row-pass work item of larger problems
 *                  (default 65536; column items are 128 columns);
 *   ctas_per_sm    persistent CTAs per SM (0: as many as fit);
 *   dense_solo_min_nm
 *                  dense problems (ACCSINK_COST_DENSE) with n*m at least this,
 *                  and a batch's only problem when it is dense, are solved one
 *                  at a time after the batched launch, exactly as
 *                  accsink_solve solves them with use_graph = 1 (res[k].loop_mode
 *                  is then 1): that path reads the stored FP32 cost (4 bytes
 *                  per entry per pass) where the batched launch reads its
 *                  double-float K (8 bytes). Default 2^24; negative: never. */
typedef struct {
    int32_t small_max_nm;
    int32_t row_tile_elems;
    int32_t ctas_per_sm;
    int32_t dense_solo_min_nm;
} accsink_batch_config;

/* Solves `count` independent problems (Sec. 1, eq. EOT, each with its own
 * a, b, cost, eps and parameters) in one persistent launch, each exactly as
 * accsink_solve would (same stopping rule, Algorithm 1 + 2, stability modes;
 * params.history and use_graph are ignored). probs, params and res are host
 * arrays of `count` records; the pointers inside probs are device pointers;
 * f_out and g_out are host arrays of `count` device pointers (n_k and m_k
 * doubles). Each problem's cost is formed once in the context's batch
 * workspace (8 bytes per entry, a double-float pair), so point clouds of any
 * dimension 1 <= d <= 4096 are accepted. Cosine costs with 32 <= d <= 480 are
 * formed on the tensor cores from exact integer slices of the vectors (dot
 * products within d 2^-39 |x||y|; the environment variable
 * ACCSINK_BATCH_FORM=cuda selects the CUDA-core expansion, exact to FP64
 * rounding, for every problem); the slices take 12 bytes per vector element
 * of workspace. Large problems (tiled, m >= 4096) run the step's per-column
 * loops as work items over many CTAs (ACCSINK_BATCH_STEP_ITEMS=0 keeps them
 * in one CTA; the potentials are the same bit for bit). The launch sequence
 * (record upload, cost formation, the persistent solve, result download) is
 * captured into a CUDA graph and replayed on `stream` as one launch
 * (ACCSINK_BATCH_GRAPH=0 issues it directly). Large dense problems
 * are solved one at a time by the single-solve path (see dense_solo_min_nm
 * above; history is not kept for them). Returns OK when every problem
 * converged, ACCSINK_ERR_MAXITER when some did not (their results are still
 * valid), another code for the first failed problem (see res[k].status), or
 * ACCSINK_ERR_TIMEOUT if a device-side wait of the scheduler ran out. */
int accsink_solve_batch(accsink_ctx *ctx, int32_t count, const accsink_problem *probs,
                        const accsink_params *params, void *stream,
                        double *const *f_out, double *const *g_out,
                        accsink_result *res);

/* The context's batch work split (NULL resets to the defaults). */
int accsink_batch_set_config(accsink_ctx *ctx, const accsink_batch_config *cfg);
int accsink_batch_get_config(const accsink_ctx *ctx, accsink_batch_config *cfg);

/* Autotuner: solves the batch once with each candidate work split, keeps the
 * fastest in the context and writes it to *best. times_ms (host, capacity
 * cap, may be NULL) receives each candidate's time of the batched launch and
 * *tried their number; the dense problems solved one at a time are solved
 * once, with the first candidate. Arguments otherwise as accsink_solve_batch
 * (the outputs hold the last candidate's solve). */
int accsink_batch_autotune(accsink_ctx *ctx, int32_t count, const accsink_problem *probs,
                           const accsink_params *params, void *stream,
                           double *const *f_out, double *const *g_out,
                           accsink_result *res, accsink_batch_config *best,
                           float *times_ms, int32_t cap, int32_t *tried);

/* Device times of the last batch on this context: total, cost formation and
 * persistent solve, in milliseconds (host pointers, any may be NULL); total
 * and solve include the dense problems solved one at a time. */
int accsink_batch_last_timing(const accsink_ctx *ctx, float *total_ms, float *form_ms,
                              float *solve_ms);

/* ---- request server: admitted by device memory, potentials kept resident */

/* A server owns a worker thread, a CUDA stream and a memory pool on one
 * device. Its calls are thread-safe (any client thread). Submitted solves
 * are admitted in FIFO order while their inputs, outputs and batch workspace
 * fit in mem_budget_bytes next to the potentials still held by clients and
 * the group stays within its entry limit (accsink_server_set_limits);
 * each admitted group runs as one accsink_solve_batch-style persistent
 * launch. A request moves QUEUED -> RUNNING -> DONE (or FAILED); its
 * potentials stay on the device until accsink_server_release. */
typedef struct accsink_server accsink_server;
typedef uint64_t accsink_ticket;
enum { ACCSINK_REQ_QUEUED = 0, ACCSINK_REQ_RUNNING = 1, ACCSINK_REQ_DONE = 2,
       ACCSINK_REQ_FAILED = 3 };

typedef struct {
    int64_t queued, solved, failed, batches;
    int64_t resident_bytes;      /* potentials held for DONE tickets          */
    int64_t peak_bytes;          /* largest admitted footprint                */
    int64_t budget_bytes;
    double busy_ms;              /* device time of all batches                */
} accsink_server_stats;

int accsink_server_create(int device, size_t mem_budget_bytes, accsink_server **out);
/* Drops queued requests, waits for the running group, frees everything. */
void accsink_server_destroy(accsink_server *srv);
const char *accsink_server_last_error(accsink_server *srv);
/* Queues one solve. prob_host's pointers (C or X, Y, and a, b) are HOST
 * pointers that must stay valid until the ticket is DONE or FAILED; they are
 * copied to the device when the request is admitted. Validation failures
 * return ACCSINK_ERR_INVALID_ARG without a ticket. */
int accsink_server_submit(accsink_server *srv, const accsink_problem *prob_host,
                          const accsink_params *params, accsink_ticket *ticket);
int accsink_server_poll(accsink_server *srv, accsink_ticket ticket, int32_t *state);
/* Waits for the ticket (timeout_ms < 0: no limit; ACCSINK_ERR_TIMEOUT when it
 * runs out). Writes the result and the submit-to-done latency (host clock,
 * ms; may be NULL) and returns the solve's status. */
int accsink_server_wait(accsink_server *srv, accsink_ticket ticket, int32_t timeout_ms,
                        accsink_result *res, double *latency_ms);
/* Device pointers to a DONE ticket's potentials f (n) and g (m), valid until
 * the ticket is released. */
int accsink_server_potentials(accsink_server *srv, accsink_ticket ticket,
                              const double **f_dev, const double **g_dev);
int accsink_server_copy_potentials(accsink_server *srv, accsink_ticket ticket,
                                   double *f_host, double *g_host);
/* Frees a DONE or FAILED ticket and its potentials. */
int accsink_server_release(accsink_server *srv, accsink_ticket ticket);
int accsink_server_get_stats(accsink_server *srv, accsink_server_stats *out);
/* Work split of the server's batches (NULL: defaults). dense_solo_min_nm is
 * not used: every admitted request runs in its group's batched launch. */
int accsink_server_set_config(accsink_server *srv, const accsink_batch_config *cfg);
/* Admission limit of one group: the sum of n m over its requests stays at or
 * below max_group_entries, except that a larger request runs alone; 0 (the
 * default) means no limit beyond the memory budget. Requests that arrive
 * while a group runs wait for its slowest problem; a limit shortens that
 * wait at the price of throughput (large groups keep every SM busy).
 * ACCSINK_ERR_INVALID_ARG for a negative limit. */
int accsink_server_set_limits(accsink_server *srv, int64_t max_group_entries);

/* ---- single passes (the hot path's steps, for tests and roofline timing) */

/* Every single-pass call serves every cost kind and honours cost_scale: with
 * MAX_TO_ONE the cost is C / max C and potentials are in its units. For
 * point clouds each call first forms the O((n + m) d) point workspace. */

/* Row pass, Sec. 2 u-update in cost units (Sec. 8 step "row LSE"):
 *   f_i = eps log a_i - eps LSE_j((g_j - C_ij) / eps).
 * a is used as given (not renormalised). g (m), a (n) and f_out (n) are
 * device FP64 arrays. */
int accsink_row_pass(accsink_ctx *ctx, const accsink_problem *prob,
                     double eps, const double *g, double *f_out, void *stream);

/* Column log-sum-exp of the v-update (Sec. 2, eq. v-update):
 *   ell_j = LSE_i((f_i - C_ij) / eps),
 * so that the column sums of P(f, g) are c_j = exp(g_j / eps + ell_j).
 * f (n) and ell_out (m) are device FP64 arrays. */
int accsink_col_lse(accsink_ctx *ctx, const accsink_problem *prob,
                    double eps, const double *f, double *ell_out, void *stream);

/* One normalised Sinkhorn map (Sec. 3, eq. normalized-sinkhorn) at x = g/eps:
 * writes f_out = eps u(x) (n), c_out = column sums of P(u(x), x) (m),
 * s_out = eps S(x) (m, cost units, mean zero), and *err_out (host) =
 * sum_j |c_j - b_j| (Sec. 5 eq. l1tol). a and b are used as given. */
int accsink_sinkhorn_map(accsink_ctx *ctx, const accsink_problem *prob,
                         double eps, const double *g, double *f_out,
                         double *c_out, double *s_out, double *err_out,
                         void *stream);

/* Transport cost <C, P> (eq. EOT) of the plan P_ij = exp((f_i + g_j - C_ij)
 * / eps) for device potentials f (n), g (m); result in *cost_out (host),
 * accumulated in FP64. */
int accsink_transport_cost(accsink_ctx *ctx, const accsink_problem *prob,
                           double eps, const double *f, const double *g,
                           double *cost_out, void *stream);

/* ---- export of a solution (one-off, after a solve; FP64 per entry) ------- */

/* The transport plan P_ij = exp((f_i + g_j - C_ij) / eps) (eq. P-from-dual)
 * of device potentials f (n), g (m) in cost units (of the scaled cost under
 * MAX_TO_ONE), any cost kind, written to the caller's device array P_out
 * (n rows of ld_p >= m entries) as FP32 (dtype 0) or FP64 (dtype 1). Every
 * entry is formed in FP64 as the problem defines it. */
int accsink_plan(accsink_ctx *ctx, const accsink_problem *prob, double eps,
                 const double *f, const double *g, void *P_out, int64_t ld_p,
                 int32_t dtype, void *stream);

/* Barycentric projection of target features through the plan (Sec. 5,
 * colour transfer): out_i = sum_j P_ij Z_j / sum_j P_ij for device FP32
 * features Z (m x dz, row-major) into device FP64 out (n x dz). */
int accsink_barycentric(accsink_ctx *ctx, const accsink_problem *prob, double eps,
                        const double *f, const double *g, const float *Z, int32_t dz,
                        double *out, void *stream);

/* ---- measurement -------------------------------------------------------- */

/* Times the two streaming passes alone on `stream` with CUDA events: after
 * one untimed row pass and column pass at g (device, m, cost units), runs
 * `reps` row passes back to back, then `reps` column passes (over the
 * transposed copy when the context can hold it, as the solver does), and
 * writes the mean device milliseconds per launch to *row_ms and *col_ms
 * (host). Used for the HBM roofline of the passes; each launch reads the
 * 4 n m bytes of the cost once plus O(n + m) operands. For point clouds the
 * two on-the-fly passes are timed (a must be given; n m cost entries each,
 * bound by FP32 arithmetic rather than by memory). */
int accsink_time_passes(accsink_ctx *ctx, const accsink_problem *prob, double eps,
                        const double *g, int reps, void *stream, float *row_ms,
                        float *col_ms);

/* Failure-path self test. Runs the solver's bounded grid barrier (the one of
 * the step kernel) in a launch where one block never arrives, so the other
 * blocks' waits run out after limit_s (0 < limit_s <= 2) seconds: they
 * record ACCSINK_ERR_TIMEOUT in the solver state and return, and the context
 * stays usable. *status_out receives the recorded status, *elapsed_s the host
 * time the launch took. Uses (and leaves for the next solve to rewrite) the
 * context's workspace state; returns ACCSINK_OK when the launch itself ran. */
int accsink_selftest_timeout(accsink_ctx *ctx, double limit_s, int32_t *status_out,
                             double *elapsed_s);

/* Launch geometry the context would use for an n x m dense cost (vec = 1 for
 * the 128-bit path): out6 = {SM count, row-pass CTAs, column-pass row splits,
 * column-pass strips, step-kernel CTAs, cost-statistics CTAs}. */
int accsink_launch_geometry(accsink_ctx *ctx, int32_t n, int32_t m, int32_t vec,
                            int32_t *out6);

/* ---- allocation-free variant -------------------------------------------- */

/* Column log-sum-exp pass of accsink_col_lse for callers that cannot
 * allocate device memory (a server whose memory pool owns the whole GPU, a
 * plugin living under another framework's allocator, a loop that cannot
 * accept cudaMalloc's implicit synchronisation). The paper has no
 * counterpart to this entry point; it exists only for those callers.
 *
 * It needs no context and calls no allocating routine. Its scratch is one
 * 16 MiB array in device memory, held until the process exits. It must fit
 * 8 n + 8 m bytes plus a few KB; larger problems return ACCSINK_ERR_BUDGET
 * before any work is queued. Everything runs on the current device and on
 * `stream`; the call returns without synchronising.
 *
 * The first call on a device looks up the array's device address once. With
 * CUDA's default lazy module loading that first call is also what loads the
 * array's module on the device and so reserves the 16 MiB: it can fail with
 * ACCSINK_ERR_CUDA when the device has no memory left. A caller whose memory
 * pool will claim the device should therefore make one call (any valid
 * size) before the pool does, or run with CUDA_MODULE_LOADING=EAGER; and it
 * should make that first call outside any stream capture. All calls share
 * the one array and reuse it without clearing what they fully rewrite:
 * calls whose work overlaps on the GPU (different streams, or host threads)
 * race and must be serialised by the caller. If a device-side wait of the
 * pass runs out (a bounded grid barrier), every ell_out entry is NaN: a NaN
 * output means that the pass did not complete.
 *
 * Arguments as accsink_col_lse (dense cost, f (n) and ell_out (m) device
 * FP64, eps > 0). Returns ACCSINK_OK, ACCSINK_ERR_INVALID_ARG,
 * ACCSINK_ERR_UNSUPPORTED (non-dense cost), ACCSINK_ERR_BUDGET (too large)
 * or ACCSINK_ERR_CUDA. */
int accsink_col_lse_noalloc(const accsink_problem *prob, double eps, const double *f,
                            double *ell_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ACCSINK_H */

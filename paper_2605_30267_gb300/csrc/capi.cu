// Host engine behind the C-ABI of include/accsink.h: context, workspace,
// validation, the device-side solve loop (a CUDA graph whose body is
// [row pass -> column pass -> step] inside a conditional WHILE node, so a
// solve needs no host round trip per iteration), a host-driven fallback loop,
// and the single-pass entry points.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "accsink.h"
#include "accsink_internal.cuh"
#include "batch_host.h"
#include "batch_internal.cuh"

using namespace accsink;

namespace accsink {
__global__ void k_set_state(DevState v, DevState *dst) { *dst = v; }

struct StageTable {
    double v[kMaxStages * kStageSlots];
};
__global__ void k_set_table(StageTable t, double *dst)
{
    for (int i = threadIdx.x; i < kMaxStages * kStageSlots; i += blockDim.x) dst[i] = t.v[i];
}

// Algorithm 2's stages: mu_s = mu0 / 2^s, alpha_s = sqrt(2 mu_s), and the
// alpha-dependent constants of Algorithm 1 and Theorem 4, per stage.
void fill_stage_table(StageTable &tab, double mu0)
{
    for (int st_i = 0; st_i < kMaxStages; ++st_i) {
        const double mu_s = mu0 * std::ldexp(1.0, -st_i);
        const double a = std::sqrt(2.0 * mu_s);
        const double an = std::sqrt(2.0 * (mu_s / 2.0));
        double *r = tab.v + st_i * kStageSlots;
        r[0] = a;
        r[1] = 1.0 / a;
        r[2] = 1.0 / (1.0 + a);
        r[3] = a * a - 2.0;
        r[4] = (4.0 - a * a - 2.0 * std::sqrt(a)) / (2.0 * a * (1.0 + a) * (1.0 + a));
        r[5] = std::pow(a, 1.5);
        r[6] = an / a;
        r[7] = 1.0 / (1.0 + an);
    }
}
}  // namespace accsink

namespace {

struct GraphKey {
    const float *C = nullptr;
    int64_t ldc = 0;
    int n = 0, m = 0, vec = 0, row_grid = 0, splits = 0, step_grid = 0, colt_grid = 0;
    int row_nfull = 0, row_parts = 0, colt_nfull = 0, colt_parts = 0;
    int prec = 0;        // kernel-argument flags that vary per solve (FP32 points)
    void *ws = nullptr;
    const float *ct = nullptr;
    bool operator==(const GraphKey &o) const
    {
        return C == o.C && ldc == o.ldc && n == o.n && m == o.m && vec == o.vec &&
               row_grid == o.row_grid && splits == o.splits && step_grid == o.step_grid &&
               colt_grid == o.colt_grid && row_nfull == o.row_nfull &&
               row_parts == o.row_parts && colt_nfull == o.colt_nfull &&
               colt_parts == o.colt_parts && prec == o.prec && ws == o.ws && ct == o.ct;
    }
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

// Row chunks of the overlapped host upload (accsink_solve_host).
constexpr int kUploadChunks = 8;

struct accsink_ctx {
    int device = 0;
    size_t budget = 0;
    std::string err;
    int num_sms = 1;
    int occ_row[2] = {1, 1}, occ_col[2] = {1, 1}, occ_row_warp = 1;
    // workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int64_t n_cap = -1, m_cap = -1, units_cap = 0;
    // the last solve's continuation state is in the workspace (x, w1)
    bool state_ok = false;
    int state_m = 0;
    const int *state_perm = nullptr;   // curve order of the columns (sorted point solves)
    double state_mu0 = 0.0;
    int splits_cap = 0, rowgrid_cap = 0, hist_cap = 0;
    Work w{};
    DevState *h_state = nullptr;      // pinned
    double *h_rowpart = nullptr;      // pinned, rowgrid_cap * 2
    // staging for accsink_solve_host
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // graph cache
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    cudaStream_t cap_stream = nullptr;
    // overlapped upload of accsink_solve_host: copy stream and chunk events
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t up_ev[kUploadChunks + 1] = {};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int last_hist_count = 0;
    bool graph_broken = false;
    std::string graph_error;
    // transposed copy of the cost for the column pass
    float *ct = nullptr;
    size_t ct_bytes = 0;
    // point-cloud workspace
    void *pts = nullptr;
    size_t pts_bytes = 0;
    int occ_pts = 1;
    // batches
    BatchWorkspace batch;
    BatchTuning batch_tuning;
    BatchTiming batch_timing;
    int occ_batch = 1;
    cudaEvent_t ev_mid = nullptr;
};

namespace {

int fail(accsink_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(accsink_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, ACCSINK_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

void free_graph(accsink_ctx *ctx)
{
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->exec = nullptr;
    ctx->graph = nullptr;
    ctx->key = GraphKey();
}

// Launch geometry of a dense solve. The warp-per-row passes may split the
// rows of a last wave into column parts (rsplit for C, csplit for C^T);
// `units` is the number of part records the larger split needs.
struct Geometry {
    int stat_grid, row_grid, splits, step_grid, vec_grid, colt_grid;
    RowSplit rsplit, csplit;
    int64_t units;
};

// Warps of the warp-per-row kernel that are resident at once.
int64_t row_warps_resident(const accsink_ctx *ctx)
{
    return (int64_t)ctx->num_sms * ctx->occ_row_warp * 8;
}

Geometry geometry(const accsink_ctx *ctx, int n, int m, int vec)
{
    Geometry g;
    const int S = ctx->num_sms;
    // eight CTAs per SM for the statistics (with the transposed copy: one read
    // of C); the workspace's statpart holds one 32-byte partial per CTA of 8 S
    g.stat_grid = std::max(1, std::min(n, 8 * S));
    g.rsplit = RowSplit();
    if (vec && row_kernel_choice() == 1) {
        // TMA row pass: one CTA per SM
        g.row_grid = std::max(1, std::min(S, n));
    } else if (vec) {
        g.rsplit = plan_row_split(n, m, row_warps_resident(ctx));
        g.row_grid = g.rsplit.grid;
    } else {
        g.row_grid = std::max(1, std::min(S * ctx->occ_row[vec], (n + 1) / 2));
    }
    const int strips = (m + kColStrip - 1) / kColStrip;
    const int target = S * ctx->occ_col[vec];
    int splits = target / strips;
    splits = std::max(1, std::min(splits, std::max(1, n / 8)));
    g.splits = splits;
    // the step kernel's FP64 column work is spread over every SM
    g.step_grid = std::max(1, std::min(S, (m + 63) / 64));
    g.vec_grid = std::max(1, std::min(S, (std::max(n, m) + 63) / 64));
    g.csplit = plan_row_split(m, n, row_warps_resident(ctx));
    g.colt_grid = g.csplit.grid;
    g.units = std::max(row_split_records(g.rsplit, n), row_split_records(g.csplit, m));
    return g;
}

// Row stride (elements) of the transposed copy: n rounded up to 4 so every
// row starts on a 16-byte boundary.
int64_t ct_ld(int n) { return (n + 3) / 4 * 4; }

// Makes room for C^T (m x ct_ld(n) floats). Returns false, without error,
// when the budget or the device cannot hold it (the strip column pass is
// used then).
bool ensure_ct(accsink_ctx *ctx, int n, int m)
{
    const size_t need = (size_t)m * (size_t)ct_ld(n) * sizeof(float);
    if (ctx->ct && ctx->ct_bytes >= need) return true;
    if (ctx->budget && ctx->ws_bytes + ctx->stage_bytes + need > ctx->budget) return false;
    if (ctx->ct) cudaFree(ctx->ct);
    ctx->ct = nullptr;
    ctx->ct_bytes = 0;
    free_graph(ctx);
    if (cudaMalloc(&ctx->ct, need) != cudaSuccess) {
        cudaGetLastError();
        ctx->ct = nullptr;
        return false;
    }
    ctx->ct_bytes = need;
    return true;
}

// (Re)allocates the workspace for n x m with the given partial counts.
int ensure_workspace(accsink_ctx *ctx, int n, int m, int splits, int row_grid, int hist,
                     int64_t units = 0)
{
    // every call that runs kernels on the workspace passes here first
    ctx->state_ok = false;
    if (n <= ctx->n_cap && m <= ctx->m_cap && splits <= ctx->splits_cap &&
        row_grid <= ctx->rowgrid_cap && hist <= ctx->hist_cap && units <= ctx->units_cap &&
        ctx->ws)
        return ACCSINK_OK;
    const int64_t N = std::max<int64_t>(n, ctx->n_cap);
    const int64_t M = std::max<int64_t>(m, ctx->m_cap);
    const int SP = std::max(splits, ctx->splits_cap);
    const int RG = std::max(row_grid, ctx->rowgrid_cap);
    const int H = std::max(hist, ctx->hist_cap);
    const int64_t U = std::max<int64_t>(std::max<int64_t>(units, ctx->units_cap), 1);
    const int64_t Mp = (M + 3) / 4 * 4;
    const int S = ctx->num_sms;
    std::vector<size_t> sizes = {
        (size_t)N * 8, (size_t)M * 8, (size_t)N * 8, (size_t)M * 8,          // a b loga logb
        (size_t)M * 8, (size_t)M * 8, (size_t)M * 8, (size_t)M * 8, (size_t)M * 8,  // x xp w pp Dp
        (size_t)M * 8, (size_t)M * 8, (size_t)M * 8, (size_t)M * 8,          // raw D1 del w1
        (size_t)N * 8,                                                         // u
        (size_t)Mp * 4, (size_t)Mp * 4,                                        // G Gk
        (size_t)N * 8,                                                         // FF
        (size_t)((N + 3) / 4 * 4) * 4, (size_t)((N + 3) / 4 * 4) * 4,          // Fh Fk
        (size_t)M * 8,                                                         // ell
        (size_t)SP * (size_t)M * 8,                                            // colpart
        (size_t)RG * 16,                                                       // rowpart
        (size_t)std::max(S, 1) * kPartStride * 8,                              // steppart
        (size_t)8 * S * 32,                                                    // statpart
        (size_t)std::max(H, 1) * 8, (size_t)std::max(H, 1) * 8, (size_t)std::max(H, 1) * 8,
        (size_t)std::max(H, 1) * 32, (size_t)std::max(H, 1) * 4,               // history
        (size_t)kMaxStages * kStageSlots * 8,                                  // stage table
        sizeof(DevState),
        (size_t)U * 16, (size_t)U * 8, (size_t)std::max(N, M) * 4};           // prec pcrec pcnt
    size_t total = 0;
    for (size_t s : sizes) total += align_up(s, 256);
    if (ctx->budget && total > ctx->budget)
        return fail(ctx, ACCSINK_ERR_BUDGET,
                    "workspace of " + std::to_string(total) + " bytes exceeds the budget");
    free_graph(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->h_rowpart) cudaFreeHost(ctx->h_rowpart);
    ctx->ws = nullptr;
    ctx->h_rowpart = nullptr;
    if (cudaMalloc(&ctx->ws, total) != cudaSuccess) {
        cudaGetLastError();
        ctx->n_cap = ctx->m_cap = -1;
        return fail(ctx, ACCSINK_ERR_OOM, "cudaMalloc of the workspace failed");
    }
    if (cudaMallocHost(&ctx->h_rowpart, (size_t)RG * 16) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, ACCSINK_ERR_OOM, "cudaMallocHost failed");
    }
    cudaMemset(ctx->ws, 0, total);
    ctx->ws_bytes = total;
    char *p = (char *)ctx->ws;
    size_t k = 0;
    auto take = [&](void) -> void * {
        void *r = p;
        p += align_up(sizes[k++], 256);
        return r;
    };
    Work &w = ctx->w;
    w = Work{};
    w.a = (double *)take(); w.b = (double *)take(); w.loga = (double *)take(); w.logb = (double *)take();
    w.x = (double *)take(); w.x_prev = (double *)take(); w.w = (double *)take();
    w.p_prev = (double *)take(); w.D_prev = (double *)take();
    w.raw = (double *)take(); w.D1 = (double *)take(); w.del = (double *)take(); w.w1 = (double *)take();
    w.u = (double *)take();
    w.G = (float *)take(); w.Gk = (float *)take();
    w.FF = (float2 *)take();
    w.Fh = (float *)take(); w.Fk = (float *)take();
    w.ell = (double *)take();
    w.colpart = (float2 *)take();
    w.rowpart = (double *)take();
    w.steppart = (double *)take();
    w.statpart = (double *)take();
    w.h_err = (double *)take(); w.h_dual = (double *)take(); w.h_mu = (double *)take();
    w.h_cond = (double *)take(); w.h_stab = (int32_t *)take();
    w.stage_table = (const double *)take();
    w.st = (DevState *)take();
    w.prec = (float4 *)take();
    w.pcrec = (float2 *)take();
    w.pcnt = (uint32_t *)take();
    ctx->n_cap = N; ctx->m_cap = M; ctx->splits_cap = SP; ctx->rowgrid_cap = RG; ctx->hist_cap = H;
    ctx->units_cap = U;
    return ACCSINK_OK;
}

int validate_problem(accsink_ctx *ctx, const accsink_problem *p, bool need_cost_dense)
{
    if (!p) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "problem is NULL");
    if (p->n < 1 || p->m < 1) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "n and m must be >= 1");
    if (p->cost_kind != ACCSINK_COST_DENSE) {
        if (p->cost_kind != ACCSINK_COST_SQEUCLID && p->cost_kind != ACCSINK_COST_COSINE)
            return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown cost_kind");
        if (need_cost_dense)
            return fail(ctx, ACCSINK_ERR_UNSUPPORTED,
                        "this entry point serves dense costs only");
        if (!p->X || !p->Y) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "X and Y must be given");
        if (p->d < 1 || p->d > 64)
            return fail(ctx, ACCSINK_ERR_INVALID_ARG, "point dimension d must be in 1..64");
        if (p->cost_scale != ACCSINK_SCALE_NONE && p->cost_scale != ACCSINK_SCALE_MAX_TO_ONE)
            return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown cost_scale");
        return ACCSINK_OK;
    }
    if (!p->C) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "C is NULL");
    const int64_t ldc = p->ldc ? p->ldc : p->m;
    if (ldc < p->m) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "ldc < m");
    if (p->cost_scale != ACCSINK_SCALE_NONE && p->cost_scale != ACCSINK_SCALE_MAX_TO_ONE)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown cost_scale");
    return ACCSINK_OK;
}

CostView make_view(const accsink_problem *p)
{
    CostView cv;
    cv.C = p->C;
    cv.ldc = p->ldc ? p->ldc : p->m;
    cv.n = p->n;
    cv.m = p->m;
    cv.vec = ((cv.ldc % 4) == 0 && (((uintptr_t)p->C) & 15u) == 0) ? 1 : 0;
    return cv;
}

int validate_params(accsink_ctx *ctx, const accsink_params *q)
{
    if (!q) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "params is NULL");
    if (!(q->eps > 0.0) || !std::isfinite(q->eps))
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "eps must be positive and finite");
    if (!(q->tol > 0.0)) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "tol must be positive");
    if (q->method != ACCSINK_PLAIN && q->method != ACCSINK_ACC)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown method");
    if (q->method == ACCSINK_ACC && !(q->mu0 > 0.0 && q->mu0 < 1.0))
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "mu0 must lie in (0, 1)");
    if (q->method == ACCSINK_ACC && q->m0 < 1)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "m0 must be >= 1");
    if (q->max_sinkhorn_steps < 1)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "max_sinkhorn_steps must be >= 1");
    if (q->stability < 0 || q->stability > 3)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown stability mode");
    if (q->carry != ACCSINK_CARRY_Y && q->carry != ACCSINK_CARRY_W)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown carry mode");
    if (q->history < 0) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "history must be >= 0");
    if (q->precision < ACCSINK_PRECISION_AUTO || q->precision > ACCSINK_PRECISION_DF32)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown precision");
    return ACCSINK_OK;
}

cudaError_t set_state(accsink_ctx *ctx, const DevState &hs, cudaStream_t s)
{
    k_set_state<<<1, 1, 0, s>>>(hs, ctx->w.st);
    return cudaGetLastError();
}

// Builds (or reuses) the graph: WHILE(cond) { row pass; column pass; step }.
// One S evaluation: row pass, then the column pass (on C^T when `ct`).
cudaError_t launch_passes(const CostView &cv, const Work &w, const Geometry &g, const float *ct,
                          cudaStream_t s)
{
    cudaError_t e = launch_row_pass(cv, w, g.row_grid, g.rsplit, false, s);
    if (e != cudaSuccess) return e;
    if (ct)
        return launch_col_pass_transposed(ct, ct_ld(cv.n), cv.n, cv.m, w, g.colt_grid,
                                          g.csplit, s);
    return launch_col_pass(cv, w, g.splits, s);
}

template <class Body>
int build_loop_graph(accsink_ctx *ctx, const GraphKey &key, Body body);

int get_graph(accsink_ctx *ctx, const CostView &cv, const Geometry &g, const float *ct)
{
    GraphKey key;
    key.C = cv.C; key.ldc = cv.ldc; key.n = cv.n; key.m = cv.m; key.vec = cv.vec;
    key.row_grid = g.row_grid; key.splits = g.splits; key.step_grid = g.step_grid;
    key.colt_grid = g.colt_grid; key.ct = ct;
    key.row_nfull = g.rsplit.nfull; key.row_parts = g.rsplit.parts;
    key.colt_nfull = g.csplit.nfull; key.colt_parts = g.csplit.parts;
    key.ws = ctx->ws;
    Work w = ctx->w;
    w.ignore_done = 0;
    return build_loop_graph(ctx, key, [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        cudaError_t e = launch_passes(cv, w, g, ct, cs);
        if (e != cudaSuccess) return e;
        return launch_step(cv, w, g.step_grid, h, cs);
    });
}

// WHILE(cond) { body x kEvalsPerTrip } with each body captured from
// `body(stream, handle)`: four S evaluations per trip through the conditional
// node, whose per-trip overhead (~4.4 us on this part, measured) is then paid
// every fourth evaluation. When a body's step stops the solve, the later
// bodies' kernels see `done` and return at once. Reuses the cached executable
// when `key` matches.
constexpr int kEvalsPerTrip = 4;
template <class Body>
int build_loop_graph(accsink_ctx *ctx, const GraphKey &key, Body body)
{
    if (ctx->exec && ctx->key == key) return ACCSINK_OK;
    free_graph(ctx);
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ctx, e, "cudaGraphConditionalHandleCreate"); }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ctx, e, "cudaGraphAddNode"); }
    cudaGraph_t body_graph = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(ctx->cap_stream, body_graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ctx, e, "cudaStreamBeginCaptureToGraph"); }
    cudaError_t e1 = cudaSuccess;
    for (int k = 0; k < kEvalsPerTrip && e1 == cudaSuccess; ++k) e1 = body(ctx->cap_stream, handle);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(ctx->cap_stream, &out);
    if (e1 != cudaSuccess || e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(ctx, e1 != cudaSuccess ? e1 : e, "capturing the solve loop");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ctx, e, "cudaGraphInstantiate"); }
    ctx->graph = graph;
    ctx->exec = exec;
    ctx->key = key;
    return ACCSINK_OK;
}

// Where a solve starts: the k_init start and, for a resumed solve, the
// homotopy position of Algorithm 2 (else mu0 and m0 of the params).
struct SolveStart {
    InitState is;
    bool stage = false;
    double mu = 0.0, mu0 = 0.0;
    int m_stage = 0, j = 0, stages = 0;
};

// Homotopy fields of the host state and the stage table of a solve.
void start_state(DevState &hs, StageTable &tab, const accsink_params *prm,
                 const SolveStart *start)
{
    const bool st = start && start->stage;
    hs.mu = st ? start->mu : prm->mu0;
    hs.m_stage = st ? start->m_stage : prm->m0;
    hs.j_in_stage = st ? start->j : 0;
    hs.stages = st ? start->stages : 0;
    fill_stage_table(tab, st ? start->mu0 : prm->mu0);
}

// Marks the workspace as holding a continuation state after a solve that
// ended converged or at the step limit.
void keep_state(accsink_ctx *ctx, const DevState &fs, int m, const accsink_params *prm,
                const SolveStart *start)
{
    ctx->state_perm = nullptr;
    ctx->state_ok = fs.status == ACCSINK_OK || fs.status == ACCSINK_ERR_MAXITER;
    ctx->state_m = m;
    ctx->state_mu0 = (start && start->stage) ? start->mu0 : prm->mu0;
}

// Core solve with device pointers, run on stream s. Fills res.
// prepared_nstat > 0: C^T and the cost statistics (that many partials) were
// already written on s (accsink_solve_host's overlapped upload).
int solve_device(accsink_ctx *ctx, const accsink_problem *prob, const accsink_params *prm,
                 cudaStream_t s, double *f_out, double *g_out, accsink_result *res,
                 const SolveStart *start = nullptr, int prepared_nstat = 0)
{
    const CostView cv = make_view(prob);
    const int n = prob->n, m = prob->m;
    const Geometry g = geometry(ctx, n, m, cv.vec);
    int rc = ensure_workspace(ctx, n, m, g.splits, g.row_grid, prm->history, g.units);
    if (rc != ACCSINK_OK) return rc;
    Work w = ctx->w;
    w.nstat = g.stat_grid;
    w.b_src = nullptr;
    w.f_given = nullptr;
    w.ignore_done = 0;

    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.eps_user = prm->eps;
    hs.tol = stop_threshold(prm->tol);
    hs.method = prm->method;
    hs.stability = prm->stability;
    hs.carry = prm->carry;
    hs.max_steps = prm->max_sinkhorn_steps;
    hs.hist_cap = prm->history;
    hs.row_grid = g.row_grid;
    hs.col_splits = g.splits;
    hs.use_cond = prm->use_graph ? 1 : 0;
    hs.first = 1;
    // column pass on a transposed copy when it fits (see ensure_ct)
    const float *ct = nullptr;
    if (prm->col_transpose && ensure_ct(ctx, n, m)) ct = ctx->ct;
    hs.col_mode = ct ? 1 : 0;

    StageTable tab;
    start_state(hs, tab, prm, start);

    CK(cudaEventRecord(ctx->ev0, s));
    CK(set_state(ctx, hs, s));
    k_set_table<<<1, 128, 0, s>>>(tab, const_cast<double *>(w.stage_table));
    CK(cudaGetLastError());
    // the cost statistics the init kernel needs, and C^T, in one read of C
    // when C is 16-byte aligned
    const bool fused = ct && cv.vec;
    if (prepared_nstat > 0 && fused) w.nstat = prepared_nstat;   // written by the caller
    else if (fused) CK(launch_transpose_stats(cv, ctx->ct, ct_ld(n), w, g.stat_grid, s));
    else CK(launch_cost_stats(cv, w, g.stat_grid, s));
    CK(launch_init(cv, w, g.vec_grid, prob->a, prob->b, prob->cost_scale == ACCSINK_SCALE_MAX_TO_ONE,
                   start ? start->is : InitState(), s));
    if (ct && !fused) CK(launch_transpose(cv, ctx->ct, ct_ld(n), s));
    CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->h_state->done) {
        const int st = ctx->h_state->status;
        std::memset(res, 0, sizeof(*res));
        res->status = st;
        res->cost_max = ctx->h_state->cmax;
        if (st == ACCSINK_ERR_NONFINITE) return fail(ctx, st, "C, a or b holds NaN or Inf");
        if (st == ACCSINK_ERR_NONPOSITIVE_MARGINAL)
            return fail(ctx, st, "every a_i and b_j must be > 0");
        if (st == ACCSINK_ERR_TIMEOUT) return fail(ctx, st, "a device barrier timed out");
        return fail(ctx, st == 0 ? ACCSINK_ERR_INVALID_ARG : st, "max C must be > 0 to scale by it");
    }

    bool use_graph = prm->use_graph && !ctx->graph_broken;
    if (use_graph) {
        rc = get_graph(ctx, cv, g, ct);
        if (rc != ACCSINK_OK) {
            // The device-side loop needs conditional graph nodes with
            // cooperative kernels; if this driver refuses, remember it and
            // run the same kernels from the host loop instead.
            ctx->graph_broken = true;
            ctx->graph_error = ctx->err;
            ctx->err.clear();
            use_graph = false;
            CK(cudaMemsetAsync(&w.st->use_cond, 0, sizeof(int32_t), s));
        }
    }
    if (use_graph) {
        CK(cudaGraphLaunch(ctx->exec, s));
    } else {
        const int unroll = 8;
        for (;;) {
            for (int u = 0; u < unroll; ++u) {
                CK(launch_passes(cv, w, g, ct, s));
                CK(launch_step(cv, w, g.step_grid, 0, s));
            }
            CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (ctx->h_state->done) break;
        }
    }
    if (prm->evaluate) {
        Work we = w;
        we.ignore_done = 1;
        CK(launch_row_pass(cv, we, g.row_grid, g.rsplit, true, s));
    }
    CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    // potentials in the units of the (possibly scaled) cost: f = eps u, g = eps x
    CK(launch_scale_out(w.u, prm->eps, f_out, n, s));
    CK(launch_scale_out(w.x, prm->eps, g_out, m, s));
    CK(cudaMemcpyAsync(ctx->h_rowpart, w.rowpart, (size_t)g.row_grid * 16, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->ev1, s));
    CK(cudaStreamSynchronize(s));

    const DevState &fs = *ctx->h_state;
    std::memset(res, 0, sizeof(*res));
    res->status = fs.status;
    res->sinkhorn_steps = fs.steps;
    res->outer_stages = fs.stages;
    res->stability_failures = fs.failures;
    res->marginal_l1 = fs.err;
    res->dual_objective = fs.dual;
    res->cost_max = fs.cmax;
    res->transport_cost = NAN;
    if (prm->evaluate) {
        double c = 0.0;
        for (int b = 0; b < g.row_grid; ++b) c += ctx->h_rowpart[2 * b + 1];
        res->transport_cost = c / fs.cost_div;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    res->gpu_ms = ms;
    res->loop_mode = use_graph ? 1 : 0;
    ctx->last_hist_count = std::min(fs.steps, prm->history);
    keep_state(ctx, fs, m, prm, start);
    if (fs.status == ACCSINK_ERR_MAXITER)
        return fail(ctx, ACCSINK_ERR_MAXITER, "not converged within max_sinkhorn_steps");
    if (fs.status != ACCSINK_OK) return fail(ctx, fs.status, "solve stopped with an error status");
    return ACCSINK_OK;
}

// A point-cloud problem's launch plan: grids, workspace views and the two
// pass views (row pass: rows of X against Y; column pass: rows of Y
// against X).
struct PointPlan {
    CostView cv;
    Geometry g;
    Work w;
    PointView pr{}, pc{};
    // sorted solve: both clouds in Hilbert-curve order (pruned passes); the views
    // read the sorted copies, outputs are scattered back through the perms
    bool sorted = false;
    PointSort sx{}, sy{};
    int prow = 1, pcol = 1, kind = 1, nblk = 1;
    double *blockmax = nullptr, *scal = nullptr;
    int32_t *hint_r = nullptr, *hint_c = nullptr;   // slot hints (sorted solves)
    float4 *qbox_r = nullptr, *qbox_c = nullptr;     // block boxes (sorted solves)
    float2 *abox_r = nullptr, *abox_c = nullptr;
    unsigned int *next_group = nullptr;              // row-group counters (sorted solves)
};

int points_grid(const accsink_ctx *ctx, int n_rows, int d)
{
    const int rw = points_rows_per_warp(d);
    const int rows = (n_rows + rw - 1) / rw;   // row tiles, one per warp pass
    const int64_t max_warps = (int64_t)ctx->num_sms * ctx->occ_pts * 8;
    const int64_t k = (rows + max_warps - 1) / max_warps;
    const int64_t warps = (rows + k - 1) / k;
    return (int)std::max<int64_t>(1, (warps + 7) / 8);
}

// Allocates the solve workspace and the O((n + m) d) point workspace and
// fills `pl`. Launches nothing.
int points_plan(accsink_ctx *ctx, const accsink_problem *prob, int hist, PointPlan &pl,
                bool sort = false)
{
    const int n = prob->n, m = prob->m, d = prob->d;
    // the spatial sort pays for solves in low dimension (colour-like clouds)
    pl.sorted = sort && d <= 4;
    pl.kind = prob->cost_kind == ACCSINK_COST_SQEUCLID ? 1 : 2;
    pl.cv.C = nullptr;
    pl.cv.ldc = m;
    pl.cv.n = n;
    pl.cv.m = m;
    pl.cv.vec = 1;
    pl.g = geometry(ctx, n, m, 1);
    pl.prow = points_grid(ctx, n, d);
    pl.pcol = points_grid(ctx, m, d);
    if (pl.sorted) {
        // the pruned passes take row groups from a counter, so every
        // resident CTA is launched (at least one group of four rows per warp)
        const int64_t full = (int64_t)ctx->num_sms * occupancy_points_pruned(d);
        auto dyn_grid = [&](int rows) {
            const int64_t groups = (rows + 3) / 4;
            return (int)std::max<int64_t>(1, std::min(full, (groups + 7) / 8));
        };
        pl.prow = dyn_grid(n);
        pl.pcol = dyn_grid(m);
    }
    int rc = ensure_workspace(ctx, n, m, 1, pl.prow, hist);
    if (rc != ACCSINK_OK) return rc;
    const int64_t ldx = (n + 3) / 4 * 4, ldy = (m + 3) / 4 * 4;
    pl.nblk = std::max(1, std::min(ctx->num_sms, (std::max(n, m) + 255) / 256));
    std::vector<size_t> sizes = {(size_t)n * 8, (size_t)m * 8, (size_t)ldx * 4, (size_t)ldx * 4,
                                 (size_t)ldy * 4, (size_t)ldy * 4, (size_t)d * ldx * 4,
                                 (size_t)d * ldx * 4, (size_t)d * ldy * 4, (size_t)d * ldy * 4,
                                 (size_t)n * 8, (size_t)pl.nblk * 40, 16};
    const size_t temp = pl.sorted ? std::max(points_sort_temp_bytes(n), points_sort_temp_bytes(m)) : 0;
    if (pl.sorted) {
        for (int c = 0; c < 2; ++c) {
            const size_t cnt = c == 0 ? (size_t)n : (size_t)m;
            for (size_t z : {(size_t)32, cnt * 4, cnt * 4, cnt * 4, cnt * 4, cnt * d * 4, cnt * 8})
                sizes.push_back(z);
        }
        sizes.push_back(std::max<size_t>(temp, 16));
        // slot hints of the pruned passes, one per group of rows of a warp
        sizes.push_back((size_t)((n + 3) / 4) * 4);
        sizes.push_back((size_t)((m + 3) / 4) * 4);
        // block boxes of the pruned passes (columns of the row pass: Y; of
        // the column pass: X)
        sizes.push_back(std::max<size_t>(16, (size_t)points_blocks(m) * 32));
        sizes.push_back(std::max<size_t>(16, (size_t)points_blocks(n) * 32));
        sizes.push_back(std::max<size_t>(16, (size_t)points_blocks(m) * 8));
        sizes.push_back(std::max<size_t>(16, (size_t)points_blocks(n) * 8));
        sizes.push_back(16);   // row-group counters of the two pruned passes
    }
    size_t need = 0;
    for (size_t z : sizes) need += align_up(z, 256);
    if (need > ctx->pts_bytes) {
        if (ctx->budget && ctx->ws_bytes + ctx->stage_bytes + ctx->ct_bytes + need > ctx->budget)
            return fail(ctx, ACCSINK_ERR_BUDGET, "point-cloud workspace exceeds the budget");
        if (ctx->pts) cudaFree(ctx->pts);
        ctx->pts = nullptr;
        ctx->pts_bytes = 0;
        free_graph(ctx);
        if (cudaMalloc(&ctx->pts, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, ACCSINK_ERR_OOM, "cudaMalloc of the point-cloud workspace failed");
        }
        ctx->pts_bytes = need;
    }
    char *p = (char *)ctx->pts;
    size_t k = 0;
    auto take = [&]() -> void * {
        void *r = p;
        p += align_up(sizes[k++], 256);
        return r;
    };
    Work &w = pl.w;
    w = ctx->w;
    w.Bx64 = (double *)take(); w.By64 = (double *)take();
    w.Bxh = (float *)take(); w.Bxl = (float *)take();
    w.Byh = (float *)take(); w.Byl = (float *)take();
    w.PXh = (float *)take(); w.PXl = (float *)take();
    w.PYh = (float *)take(); w.PYl = (float *)take();
    w.rowmax = (double *)take();
    pl.blockmax = (double *)take();
    pl.scal = (double *)take();
    if (pl.sorted) {
        for (PointSort *ps : {&pl.sx, &pl.sy}) {
            ps->box = (uint32_t *)take();
            ps->code = (uint32_t *)take();
            ps->code2 = (uint32_t *)take();
            ps->idx = (int *)take();
            ps->perm = (int *)take();
            ps->P = (float *)take();
            ps->a = (double *)take();
        }
        pl.sx.temp = pl.sy.temp = take();
        pl.sx.temp_bytes = pl.sy.temp_bytes = std::max<size_t>(temp, 16);
        pl.hint_r = (int32_t *)take();
        pl.hint_c = (int32_t *)take();
        pl.qbox_r = (float4 *)take();
        pl.qbox_c = (float4 *)take();
        pl.abox_r = (float2 *)take();
        pl.abox_c = (float2 *)take();
        pl.next_group = (unsigned int *)take();
    }
    w.ldx = ldx;
    w.ldy = ldy;
    w.nstat = 1;
    w.b_src = nullptr;
    w.f_given = nullptr;
    w.ignore_done = 0;
    PointView &pr = pl.pr, &pc = pl.pc;
    const float *Xv = pl.sorted ? pl.sx.P : prob->X, *Yv = pl.sorted ? pl.sy.P : prob->Y;
    pr.prune = pc.prune = pl.sorted ? 1 : 0;
    pr.P = Xv; pr.Pc = Yv; pr.Ah = w.G; pr.Al = w.Gk; pr.B64 = w.Bx64;
    pr.Qh = w.PYh; pr.Ql = w.PYl; pr.scal = pl.scal; pr.ldq = ldy;
    pr.nr = n; pr.nc = m; pr.d = d; pr.kind = pl.kind;
    pc.P = Yv; pc.Pc = Xv; pc.Ah = w.Fh; pc.Al = w.Fk; pc.B64 = w.By64;
    pc.Qh = w.PXh; pc.Ql = w.PXl; pc.scal = pl.scal; pc.ldq = ldx;
    pc.nr = m; pc.nc = n; pc.d = d; pc.kind = pl.kind;
    // the pruned kernels group rows by four (d <= 4)
    pr.hint = (pl.sorted && points_rows_per_warp(d) == 4) ? pl.hint_r : nullptr;
    pc.hint = (pl.sorted && points_rows_per_warp(d) == 4) ? pl.hint_c : nullptr;
    pr.skip = points_skip_log2(m);
    pc.skip = points_skip_log2(n);
    pr.qbox = pl.sorted ? pl.qbox_r : nullptr;
    pc.qbox = pl.sorted ? pl.qbox_c : nullptr;
    pr.abox = pl.sorted ? pl.abox_r : nullptr;
    pc.abox = pl.sorted ? pl.abox_c : nullptr;
    pr.next_group = pl.sorted ? pl.next_group : nullptr;
    pc.next_group = pl.sorted ? pl.next_group + 1 : nullptr;
    return ACCSINK_OK;
}

// Row maxima (for max C and the MAX_TO_ONE scale), then the FP64 norms, the
// scaled SoA copies of the points and the cost-statistics record.
cudaError_t points_prologue(const accsink_problem *prob, const PointPlan &pl, double eps,
                            cudaStream_t s)
{
    cudaError_t e = launch_points_rowmax(prob->X, prob->Y, prob->n, prob->m, prob->d, pl.kind,
                                         pl.w.rowmax, pl.prow, s);
    if (e != cudaSuccess) return e;
    return launch_points_setup(prob->X, prob->Y, prob->n, prob->m, prob->d, pl.kind,
                               prob->cost_scale == ACCSINK_SCALE_MAX_TO_ONE, eps, pl.w,
                               pl.scal, pl.blockmax, pl.nblk, s);
}

// Point-cloud costs (squared Euclidean, cosine) built on the fly: the same
// loop as solve_device with the two point passes of points.cu.
int solve_points(accsink_ctx *ctx, const accsink_problem *prob, const accsink_params *prm,
                 cudaStream_t s, double *f_out, double *g_out, accsink_result *res,
                 const SolveStart *start = nullptr)
{
    const int n = prob->n, m = prob->m;
    PointPlan pl;
    int rc = points_plan(ctx, prob, prm->history, pl, true);
    if (rc != ACCSINK_OK) return rc;
    // FP32 arguments on request (header: precision)
    pl.pr.fp32 = pl.pc.fp32 = prm->precision == ACCSINK_PRECISION_FP32 ? 1 : 0;
    // a sorted solve runs on the clouds (and marginals) in Hilbert-curve order
    accsink_problem ps = *prob;
    InitState is0 = start ? start->is : InitState();
    if (pl.sorted) {
        ps.X = pl.sx.P;
        ps.Y = pl.sy.P;
        ps.a = pl.sx.a;
        ps.b = pl.sy.a;
        is0.perm = pl.sy.perm;
    }
    const CostView &cv = pl.cv;
    const Geometry &g = pl.g;
    const Work &w = pl.w;
    const PointView &pr = pl.pr, &pc = pl.pc;
    const int prow = pl.prow, pcol = pl.pcol, kind = pl.kind;

    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.eps_user = prm->eps;
    hs.tol = stop_threshold(prm->tol);
    hs.method = prm->method;
    hs.stability = prm->stability;
    hs.carry = prm->carry;
    hs.max_steps = prm->max_sinkhorn_steps;
    hs.hist_cap = prm->history;
    hs.row_grid = prow;
    hs.col_splits = 1;
    hs.use_cond = prm->use_graph ? 1 : 0;
    hs.first = 1;
    hs.col_mode = 1;
    StageTable tab;
    start_state(hs, tab, prm, start);

    CK(cudaEventRecord(ctx->ev0, s));
    CK(set_state(ctx, hs, s));
    k_set_table<<<1, 128, 0, s>>>(tab, const_cast<double *>(w.stage_table));
    CK(cudaGetLastError());
    if (pl.sorted) {
        CK(launch_points_sort(prob->X, prob->a, n, prob->d, pl.sx, s));
        CK(launch_points_sort(prob->Y, prob->b, m, prob->d, pl.sy, s));
    }
    CK(points_prologue(&ps, pl, prm->eps, s));
    if (pl.sorted) {
        // slot hints of the pruned passes, from the sorted points alone
        CK(launch_points_hint(pl.sx.P, n, pl.sy.P, m, prob->d, kind, pl.hint_r, prow, s));
        CK(launch_points_hint(pl.sy.P, m, pl.sx.P, n, prob->d, kind, pl.hint_c, pcol, s));
        // coordinate boxes of the column blocks, from the scaled copies
        CK(launch_points_qbox(w.PYh, w.ldy, m, prob->d, pl.qbox_r, s));
        CK(launch_points_qbox(w.PXh, w.ldx, n, prob->d, pl.qbox_c, s));
    }
    CK(launch_init(cv, w, g.vec_grid, ps.a, ps.b, 0, is0, s));
    CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->h_state->done) {
        const int st = ctx->h_state->status;
        std::memset(res, 0, sizeof(*res));
        res->status = st;
        if (st == ACCSINK_ERR_NONFINITE) return fail(ctx, st, "X, Y, a or b holds NaN or Inf");
        if (st == ACCSINK_ERR_NONPOSITIVE_MARGINAL)
            return fail(ctx, st, "every a_i and b_j must be > 0");
        return fail(ctx, st == 0 ? ACCSINK_ERR_INVALID_ARG : st, "set-up failed");
    }
    auto body = [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        cudaError_t e = launch_points_pass(pr, w, prow, 0, false, cs);
        if (e != cudaSuccess) return e;
        e = launch_points_pass(pc, w, pcol, 1, false, cs);
        if (e != cudaSuccess) return e;
        return launch_step(cv, w, g.step_grid, h, cs);
    };
    bool use_graph = prm->use_graph && !ctx->graph_broken;
    if (use_graph) {
        GraphKey key;
        key.C = prob->X; key.ct = prob->Y; key.ldc = prob->d; key.n = n; key.m = m;
        key.vec = 100 + kind; key.row_grid = prow; key.colt_grid = pcol;
        key.step_grid = g.step_grid; key.ws = ctx->pts;
        key.prec = pr.fp32 * 2 + pr.prune;
        rc = build_loop_graph(ctx, key, body);
        if (rc != ACCSINK_OK) {
            ctx->graph_broken = true;
            ctx->graph_error = ctx->err;
            ctx->err.clear();
            use_graph = false;
            CK(cudaMemsetAsync(&w.st->use_cond, 0, sizeof(int32_t), s));
        }
    }
    if (use_graph) {
        CK(cudaGraphLaunch(ctx->exec, s));
    } else {
        for (;;) {
            for (int u = 0; u < 8; ++u) CK(body(s, 0));
            CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (ctx->h_state->done) break;
        }
    }
    if (prm->evaluate) {
        Work we = w;
        we.ignore_done = 1;
        CK(launch_points_pass(pr, we, prow, 0, true, s));
    }
    CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    if (pl.sorted) {
        CK(launch_scatter_scaled(w.u, prm->eps, pl.sx.perm, n, f_out, s));
        CK(launch_scatter_scaled(w.x, prm->eps, pl.sy.perm, m, g_out, s));
    } else {
        CK(launch_scale_out(w.u, prm->eps, f_out, n, s));
        CK(launch_scale_out(w.x, prm->eps, g_out, m, s));
    }
    CK(cudaMemcpyAsync(ctx->h_rowpart, w.rowpart, (size_t)prow * 16, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->ev1, s));
    CK(cudaStreamSynchronize(s));
    const DevState &fs = *ctx->h_state;
    std::memset(res, 0, sizeof(*res));
    res->status = fs.status;
    res->sinkhorn_steps = fs.steps;
    res->outer_stages = fs.stages;
    res->stability_failures = fs.failures;
    res->marginal_l1 = fs.err;
    res->dual_objective = fs.dual;
    res->cost_max = fs.cmax;
    res->transport_cost = NAN;
    if (prm->evaluate) {
        double c = 0.0;
        for (int b = 0; b < prow; ++b) c += ctx->h_rowpart[2 * b + 1];
        res->transport_cost = c;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    res->gpu_ms = ms;
    res->loop_mode = use_graph ? 1 : 0;
    ctx->last_hist_count = std::min(fs.steps, prm->history);
    keep_state(ctx, fs, m, prm, start);
    ctx->state_perm = pl.sorted ? pl.sy.perm : nullptr;
    if (fs.status == ACCSINK_ERR_MAXITER)
        return fail(ctx, ACCSINK_ERR_MAXITER, "not converged within max_sinkhorn_steps");
    if (fs.status != ACCSINK_OK) return fail(ctx, fs.status, "solve stopped with an error status");
    return ACCSINK_OK;
}

int begin(accsink_ctx *ctx)
{
    if (!ctx) return ACCSINK_ERR_INVALID_ARG;
    ctx->err.clear();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return ACCSINK_OK;
}

// Launch plan of the single-pass calls, dense or point-cloud. pass_setup
// makes the workspace, resets the state and computes the cost statistics.
struct PassPlan {
    bool pts = false;
    int scale = 0;        // dense MAX_TO_ONE: eps_c = eps max C in the prep kernels
    CostView cv;
    Geometry geo;
    Work w;
    PointPlan pp;
    int row_grid() const { return pts ? pp.prow : geo.row_grid; }
};

int pass_setup(accsink_ctx *ctx, const accsink_problem *prob, double eps, cudaStream_t s,
               PassPlan &pl)
{
    int rc = validate_problem(ctx, prob, false);
    if (rc != ACCSINK_OK) return rc;
    if (!(eps > 0.0) || !std::isfinite(eps))
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "eps must be positive and finite");
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.eps_user = eps;
    hs.mode = STEP_MAP;
    pl.pts = prob->cost_kind != ACCSINK_COST_DENSE;
    if (pl.pts) {
        rc = points_plan(ctx, prob, 0, pl.pp);
        if (rc != ACCSINK_OK) return rc;
        pl.cv = pl.pp.cv;
        pl.geo = pl.pp.g;
        pl.w = pl.pp.w;
        pl.w.ignore_done = 1;
        pl.scale = 0;   // the point set-up applies the scale inside the cost
        hs.row_grid = pl.pp.prow;
        hs.col_splits = 1;
        hs.col_mode = 1;
        CK(set_state(ctx, hs, s));
        CK(points_prologue(prob, pl.pp, eps, s));
        return ACCSINK_OK;
    }
    pl.cv = make_view(prob);
    pl.geo = geometry(ctx, prob->n, prob->m, pl.cv.vec);
    rc = ensure_workspace(ctx, prob->n, prob->m, pl.geo.splits, pl.geo.row_grid, 0,
                          pl.geo.units);
    if (rc != ACCSINK_OK) return rc;
    pl.scale = prob->cost_scale == ACCSINK_SCALE_MAX_TO_ONE;
    Work &w = pl.w;
    w = ctx->w;
    w.nstat = pl.geo.stat_grid;
    w.b_src = nullptr;
    w.f_given = nullptr;
    w.ignore_done = 1;
    hs.row_grid = pl.geo.row_grid;
    hs.col_splits = pl.geo.splits;
    CK(set_state(ctx, hs, s));
    CK(launch_cost_stats(pl.cv, w, pl.geo.stat_grid, s));
    return ACCSINK_OK;
}

cudaError_t plan_row_pass(const PassPlan &pl, const Work &w, bool with_cost, cudaStream_t s)
{
    if (pl.pts) return launch_points_pass(pl.pp.pr, w, pl.pp.prow, 0, with_cost, s);
    return launch_row_pass(pl.cv, w, pl.geo.row_grid, pl.geo.rsplit, with_cost, s);
}

// Column pass in the layout the step kernel reads (partials for a dense
// cost, ell for point clouds).
cudaError_t plan_col_pass(const PassPlan &pl, const Work &w, cudaStream_t s)
{
    if (pl.pts) return launch_points_pass(pl.pp.pc, w, pl.pp.pcol, 1, false, s);
    return launch_col_pass(pl.cv, w, pl.geo.splits, s);
}

}  // namespace

// ============================================================ C-ABI ========

extern "C" {

const char *accsink_version(void) { return "accsink 1.0 sm_103a"; }

void accsink_params_default(accsink_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->method = ACCSINK_ACC;
    p->m0 = 4;
    p->eps = 1e-2;
    p->tol = 1e-6;
    p->mu0 = 0.25;
    p->max_sinkhorn_steps = 100000;
    p->stability = ACCSINK_STAB_REPORT;
    p->carry = ACCSINK_CARRY_Y;
    p->evaluate = 1;
    p->use_graph = 1;
    p->history = 0;
    p->col_transpose = 1;
}

int accsink_create(accsink_ctx **out, int device, size_t mem_budget_bytes)
{
    if (!out) return ACCSINK_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return ACCSINK_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return ACCSINK_ERR_CUDA;
    accsink_ctx *ctx = new accsink_ctx();
    ctx->device = device;
    ctx->budget = mem_budget_bytes;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    setup_col_pass();
    for (int v = 0; v < 2; ++v) {
        ctx->occ_row[v] = occupancy_row_pass(v);
        ctx->occ_col[v] = occupancy_col_pass(v);
    }
    ctx->occ_row_warp = occupancy_row_pass_warp();
    ctx->occ_pts = occupancy_points_pass();
    ctx->occ_batch = occupancy_batch_solve();
    ctx->batch_tuning = batch_default_tuning(ctx->num_sms);
    if (setup_row_pass_tma() != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return ACCSINK_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        cudaEventCreate(&ctx->ev_mid) != cudaSuccess ||
        cudaMallocHost(&ctx->h_state, sizeof(DevState)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return ACCSINK_ERR_CUDA;
    }
    *out = ctx;
    return ACCSINK_OK;
}

void accsink_destroy(accsink_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_graph(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->ct) cudaFree(ctx->ct);
    if (ctx->pts) cudaFree(ctx->pts);
    batch_workspace_free(ctx->batch);
    if (ctx->ev_mid) cudaEventDestroy(ctx->ev_mid);
    if (ctx->h_rowpart) cudaFreeHost(ctx->h_rowpart);
    if (ctx->h_state) cudaFreeHost(ctx->h_state);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t e : ctx->up_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
}

const char *accsink_last_error(const accsink_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : "NULL context";
}

int accsink_solve(accsink_ctx *ctx, const accsink_problem *prob, const accsink_params *params,
                  void *stream, double *f_out, double *g_out, accsink_result *res)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!res) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "res is NULL");
    std::memset(res, 0, sizeof(*res));
    res->status = ACCSINK_ERR_INVALID_ARG;
    rc = validate_problem(ctx, prob, false);
    if (rc == ACCSINK_OK) rc = validate_params(ctx, params);
    if (rc == ACCSINK_OK && (!prob->a || !prob->b))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "a and b must be given");
    if (rc == ACCSINK_OK && (!f_out || !g_out))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "f_out and g_out must be given");
    if (rc != ACCSINK_OK) { res->status = rc; return rc; }
    if (prob->cost_kind == ACCSINK_COST_DENSE)
        rc = solve_device(ctx, prob, params, (cudaStream_t)stream, f_out, g_out, res);
    else
        rc = solve_points(ctx, prob, params, (cudaStream_t)stream, f_out, g_out, res);
    res->status = rc;
    return rc;
}

// Shared validation of a solve's arguments (device pointers).
static int check_solve_args(accsink_ctx *ctx, const accsink_problem *prob,
                            const accsink_params *params, double *f_out, double *g_out)
{
    int rc = validate_problem(ctx, prob, false);
    if (rc == ACCSINK_OK) rc = validate_params(ctx, params);
    if (rc == ACCSINK_OK && (!prob->a || !prob->b))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "a and b must be given");
    if (rc == ACCSINK_OK && (!f_out || !g_out))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "f_out and g_out must be given");
    return rc;
}

static int run_solve(accsink_ctx *ctx, const accsink_problem *prob, const accsink_params *params,
                     void *stream, double *f_out, double *g_out, accsink_result *res,
                     const SolveStart &start)
{
    int rc;
    if (prob->cost_kind == ACCSINK_COST_DENSE)
        rc = solve_device(ctx, prob, params, (cudaStream_t)stream, f_out, g_out, res, &start);
    else
        rc = solve_points(ctx, prob, params, (cudaStream_t)stream, f_out, g_out, res, &start);
    res->status = rc;
    return rc;
}

int accsink_export_state(accsink_ctx *ctx, accsink_state *state, void *stream)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!state || !state->x || !state->w)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "state, state->x and state->w must be given");
    if (!ctx->state_ok)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG,
                    "no solve state on this context (the last kernel-running call was not a "
                    "completed solve)");
    if (state->m != ctx->state_m)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "state->m differs from the last solve's m");
    const DevState &fs = *ctx->h_state;
    const Work &w = ctx->w;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)state->m * sizeof(double);
    if (ctx->state_perm) {
        // the solve ran on sorted columns: back to the caller's order
        CK(launch_scatter_scaled(w.x, 1.0, ctx->state_perm, state->m, state->x, s));
        if (fs.method == ACCSINK_ACC)
            CK(launch_scatter_scaled(w.w1, 1.0, ctx->state_perm, state->m, state->w, s));
        else
            CK(cudaMemsetAsync(state->w, 0, bytes, s));
    } else {
        CK(cudaMemcpyAsync(state->x, w.x, bytes, cudaMemcpyDeviceToDevice, s));
        if (fs.method == ACCSINK_ACC) CK(cudaMemcpyAsync(state->w, w.w1, bytes, cudaMemcpyDeviceToDevice, s));
        else CK(cudaMemsetAsync(state->w, 0, bytes, s));
    }
    state->method = fs.method;
    state->m_stage = fs.m_stage;
    state->j_in_stage = fs.j_in_stage;
    state->stages = fs.stages;
    state->carry = fs.carry;
    state->eps = fs.eps_user;
    state->mu0 = ctx->state_mu0;
    state->mu = fs.mu;
    state->shift_g = fs.shift_g;
    state->shift_f = fs.shift_f;
    state->cost_abs = fs.cabs;
    state->cost_min = fs.cmin;
    state->eps_c = fs.eps_c;
    CK(cudaStreamSynchronize(s));
    return ACCSINK_OK;
}

int accsink_solve_from(accsink_ctx *ctx, const accsink_problem *prob, const accsink_params *params,
                       const accsink_state *state, void *stream, double *f_out, double *g_out,
                       accsink_result *res)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!res) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "res is NULL");
    std::memset(res, 0, sizeof(*res));
    res->status = ACCSINK_ERR_INVALID_ARG;
    rc = check_solve_args(ctx, prob, params, f_out, g_out);
    if (rc == ACCSINK_OK && (!state || !state->x || !state->w))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "state, state->x and state->w must be given");
    if (rc == ACCSINK_OK && state->m != prob->m)
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "state->m must equal the problem's m");
    if (rc == ACCSINK_OK && state->method != params->method)
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "params->method must equal state->method");
    if (rc == ACCSINK_OK && !(state->eps > 0.0 && std::isfinite(state->eps)))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "state->eps must be finite and > 0");
    if (rc == ACCSINK_OK && state->method == ACCSINK_ACC &&
        !(state->mu0 > 0.0 && state->mu0 < 1.0 && state->mu > 0.0 && state->m_stage >= 1 &&
          state->j_in_stage >= 0 && state->j_in_stage < state->m_stage && state->stages >= 0 &&
          state->stages < kMaxStages))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "the state's homotopy position is not valid");
    if (rc != ACCSINK_OK) { res->status = rc; return rc; }
    SolveStart st;
    st.is.x = state->x;
    st.is.w = state->method == ACCSINK_ACC ? state->w : nullptr;
    st.is.mul = state->eps / params->eps;
    st.is.keep_shifts = state->eps == params->eps ? 1 : 0;
    st.is.shift_g = state->shift_g;
    st.is.shift_f = state->shift_f;
    st.is.cabs = state->cost_abs;
    st.is.cmin = state->cost_min;
    st.is.eps_c = state->eps_c;
    if (state->method == ACCSINK_ACC) {
        st.stage = true;
        st.mu = state->mu;
        st.mu0 = state->mu0;
        st.m_stage = state->m_stage;
        st.j = state->j_in_stage;
        st.stages = state->stages;
    }
    return run_solve(ctx, prob, params, stream, f_out, g_out, res, st);
}

int accsink_warm_start(accsink_ctx *ctx, const accsink_problem *prob, const accsink_params *params,
                       const double *g0, void *stream, double *f_out, double *g_out,
                       accsink_result *res)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!res) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "res is NULL");
    std::memset(res, 0, sizeof(*res));
    res->status = ACCSINK_ERR_INVALID_ARG;
    rc = check_solve_args(ctx, prob, params, f_out, g_out);
    if (rc == ACCSINK_OK && !g0) rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "g0 must be given");
    if (rc != ACCSINK_OK) { res->status = rc; return rc; }
    SolveStart st;
    st.is.x = g0;
    st.is.div = params->eps;
    return run_solve(ctx, prob, params, stream, f_out, g_out, res, st);
}

namespace {

// Uploads a dense host cost into pd->C (the device staging buffer, row
// stride pd->ldc) in row chunks on a copy stream, and writes C^T and the
// cost statistics of each chunk on s as soon as it has landed, so the one
// read of C they need overlaps with the rest of the upload. Only where the
// solve would take that fused path (a transposed copy, 16-byte rows);
// returns the number of statistics partials written, 0 when it did nothing
// (the caller uploads C whole), or -1 on a CUDA error.
int upload_dense_overlapped(accsink_ctx *ctx, const accsink_problem *pd, const float *C_host,
                            const accsink_params *prm, cudaStream_t s)
{
    const CostView cv = make_view(pd);
    const int n = pd->n, m = pd->m;
    if (!cv.vec || !prm->col_transpose || n < 2 * 64) return 0;
    const Geometry g = geometry(ctx, n, m, cv.vec);
    if (ensure_workspace(ctx, n, m, g.splits, g.row_grid, prm->history, g.units) != ACCSINK_OK)
        return 0;
    if (!ensure_ct(ctx, n, m)) return 0;
    if (!ctx->copy_stream &&
        cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return -1;
    for (cudaEvent_t &e : ctx->up_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return -1;
    const int grid = std::max(1, g.stat_grid / kUploadChunks);
    const int rows = (int)(((n + kUploadChunks - 1) / kUploadChunks + 63) / 64 * 64);
    const int64_t ldc = cv.ldc;
    // the staging buffer may still be read by earlier work on s
    if (cudaEventRecord(ctx->up_ev[kUploadChunks], s) != cudaSuccess ||
        cudaStreamWaitEvent(ctx->copy_stream, ctx->up_ev[kUploadChunks], 0) != cudaSuccess)
        return -1;
    const Work w = ctx->w;
    int parts = 0;
    for (int c = 0, r0 = 0; r0 < n; ++c, r0 += rows) {
        const int r1 = std::min(n, r0 + rows);
        const size_t off = (size_t)r0 * (size_t)ldc;
        const size_t cnt = (size_t)(r1 - 1 - r0) * (size_t)ldc + (size_t)m;
        if (cudaMemcpyAsync(const_cast<float *>(pd->C) + off, C_host + off, cnt * sizeof(float),
                            cudaMemcpyHostToDevice, ctx->copy_stream) != cudaSuccess ||
            cudaEventRecord(ctx->up_ev[c], ctx->copy_stream) != cudaSuccess ||
            cudaStreamWaitEvent(s, ctx->up_ev[c], 0) != cudaSuccess ||
            launch_transpose_stats(cv, ctx->ct, ct_ld(n), w, grid, s, r0, r1, parts) != cudaSuccess)
            return -1;
        parts += grid;
    }
    return parts;
}

}  // namespace

int accsink_solve_host(accsink_ctx *ctx, const accsink_problem *prob_host,
                       const accsink_params *params, void *stream, double *f_out_host,
                       double *g_out_host, accsink_result *res)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!res) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "res is NULL");
    std::memset(res, 0, sizeof(*res));
    rc = validate_problem(ctx, prob_host, false);
    if (rc == ACCSINK_OK) rc = validate_params(ctx, params);
    if (rc == ACCSINK_OK && (!prob_host->a || !prob_host->b || !f_out_host || !g_out_host))
        rc = fail(ctx, ACCSINK_ERR_INVALID_ARG, "a, b, f_out and g_out must be given");
    if (rc != ACCSINK_OK) { res->status = rc; return rc; }
    const int n = prob_host->n, m = prob_host->m;
    const bool dense = prob_host->cost_kind == ACCSINK_COST_DENSE;
    const int64_t ldc = prob_host->ldc ? prob_host->ldc : m;
    // dense: C; point clouds: X (n x d) then Y (m x d)
    const size_t xbytes = dense ? 0 : (size_t)n * (size_t)prob_host->d * sizeof(float);
    const size_t ybytes = dense ? 0 : (size_t)m * (size_t)prob_host->d * sizeof(float);
    const size_t cbytes = dense ? ((size_t)(n - 1) * (size_t)ldc + (size_t)m) * sizeof(float)
                                : align_up(xbytes, 256) + ybytes;
    const size_t need = align_up(cbytes, 256) + align_up((size_t)n * 8, 256) * 2 +
                        align_up((size_t)m * 8, 256) * 2;
    if (need > ctx->stage_bytes) {
        if (ctx->stage) cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        if (ctx->budget && need > ctx->budget) {
            res->status = ACCSINK_ERR_BUDGET;
            return fail(ctx, ACCSINK_ERR_BUDGET, "staging buffers exceed the budget");
        }
        if (cudaMalloc(&ctx->stage, need) != cudaSuccess) {
            cudaGetLastError();
            res->status = ACCSINK_ERR_OOM;
            return fail(ctx, ACCSINK_ERR_OOM, "cudaMalloc of the staging buffers failed");
        }
        ctx->stage_bytes = need;
    }
    char *p = (char *)ctx->stage;
    float *dC = (float *)p; p += align_up(cbytes, 256);
    double *da = (double *)p; p += align_up((size_t)n * 8, 256);
    double *df = (double *)p; p += align_up((size_t)n * 8, 256);
    double *db = (double *)p; p += align_up((size_t)m * 8, 256);
    double *dg = (double *)p;
    cudaStream_t s = (cudaStream_t)stream;
    accsink_problem pd = *prob_host;
    int prepared = 0;
    if (dense) {
        pd.C = dC;
        pd.ldc = ldc;
        prepared = upload_dense_overlapped(ctx, &pd, prob_host->C, params, s);
        if (prepared < 0) {
            res->status = ACCSINK_ERR_CUDA;
            return fail(ctx, ACCSINK_ERR_CUDA, "overlapped upload of C failed");
        }
        if (prepared == 0) CK(cudaMemcpyAsync(dC, prob_host->C, cbytes, cudaMemcpyHostToDevice, s));
    } else {
        float *dY = (float *)((char *)dC + align_up(xbytes, 256));
        CK(cudaMemcpyAsync(dC, prob_host->X, xbytes, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dY, prob_host->Y, ybytes, cudaMemcpyHostToDevice, s));
        pd.X = dC;
        pd.Y = dY;
    }
    CK(cudaMemcpyAsync(da, prob_host->a, (size_t)n * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(db, prob_host->b, (size_t)m * 8, cudaMemcpyHostToDevice, s));
    pd.a = da;
    pd.b = db;
    rc = dense ? solve_device(ctx, &pd, params, s, df, dg, res, nullptr, prepared)
               : solve_points(ctx, &pd, params, s, df, dg, res);
    if (rc != ACCSINK_OK && rc != ACCSINK_ERR_MAXITER) { res->status = rc; return rc; }
    CK(cudaMemcpyAsync(f_out_host, df, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(g_out_host, dg, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    res->status = rc;
    return rc;
}

int accsink_get_history(accsink_ctx *ctx, int32_t capacity, double *err, double *dual,
                        double *mu, int32_t *stab, double *cond, int32_t *count)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!count || capacity < 0) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "bad history arguments");
    const int k = std::min(capacity, ctx->last_hist_count);
    *count = k;
    if (k == 0) return ACCSINK_OK;
    if (err) CK(cudaMemcpy(err, ctx->w.h_err, (size_t)k * 8, cudaMemcpyDeviceToHost));
    if (dual) CK(cudaMemcpy(dual, ctx->w.h_dual, (size_t)k * 8, cudaMemcpyDeviceToHost));
    if (mu) CK(cudaMemcpy(mu, ctx->w.h_mu, (size_t)k * 8, cudaMemcpyDeviceToHost));
    if (stab) CK(cudaMemcpy(stab, ctx->w.h_stab, (size_t)k * 4, cudaMemcpyDeviceToHost));
    if (cond) CK(cudaMemcpy(cond, ctx->w.h_cond, (size_t)k * 32, cudaMemcpyDeviceToHost));
    return ACCSINK_OK;
}

int accsink_row_pass(accsink_ctx *ctx, const accsink_problem *prob, double eps, const double *g,
                     double *f_out, void *stream)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!prob || !g || !f_out || !prob->a)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "g, f_out and a must be given");
    cudaStream_t s = (cudaStream_t)stream;
    PassPlan pl;
    rc = pass_setup(ctx, prob, eps, s, pl);
    if (rc != ACCSINK_OK) return rc;
    CK(launch_prep_g(pl.cv, pl.w, pl.geo.vec_grid, g, prob->a, eps, pl.scale, s));
    CK(plan_row_pass(pl, pl.w, false, s));
    CK(launch_scale_out(pl.w.u, eps, f_out, prob->n, s));
    return ACCSINK_OK;
}

int accsink_col_lse(accsink_ctx *ctx, const accsink_problem *prob, double eps, const double *f,
                    double *ell_out, void *stream)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!prob || !f || !ell_out) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "f and ell_out must be given");
    cudaStream_t s = (cudaStream_t)stream;
    PassPlan pl;
    rc = pass_setup(ctx, prob, eps, s, pl);
    if (rc != ACCSINK_OK) return rc;
    CK(launch_prep_f(pl.cv, pl.w, pl.geo.vec_grid, f, eps, pl.scale, s));
    CK(plan_col_pass(pl, pl.w, s));
    if (pl.pts)
        CK(cudaMemcpyAsync(ell_out, pl.w.ell, (size_t)prob->m * 8, cudaMemcpyDeviceToDevice, s));
    else
        CK(launch_col_finish_lse(pl.w, prob->m, ell_out, s));
    return ACCSINK_OK;
}

int accsink_sinkhorn_map(accsink_ctx *ctx, const accsink_problem *prob, double eps,
                         const double *g, double *f_out, double *c_out, double *s_out,
                         double *err_out, void *stream)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!prob || !g || !f_out || !c_out || !s_out || !err_out || !prob->a || !prob->b)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "every pointer argument must be given");
    cudaStream_t s = (cudaStream_t)stream;
    PassPlan pl;
    rc = pass_setup(ctx, prob, eps, s, pl);
    if (rc != ACCSINK_OK) return rc;
    Work w = pl.w;
    w.b_src = prob->b;
    CK(launch_prep_g(pl.cv, w, pl.geo.vec_grid, g, prob->a, eps, pl.scale, s));
    CK(plan_row_pass(pl, w, false, s));
    CK(plan_col_pass(pl, w, s));
    CK(launch_step_map(pl.cv, w, pl.geo.step_grid, c_out, s_out, s));
    CK(launch_scale_out(w.u, eps, f_out, prob->n, s));
    CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *err_out = ctx->h_state->err;
    if (ctx->h_state->nonfinite)
        return fail(ctx, ACCSINK_ERR_NONFINITE, "the cost or the points hold NaN or Inf");
    return ACCSINK_OK;
}

int accsink_transport_cost(accsink_ctx *ctx, const accsink_problem *prob, double eps,
                           const double *f, const double *g, double *cost_out, void *stream)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!prob || !f || !g || !cost_out)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "f, g and cost_out must be given");
    cudaStream_t s = (cudaStream_t)stream;
    PassPlan pl;
    rc = pass_setup(ctx, prob, eps, s, pl);
    if (rc != ACCSINK_OK) return rc;
    // The row pass at g weighs row i by w_i = exp(f_i/eps + LSE_i), so that
    // w_i * (sum_j C_ij t_ij) / (sum_j t_ij) = sum_j C_ij P_ij.
    Work w = pl.w;
    w.f_given = f;
    CK(launch_prep_g(pl.cv, w, pl.geo.vec_grid, g, nullptr, eps, pl.scale, s));
    CK(plan_row_pass(pl, w, true, s));
    const int rg = pl.row_grid();
    CK(cudaMemcpyAsync(ctx->h_rowpart, w.rowpart, (size_t)rg * 16, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double c = 0.0;
    for (int b = 0; b < rg; ++b) c += ctx->h_rowpart[2 * b + 1];
    *cost_out = c / ctx->h_state->cost_div;   // in units of the scaled cost
    return ACCSINK_OK;
}

int accsink_time_passes(accsink_ctx *ctx, const accsink_problem *prob, double eps,
                        const double *g, int reps, void *stream, float *row_ms, float *col_ms)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!prob || !g || !prob->a || reps < 1)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "g and a must be given and reps >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    PassPlan pl;
    rc = pass_setup(ctx, prob, eps, s, pl);
    if (rc != ACCSINK_OK) return rc;
    const CostView &cv = pl.cv;
    const Geometry &geo = pl.geo;
    const Work &w = pl.w;
    if (pl.pts) {
        // the two point passes, as the solver launches them
        CK(launch_prep_g(cv, w, geo.vec_grid, g, prob->a, eps, 0, s));
        CK(plan_row_pass(pl, w, false, s));                 // warm-up, writes A'
        CK(plan_col_pass(pl, w, s));
        float ms = 0.0f;
        CK(cudaEventRecord(ctx->ev0, s));
        for (int r = 0; r < reps; ++r) CK(plan_row_pass(pl, w, false, s));
        CK(cudaEventRecord(ctx->ev1, s));
        CK(cudaEventSynchronize(ctx->ev1));
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        if (row_ms) *row_ms = ms / reps;
        CK(cudaEventRecord(ctx->ev0, s));
        for (int r = 0; r < reps; ++r) CK(plan_col_pass(pl, w, s));
        CK(cudaEventRecord(ctx->ev1, s));
        CK(cudaEventSynchronize(ctx->ev1));
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        if (col_ms) *col_ms = ms / reps;
        return ACCSINK_OK;
    }
    // the column pass the solver would use: on C^T when it fits
    const float *ct = ensure_ct(ctx, prob->n, prob->m) ? ctx->ct : nullptr;
    CK(launch_prep_g(cv, w, geo.vec_grid, g, prob->a, eps, pl.scale, s));
    if (ct) CK(launch_transpose(cv, ctx->ct, ct_ld(prob->n), s));
    CK(launch_passes(cv, w, geo, ct, s));                 // warm-up, writes F
    CK(cudaEventRecord(ctx->ev0, s));
    for (int r = 0; r < reps; ++r) CK(launch_row_pass(cv, w, geo.row_grid, geo.rsplit, false, s));
    CK(cudaEventRecord(ctx->ev1, s));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (row_ms) *row_ms = ms / reps;
    CK(cudaEventRecord(ctx->ev0, s));
    for (int r = 0; r < reps; ++r) {
        if (ct) CK(launch_col_pass_transposed(ct, ct_ld(prob->n), prob->n, prob->m, w,
                                              geo.colt_grid, geo.csplit, s));
        else CK(launch_col_pass(cv, w, geo.splits, s));
    }
    CK(cudaEventRecord(ctx->ev1, s));
    CK(cudaEventSynchronize(ctx->ev1));
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (col_ms) *col_ms = ms / reps;
    return ACCSINK_OK;
}

int accsink_selftest_timeout(accsink_ctx *ctx, double limit_s, int32_t *status_out,
                             double *elapsed_s)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!status_out || !elapsed_s || !(limit_s > 0.0) || limit_s > 2.0)
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "status_out, elapsed_s and 0 < limit_s <= 2");
    // the solver's own workspace and state (the next solve rewrites both)
    rc = ensure_workspace(ctx, 64, 64, 1, 1, 0);
    if (rc != ACCSINK_OK) return rc;
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    cudaStream_t s = nullptr;
    CK(set_state(ctx, hs, s));
    const int grid = std::max(2, std::min(ctx->num_sms, 8));
    const auto t0 = std::chrono::steady_clock::now();
    CK(launch_barrier_selftest(ctx->w.st, grid, (uint64_t)(limit_s * 1e9), s));
    CK(cudaMemcpyAsync(ctx->h_state, ctx->w.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *elapsed_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *status_out = ctx->h_state->status;
    return ACCSINK_OK;
}

int accsink_launch_geometry(accsink_ctx *ctx, int32_t n, int32_t m, int32_t vec, int32_t *out6)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    if (!out6 || n < 1 || m < 1) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "bad arguments");
    const Geometry g = geometry(ctx, n, m, vec ? 1 : 0);
    out6[0] = ctx->num_sms;
    out6[1] = g.row_grid;
    out6[2] = g.splits;
    out6[3] = (m + kColStrip - 1) / kColStrip;
    out6[4] = g.step_grid;
    out6[5] = g.stat_grid;
    return ACCSINK_OK;
}

}  // extern "C"

// ------------------------------------------------------------- batches --

namespace {

int validate_batch(accsink_ctx *ctx, int32_t count, const accsink_problem *probs,
                   const accsink_params *params, double *const *f_out, double *const *g_out,
                   accsink_result *res)
{
    if (count < 0) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "count must be >= 0");
    if (count > 0 && (!probs || !params || !f_out || !g_out || !res))
        return fail(ctx, ACCSINK_ERR_INVALID_ARG, "probs, params, f_out, g_out and res must be given");
    for (int k = 0; k < count; ++k) {
        const accsink_problem *p = &probs[k];
        const std::string at = " (problem " + std::to_string(k) + ")";
        if (p->n < 1 || p->m < 1) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "n and m must be >= 1" + at);
        if (p->cost_kind == ACCSINK_COST_DENSE) {
            if (!p->C) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "C is NULL" + at);
            if (p->ldc && p->ldc < p->m) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "ldc < m" + at);
        } else if (p->cost_kind == ACCSINK_COST_SQEUCLID || p->cost_kind == ACCSINK_COST_COSINE) {
            if (!p->X || !p->Y) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "X and Y must be given" + at);
            if (p->d < 1 || p->d > 4096)
                return fail(ctx, ACCSINK_ERR_INVALID_ARG, "point dimension d must be in 1..4096" + at);
        } else {
            return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown cost_kind" + at);
        }
        if (p->cost_scale != ACCSINK_SCALE_NONE && p->cost_scale != ACCSINK_SCALE_MAX_TO_ONE)
            return fail(ctx, ACCSINK_ERR_INVALID_ARG, "unknown cost_scale" + at);
        if (!p->a || !p->b) return fail(ctx, ACCSINK_ERR_INVALID_ARG, "a and b must be given" + at);
        if (!f_out[k] || !g_out[k])
            return fail(ctx, ACCSINK_ERR_INVALID_ARG, "f_out and g_out must be given" + at);
        const int rc = validate_params(ctx, &params[k]);
        if (rc != ACCSINK_OK) { ctx->err += at; return rc; }
    }
    return ACCSINK_OK;
}

// A dense problem that the single-solve path (graph loop over the stored
// cost, 4 bytes per entry per pass) serves better than the batched launch
// (8 bytes of K per entry per pass, items shared with the other problems):
// a batch's only dense problem at any size (about 3x faster alone at every
// size measured, 256^2 to 8192^2), and from tn.dense_solo_min_nm entries on
// (there a dense problem costs the batched launch more device time than it
// takes alone).
bool dense_solo(const BatchTuning &tn, int32_t count, const accsink_problem &p)
{
    if (p.cost_kind != ACCSINK_COST_DENSE || tn.dense_solo_min_nm < 0) return false;
    return count == 1 || (int64_t)p.n * p.m >= (int64_t)tn.dense_solo_min_nm;
}

// The batch's return code from the parts' codes: OK, MAXITER when some
// problems did not converge, else the first other error.
int merge_status(int rc, int part)
{
    if (part == ACCSINK_OK) return rc;
    if (rc == ACCSINK_OK || (rc == ACCSINK_ERR_MAXITER && part != ACCSINK_ERR_MAXITER)) return part;
    return rc;
}

// Solves a batch: the dense problems that dense_solo picks one at a time by
// the single-solve path (after the batched launch, with use_graph set and no
// history), the others in one batched launch. with_solo = false leaves the
// solo problems' outputs and results untouched (the autotuner solves them
// once).
int run_batch(accsink_ctx *ctx, const BatchTuning &tn, int32_t count, const accsink_problem *probs,
              const accsink_params *params, void *stream, double *const *f_out,
              double *const *g_out, accsink_result *res, bool with_solo = true)
{
    ctx->batch_timing = BatchTiming{};
    if (count == 0) return ACCSINK_OK;
    std::vector<int> solo, rest;
    for (int k = 0; k < count; ++k) (dense_solo(tn, count, probs[k]) ? solo : rest).push_back(k);
    int rc = ACCSINK_OK;
    std::string err;
    if (!rest.empty()) {
        const int nr = (int)rest.size();
        std::vector<accsink_problem> rp(nr);
        std::vector<accsink_params> rq(nr);
        std::vector<double *> rf(nr), rg(nr);
        std::vector<accsink_result> rr(nr);
        for (int i = 0; i < nr; ++i) {
            rp[i] = probs[rest[i]];
            rq[i] = params[rest[i]];
            rf[i] = f_out[rest[i]];
            rg[i] = g_out[rest[i]];
        }
        BatchEnv env;
        env.num_sms = ctx->num_sms;
        env.occ_solve = ctx->occ_batch;
        const size_t used = ctx->ws_bytes + ctx->stage_bytes + ctx->ct_bytes + ctx->pts_bytes;
        env.budget_left = ctx->budget ? (ctx->budget > used ? ctx->budget - used : 1) : 0;
        env.ev0 = ctx->ev0;
        env.ev_mid = ctx->ev_mid;
        env.ev1 = ctx->ev1;
        rc = batch_run(env, ctx->batch, tn, nr, rp.data(), rq.data(), rf.data(), rg.data(),
                       rr.data(), (cudaStream_t)stream, err, &ctx->batch_timing);
        for (int i = 0; i < nr; ++i) res[rest[i]] = rr[i];
        if (rc != ACCSINK_OK && rc != ACCSINK_ERR_MAXITER) return fail(ctx, rc, err);
    }
    if (!with_solo) {
        if (rc != ACCSINK_OK) return fail(ctx, rc, err);
        return ACCSINK_OK;
    }
    float solo_ms = 0.0f;
    for (int k : solo) {
        accsink_params q = params[k];
        q.use_graph = 1;
        q.history = 0;
        std::memset(&res[k], 0, sizeof(res[k]));
        const int r = solve_device(ctx, &probs[k], &q, (cudaStream_t)stream, f_out[k], g_out[k],
                                   &res[k]);
        res[k].status = r;
        if (r != ACCSINK_OK && r != ACCSINK_ERR_MAXITER && err.empty())
            err = "problem " + std::to_string(k) + ": " + ctx->err;
        solo_ms += (float)res[k].gpu_ms;
        rc = merge_status(rc, r);
    }
    ctx->batch_timing.solo_ms = solo_ms;
    ctx->batch_timing.total_ms += solo_ms;
    ctx->batch_timing.solve_ms += solo_ms;
    if (rc == ACCSINK_ERR_MAXITER) err = "some problems did not converge within max_sinkhorn_steps";
    else if (rc != ACCSINK_OK && err.empty())
        err = "some problems stopped with an error status (see res[k].status)";
    if (rc != ACCSINK_OK) return fail(ctx, rc, err);
    return ACCSINK_OK;
}

}  // namespace

extern "C" {

int accsink_solve_batch(accsink_ctx *ctx, int32_t count, const accsink_problem *probs,
                        const accsink_params *params, void *stream, double *const *f_out,
                        double *const *g_out, accsink_result *res)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    rc = validate_batch(ctx, count, probs, params, f_out, g_out, res);
    if (rc != ACCSINK_OK) return rc;
    return run_batch(ctx, ctx->batch_tuning, count, probs, params, stream, f_out, g_out, res);
}

int accsink_batch_set_config(accsink_ctx *ctx, const accsink_batch_config *cfg)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    BatchTuning t = batch_default_tuning(ctx->num_sms);
    if (cfg) {
        if (cfg->small_max_nm < 0 || cfg->row_tile_elems < 0 || cfg->ctas_per_sm < 0)
            return fail(ctx, ACCSINK_ERR_INVALID_ARG,
                        "small_max_nm, row_tile_elems and ctas_per_sm must be >= 0");
        if (cfg->small_max_nm) t.small_max_nm = cfg->small_max_nm;
        if (cfg->row_tile_elems) t.row_tile_elems = cfg->row_tile_elems;
        t.ctas_per_sm = cfg->ctas_per_sm;
        if (cfg->dense_solo_min_nm) t.dense_solo_min_nm = cfg->dense_solo_min_nm < 0 ? -1 : cfg->dense_solo_min_nm;
    }
    ctx->batch_tuning = t;
    return ACCSINK_OK;
}

int accsink_batch_get_config(const accsink_ctx *ctx, accsink_batch_config *cfg)
{
    if (!ctx || !cfg) return ACCSINK_ERR_INVALID_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->small_max_nm = ctx->batch_tuning.small_max_nm;
    cfg->row_tile_elems = ctx->batch_tuning.row_tile_elems;
    cfg->ctas_per_sm = ctx->batch_tuning.ctas_per_sm;
    cfg->dense_solo_min_nm = ctx->batch_tuning.dense_solo_min_nm;
    return ACCSINK_OK;
}

int accsink_batch_autotune(accsink_ctx *ctx, int32_t count, const accsink_problem *probs,
                           const accsink_params *params, void *stream, double *const *f_out,
                           double *const *g_out, accsink_result *res, accsink_batch_config *best,
                           float *times_ms, int32_t cap, int32_t *tried)
{
    int rc = begin(ctx);
    if (rc != ACCSINK_OK) return rc;
    rc = validate_batch(ctx, count, probs, params, f_out, g_out, res);
    if (rc != ACCSINK_OK) return rc;
    // Candidates: the small-problem cut-off, the row-item size and the
    // persistent CTAs per SM, around the defaults.
    const int smalls[] = {1 << 14, 1 << 16, 1 << 18};
    const int tiles[] = {1 << 14, 1 << 16, 1 << 18};
    const int per_sm[] = {0, 1};
    // The dense problems solved one at a time are solved with the first
    // candidate only; the candidates are compared on the batched launch.
    BatchTuning bt = ctx->batch_tuning;
    float best_ms = INFINITY;
    int k = 0;
    for (int sm : smalls)
        for (int tl : tiles)
            for (int ps : per_sm) {
                BatchTuning t = ctx->batch_tuning;
                t.small_max_nm = sm;
                t.row_tile_elems = tl;
                t.ctas_per_sm = ps;
                const int r = run_batch(ctx, t, count, probs, params, stream, f_out, g_out, res,
                                        k == 0);
                if (r != ACCSINK_OK && r != ACCSINK_ERR_MAXITER) return r;
                const float ms = ctx->batch_timing.total_ms - ctx->batch_timing.solo_ms;
                if (times_ms && k < cap) times_ms[k] = ms;
                ++k;
                if (ms < best_ms) { best_ms = ms; bt = t; }
            }
    ctx->batch_tuning = bt;
    if (tried) *tried = k;
    if (best) {
        std::memset(best, 0, sizeof(*best));
        best->small_max_nm = bt.small_max_nm;
        best->row_tile_elems = bt.row_tile_elems;
        best->ctas_per_sm = bt.ctas_per_sm;
        best->dense_solo_min_nm = bt.dense_solo_min_nm;
    }
    return ACCSINK_OK;
}

int accsink_batch_last_timing(const accsink_ctx *ctx, float *total_ms, float *form_ms,
                              float *solve_ms)
{
    if (!ctx) return ACCSINK_ERR_INVALID_ARG;
    if (total_ms) *total_ms = ctx->batch_timing.total_ms;
    if (form_ms) *form_ms = ctx->batch_timing.form_ms;
    if (solve_ms) *solve_ms = ctx->batch_timing.solve_ms;
    return ACCSINK_OK;
}

}  // extern "C"

// Host side of the batched solver: plans a batch (work split, workspace
// layout, initial queue), launches the formation and the persistent solve,
// and collects the results. Called by accsink_solve_batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "accsink.h"
#include "accsink_internal.cuh"
#include "batch_internal.cuh"
#include "batch_host.h"

namespace accsink {

namespace {

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Sizes of one problem's arrays, in the order they are carved.
struct ProbLayout {
    size_t kh, kl, kth, ktl, a, loga, u, fh, fl, mvec, gh, gl, rowpart, colrec, p2rec;
    size_t total() const
    {
        return kh + kl + kth + ktl + a + loga + u + fh + fl + 12 * mvec + gh + gl + rowpart +
               colrec + p2rec;
    }
};

ProbLayout layout(int64_t n, int64_t m, int row_tiles, int col_tiles, bool transposed,
                  int step_items)
{
    const int64_t ldm = (m + 3) / 4 * 4, n4 = (n + 3) / 4 * 4;
    ProbLayout L;
    L.kh = L.kl = up256((size_t)n * ldm * 4);
    L.kth = L.ktl = transposed ? up256((size_t)m * n4 * 4) : 0;
    L.a = L.loga = L.u = up256((size_t)n * 8);
    L.fh = L.fl = up256((size_t)n4 * 4);
    L.mvec = up256((size_t)m * 8);
    L.gh = L.gl = up256((size_t)ldm * 4);
    L.rowpart = up256((size_t)row_tiles * 16);
    L.colrec = up256((size_t)col_tiles * kBatchColRec * 8);
    L.p2rec = up256((size_t)step_items * 3 * 8);
    return L;
}

unsigned long long pow2_at_least(unsigned long long v)
{
    unsigned long long c = 1;
    while (c < v) c <<= 1;
    return c;
}

}  // namespace

void batch_workspace_free(BatchWorkspace &ws)
{
    if (ws.exec) cudaGraphExecDestroy(ws.exec);
    if (ws.cap) cudaStreamDestroy(ws.cap);
    if (ws.dev) cudaFree(ws.dev);
    if (ws.host) cudaFreeHost(ws.host);
    ws = BatchWorkspace{};
}

BatchTuning batch_default_tuning(int num_sms)
{
    BatchTuning t;
    t.small_max_nm = 1 << 16;
    t.row_tile_elems = 1 << 16;
    t.ctas_per_sm = 0;          // occupancy
    t.dense_solo_min_nm = 1 << 24;
    (void)num_sms;
    return t;
}

namespace {

// The work split and sizes of a batch (host records; device pointers are
// filled in when the workspace is carved).
struct BatchPlan {
    std::vector<BatchProb> hp;
    std::vector<ProbLayout> lay;
    // formation tiles: CUDA-core (64 x 64), then scaling (64 x 64, scaled
    // problems), then tensor-core (128 x 64)
    std::vector<BatchTile> tiles;
    int nform = 0, nscale = 0, ntct = 0;
    std::vector<int32_t> tcp;       // tensor-core problems
    std::vector<int64_t> tcs;       // their first slice rows
    int64_t R = 0;                  // slice rows
    int dpad = 0;
    size_t slice_bytes = 0, expo_bytes = 0;
    unsigned long long cap = 0;
    size_t head_bytes = 0, data_bytes = 0;
};

// ACCSINK_BATCH_STEP_ITEMS=0 keeps a large problem's step in one CTA.
bool step_items_enabled()
{
    const char *e = std::getenv("ACCSINK_BATCH_STEP_ITEMS");
    return !(e && std::strcmp(e, "0") == 0);
}

// ACCSINK_BATCH_GRAPH=0 issues a batch's launch sequence directly instead of
// replaying it as a CUDA graph.
bool batch_graph_enabled()
{
    const char *e = std::getenv("ACCSINK_BATCH_GRAPH");
    return !(e && e[0] == '0');
}

// Cosine costs with kBatchTcMinD <= d <= kBatchTcMaxD are formed on the
// tensor cores unless ACCSINK_BATCH_FORM=cuda selects the CUDA-core
// expansion for every problem.
bool tc_form_enabled()
{
    const char *e = std::getenv("ACCSINK_BATCH_FORM");
    if (e && std::strcmp(e, "cuda") == 0) return false;
    return batch_tc_available();
}

// The work split of one problem that depends only on its size, the tuning
// and whether the batch is wide (the BatchProb fields small, rows_per_tile,
// row_tiles, col_tiles, ldn, cols_per_item, col_items, step_cols,
// step_items) and its layout.
struct ProbShape {
    int small = 0, rows_per_tile = 0, row_tiles = 0, col_tiles = 0, cols_per_item = 0,
        col_items = 0, step_cols = 0, step_items = 0;
    bool transposed = false;
    ProbLayout lay{};
};

// Problems from kBatchTransposeMin entries are always tiled over K and K^T,
// whatever the split, so a problem's layout (and its last bits) depends only
// on its size.
bool is_small(const BatchTuning &tn, const accsink_problem &q)
{
    const int64_t nm = (int64_t)q.n * q.m;
    return nm <= tn.small_max_nm && nm < kBatchTransposeMin;
}

// Rows of a row item that give every (virtual) warp of the CTA four rows:
// the row pass works on four rows at a time per segment of L lanes (L the
// lanes a row of m columns takes, at most 32).
int full_rows(int m)
{
    const int m4 = (m + 3) / 4;
    int L = 1;
    while (L < m4 && L < 32) L <<= 1;
    return 4 * (kBatchThreads / 32) * (32 / L);
}

// wide: the batch has row items of full_rows rows enough for the resident
// CTAs (see plan_batch). The rows of an item do not change any potential
// (each row is reduced by one warp segment whatever the item), only the
// order of the per-item dual and cost partials.
ProbShape prob_shape(const BatchTuning &tn, const accsink_problem &q, bool wide = false)
{
    ProbShape S;
    const int64_t nm = (int64_t)q.n * q.m;
    S.small = is_small(tn, q) ? 1 : 0;
    if (S.small) {
        S.rows_per_tile = q.n;
        S.row_tiles = 1;
    } else {
        // at least one row for each of the CTA's warps, so none idles;
        // when the batch is wide or the problem has rows enough for 512
        // items of them, four rows for each (virtual) warp: fewer leave
        // loads out of flight (8-row tiles of a 16384-column problem ran at
        // 65% of HBM bandwidth; with 32 rows, 16384^2 steps took 6% less
        // time, while 8192^2 and 4096^2 ones alone, then short of items
        // for the resident CTAs, took 13-20% more; in a batch of 256
        // serving requests the solve took 11% less time, in the 512-problem
        // word-alignment batch 5% less)
        const int full = full_rows(q.m);
        const int rmin = (wide || q.n / full >= 512) ? full : kBatchThreads / 32;
        int rpt = (int)std::max<int64_t>(rmin, tn.row_tile_elems / std::max(1, q.m));
        rpt = std::min(rpt, q.n);
        S.rows_per_tile = rpt;
        S.row_tiles = (q.n + rpt - 1) / rpt;
    }
    S.col_tiles = (q.m + kBatchColTile - 1) / kBatchColTile;
    S.transposed = nm >= kBatchTransposeMin;
    if (S.transposed) {
        // column items: K^T rows in whole warps (32), about row_tile_elems each
        int cpi = (int)std::max<int64_t>(1, tn.row_tile_elems / std::max(1, q.n));
        cpi = std::max(32, cpi / 32 * 32);
        S.cols_per_item = cpi;
        S.col_items = (q.m + cpi - 1) / cpi;
    } else {
        S.cols_per_item = kBatchColTile;
        S.col_items = S.col_tiles;
    }
    // the step's column loops as items for large tiled problems
    // (ACCSINK_BATCH_STEP_ITEMS=0 keeps them in one CTA)
    if (!S.small && q.m >= kBatchStepSplitMin && step_items_enabled()) {
        S.step_cols = kBatchStepCols;
        S.step_items = (q.m + kBatchStepCols - 1) / kBatchStepCols;
    }
    S.lay = layout(q.n, q.m, S.row_tiles, S.col_tiles, S.transposed, S.step_items);
    return S;
}

// Formation tiles of a problem: tensor-core (kBatchTcRows x kBatchTcCols)
// or CUDA-core (kBatchFormTile square), and scaling tiles.
int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

bool tc_eligible(bool tc_on, const accsink_problem &q, int64_t R)
{
    return tc_on && q.cost_kind == ACCSINK_COST_COSINE && q.d >= kBatchTcMinD &&
           q.d <= kBatchTcMaxD && R + q.n + q.m < ((int64_t)1 << 31) - kBatchTcRows;
}

// resident: the persistent CTAs of the launch (0: size the plan for any
// launch, as the workspace sizers do). A batch is wide when its tiled
// problems' row items of full_rows rows number at least twice the resident
// CTAs; its rows per item then never fall below full_rows. A wide plan has
// no more row items, hence no more bytes, than the same plan not wide.
void plan_batch(const BatchTuning &tn, int count, const accsink_problem *probs,
                const accsink_params *params, BatchPlan &pl, int resident = 0)
{
    int64_t full_items = 0;
    for (int k = 0; k < count; ++k)
        if (!is_small(tn, probs[k])) full_items += ceil_div(probs[k].n, full_rows(probs[k].m));
    const bool wide = resident > 0 && full_items >= 2 * (int64_t)resident;
    pl.hp.assign(count, BatchProb{});
    pl.lay.resize(count);
    pl.tiles.clear();
    pl.data_bytes = 0;
    size_t outstanding = 0;
    const bool tc_on = tc_form_enabled();
    std::vector<BatchTile> scale_tiles, tc_tiles;
    for (int k = 0; k < count; ++k) {
        const accsink_problem &q = probs[k];
        BatchProb &P = pl.hp[k];
        std::memset(&P, 0, sizeof(P));
        P.C = q.C; P.X = q.X; P.Y = q.Y;
        P.a_in = q.a; P.b_in = q.b;
        P.ldc = q.ldc ? q.ldc : q.m;
        P.n = q.n; P.m = q.m; P.d = q.d; P.kind = q.cost_kind;
        P.scale = q.cost_scale == ACCSINK_SCALE_MAX_TO_ONE ? 1 : 0;
        if (params) {
            const accsink_params &pp = params[k];
            P.method = pp.method; P.stability = pp.stability; P.carry = pp.carry;
            P.max_steps = pp.max_sinkhorn_steps; P.m0 = pp.m0; P.evaluate = pp.evaluate ? 1 : 0;
            P.eps = pp.eps; P.tol = stop_threshold(pp.tol); P.mu0 = pp.mu0;
        }
        P.ldm = ((int64_t)q.m + 3) / 4 * 4;
        const ProbShape S = prob_shape(tn, q, wide);
        P.small = S.small;
        P.rows_per_tile = S.rows_per_tile;
        P.row_tiles = S.row_tiles;
        P.col_tiles = S.col_tiles;
        P.ldn = ((int64_t)q.n + 3) / 4 * 4;
        P.cols_per_item = S.cols_per_item;
        P.col_items = S.col_items;
        P.cmax_enc = 0ull;             // below every encoded value
        P.cmin_enc = ~0ull;            // above every encoded value
        P.cabs_enc = 0ull;
        P.step_cols = S.step_cols;
        P.step_items = S.step_items;
        pl.lay[k] = S.lay;
        pl.data_bytes += pl.lay[k].total();
        outstanding += (size_t)std::max(P.row_tiles, P.col_items);
        P.tc = tc_eligible(tc_on, q, pl.R) ? 1 : 0;
        if (P.tc) {
            pl.tcp.push_back(k);
            pl.tcs.push_back(pl.R);
            P.tc_xoff = (int32_t)pl.R;
            P.tc_yoff = (int32_t)(pl.R + q.n);
            pl.R += (int64_t)q.n + q.m;
            pl.dpad = std::max(pl.dpad, (q.d + kBatchTcK - 1) / kBatchTcK * kBatchTcK);
            for (int r = 0; r < q.n; r += kBatchTcRows)
                for (int c = 0; c < q.m; c += kBatchTcCols) tc_tiles.push_back({k, r, c, 0});
        } else {
            for (int r = 0; r < q.n; r += kBatchFormTile)
                for (int c = 0; c < q.m; c += kBatchFormTile) pl.tiles.push_back({k, r, c, 0});
        }
        if (P.scale)
            for (int r = 0; r < q.n; r += kBatchFormTile)
                for (int c = 0; c < q.m; c += kBatchFormTile) scale_tiles.push_back({k, r, c, 0});
    }
    pl.nform = (int)pl.tiles.size();
    pl.nscale = (int)scale_tiles.size();
    pl.ntct = (int)tc_tiles.size();
    pl.tiles.insert(pl.tiles.end(), scale_tiles.begin(), scale_tiles.end());
    pl.tiles.insert(pl.tiles.end(), tc_tiles.begin(), tc_tiles.end());
    if (pl.R > 0) {
        pl.slice_bytes = up256(batch_tc_slice_bytes(pl.R, pl.dpad));
        pl.expo_bytes = up256((size_t)pl.R * 4);
        pl.data_bytes += pl.slice_bytes + pl.expo_bytes;
    }
    const size_t ntc = pl.tcp.size();
    pl.cap = pow2_at_least(std::max<unsigned long long>(
        4096, 2 * (unsigned long long)(outstanding + count)));
    pl.head_bytes = up256(sizeof(BatchProb) * count) + up256(sizeof(BatchResult) * count) +
                    up256(sizeof(BatchQueue)) + up256(pl.cap * 8) + up256(pl.cap * 8) +
                    up256(sizeof(BatchTile) * pl.tiles.size()) + up256(8 * (size_t)count) +
                    up256(4 * ntc) + up256(8 * ntc);
}

}  // namespace

// The public result of one problem of a batched launch.
void to_result(const BatchResult &r, float ms, accsink_result &o)
{
    std::memset(&o, 0, sizeof(o));
    o.status = r.status;
    o.sinkhorn_steps = r.steps;
    o.outer_stages = r.stages;
    o.stability_failures = r.failures;
    o.marginal_l1 = r.marginal_l1;
    o.transport_cost = r.transport_cost;
    o.dual_objective = r.dual;
    o.cost_max = r.cost_max;
    o.gpu_ms = ms;
    o.loop_mode = 2;
}

size_t batch_workspace_bytes(const BatchTuning &tn, int count, const accsink_problem *probs)
{
    BatchSizer sz(tn);
    for (int k = 0; k < count; ++k) sz.add(probs[k]);
    return sz.bytes();
}

BatchSizer::BatchSizer(const BatchTuning &tn) : tn_(tn), tc_on_(tc_form_enabled()) {}

void BatchSizer::add(const accsink_problem &q)
{
    const ProbShape S = prob_shape(tn_, q);
    data_ += S.lay.total();
    outstanding_ += (size_t)std::max(S.row_tiles, S.col_items);
    if (tc_eligible(tc_on_, q, R_)) {
        R_ += (int64_t)q.n + q.m;
        dpad_ = std::max(dpad_, (q.d + kBatchTcK - 1) / kBatchTcK * kBatchTcK);
        tiles_ += ceil_div(q.n, kBatchTcRows) * ceil_div(q.m, kBatchTcCols);
        ++ntc_;
    } else {
        tiles_ += ceil_div(q.n, kBatchFormTile) * ceil_div(q.m, kBatchFormTile);
    }
    if (q.cost_scale == ACCSINK_SCALE_MAX_TO_ONE)
        tiles_ += ceil_div(q.n, kBatchFormTile) * ceil_div(q.m, kBatchFormTile);
    ++count_;
}

size_t BatchSizer::bytes() const
{
    size_t data = data_;
    if (R_ > 0) data += up256(batch_tc_slice_bytes(R_, dpad_)) + up256((size_t)R_ * 4);
    const unsigned long long cap = pow2_at_least(std::max<unsigned long long>(
        4096, 2 * (unsigned long long)(outstanding_ + count_)));
    const size_t head = up256(sizeof(BatchProb) * count_) + up256(sizeof(BatchResult) * count_) +
                        up256(sizeof(BatchQueue)) + up256(cap * 8) + up256(cap * 8) +
                        up256(sizeof(BatchTile) * (size_t)tiles_) + up256(8 * (size_t)count_) +
                        up256(4 * (size_t)ntc_) + up256(8 * (size_t)ntc_);
    return head + data;
}

size_t batch_workspace_bytes_planned(const BatchTuning &tn, int count,
                                     const accsink_problem *probs)
{
    BatchPlan pl;
    plan_batch(tn, count, probs, nullptr, pl);
    return pl.head_bytes + pl.data_bytes;
}

int batch_run(const BatchEnv &env, BatchWorkspace &ws, const BatchTuning &tn, int count,
              const accsink_problem *probs, const accsink_params *params, double *const *f_out,
              double *const *g_out, accsink_result *res, cudaStream_t s, std::string &err,
              BatchTiming *timing)
{
    // ---- plan
    const int per_sm = tn.ctas_per_sm > 0 ? std::min(tn.ctas_per_sm, env.occ_solve) : env.occ_solve;
    const int grid = std::max(1, env.num_sms * per_sm);
    BatchPlan pl;
    plan_batch(tn, count, probs, params, pl, grid);
    std::vector<BatchProb> &hp = pl.hp;
    const std::vector<ProbLayout> &lay = pl.lay;
    const std::vector<BatchTile> &tiles = pl.tiles;
    const unsigned long long cap = pl.cap;
    for (int k = 0; k < count; ++k) {
        hp[k].f_out = f_out[k];
        hp[k].g_out = g_out[k];
    }
    const size_t need = pl.head_bytes + pl.data_bytes;
    if (need > ws.bytes) {
        if (env.budget_left && need > env.budget_left) {
            err = "batch workspace of " + std::to_string(need) + " bytes exceeds the budget";
            return ACCSINK_ERR_BUDGET;
        }
        if (ws.dev) cudaFree(ws.dev);
        ws.dev = nullptr;
        ws.bytes = 0;
        if (cudaMalloc(&ws.dev, need) != cudaSuccess) {
            cudaGetLastError();
            err = "cudaMalloc of the batch workspace failed";
            return ACCSINK_ERR_OOM;
        }
        ws.bytes = need;
    }
    // ---- carve
    char *p = (char *)ws.dev;
    BatchProb *dP = (BatchProb *)p;        p += up256(sizeof(BatchProb) * count);
    BatchResult *dR = (BatchResult *)p;    p += up256(sizeof(BatchResult) * count);
    BatchQueue *dQ = (BatchQueue *)p;      p += up256(sizeof(BatchQueue));
    unsigned long long *dItems = (unsigned long long *)p;  p += up256(cap * 8);
    unsigned long long *dSeq = (unsigned long long *)p;    p += up256(cap * 8);
    BatchTile *dT = (BatchTile *)p;        p += up256(sizeof(BatchTile) * tiles.size());
    unsigned long long *dInit = (unsigned long long *)p;   p += up256(8 * (size_t)count);
    const size_t ntc = pl.tcp.size();
    int32_t *dTcp = (int32_t *)p;          p += up256(4 * ntc);
    int64_t *dTcs = (int64_t *)p;          p += up256(8 * ntc);
    for (int k = 0; k < count; ++k) {
        BatchProb &P = hp[k];
        const ProbLayout &L = lay[k];
        auto take = [&](size_t b) { char *r = p; p += b; return r; };
        P.Kh = (float *)take(L.kh); P.Kl = (float *)take(L.kl);
        if (L.kth) { P.KTh = (float *)take(L.kth); P.KTl = (float *)take(L.ktl); }
        else { P.KTh = nullptr; P.KTl = nullptr; }
        P.a = (double *)take(L.a); P.loga = (double *)take(L.loga); P.u = (double *)take(L.u);
        P.Fh = (float *)take(L.fh); P.Fl = (float *)take(L.fl);
        double **mv[12] = {&P.b, &P.logb, &P.x, &P.x_prev, &P.w, &P.w1, &P.p_prev, &P.D_prev,
                           &P.raw, &P.D1, &P.del, &P.ell};
        for (double **v : mv) *v = (double *)take(L.mvec);
        P.Gh = (float *)take(L.gh); P.Gl = (float *)take(L.gl);
        P.rowpart = (double *)take(L.rowpart);
        P.colrec = (double *)take(L.colrec);
        P.p2rec = L.p2rec ? (double *)take(L.p2rec) : nullptr;
    }
    BatchTcLaunch tcl{};
    if (pl.R > 0) {
        tcl.tiles = dT + pl.nform + pl.nscale;
        tcl.ntiles = pl.ntct;
        tcl.tcp = dTcp;
        tcl.tcs = dTcs;
        tcl.ntc = (int)ntc;
        tcl.dpad = pl.dpad;
        tcl.R = pl.R;
        tcl.SL = p;                         p += pl.slice_bytes;
        tcl.expo = (int32_t *)p;            p += pl.expo_bytes;
    }
    // initial items, largest problems first
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (int64_t)hp[x].n * hp[x].m > (int64_t)hp[y].n * hp[y].m;
    });
    std::vector<unsigned long long> init(count);
    for (int i = 0; i < count; ++i) {
        const int k = order[i];
        init[i] = batch_item(hp[k].small ? BI_SMALL : BI_INIT, k, 0);
    }
    BatchQueue hq;
    std::memset(&hq, 0, sizeof(hq));
    hq.head = 0;
    hq.tail = (unsigned long long)count;
    hq.items = dItems;
    hq.seq = dSeq;
    hq.cap = cap;
    hq.count = count;
    hq.early = env.on_done ? env.early_dev : nullptr;
    hq.early_flag = env.on_done ? env.flag_dev : nullptr;
    // ---- stage the host records (pinned) and launch
    const size_t hbytes = up256(sizeof(BatchProb) * count) + up256(sizeof(BatchTile) * tiles.size()) +
                          up256(8 * (size_t)count) + up256(sizeof(BatchQueue)) +
                          up256(sizeof(BatchResult) * count) + up256(4 * ntc) + up256(8 * ntc);
    if (hbytes > ws.host_bytes) {
        if (ws.host) cudaFreeHost(ws.host);
        ws.host = nullptr;
        ws.host_bytes = 0;
        if (cudaMallocHost(&ws.host, hbytes) != cudaSuccess) {
            cudaGetLastError();
            err = "cudaMallocHost of the batch staging failed";
            return ACCSINK_ERR_OOM;
        }
        ws.host_bytes = hbytes;
    }
    char *h = (char *)ws.host;
    BatchProb *hP = (BatchProb *)h;        h += up256(sizeof(BatchProb) * count);
    BatchTile *hT = (BatchTile *)h;        h += up256(sizeof(BatchTile) * tiles.size());
    unsigned long long *hI = (unsigned long long *)h;  h += up256(8 * (size_t)count);
    BatchQueue *hQ = (BatchQueue *)h;      h += up256(sizeof(BatchQueue));
    BatchResult *hR = (BatchResult *)h;    h += up256(sizeof(BatchResult) * count);
    int32_t *hTcp = (int32_t *)h;          h += up256(4 * ntc);
    int64_t *hTcs = (int64_t *)h;
    if (ntc) {
        std::memcpy(hTcp, pl.tcp.data(), 4 * ntc);
        std::memcpy(hTcs, pl.tcs.data(), 8 * ntc);
    }
    std::memcpy(hP, hp.data(), sizeof(BatchProb) * count);
    if (!tiles.empty()) std::memcpy(hT, tiles.data(), sizeof(BatchTile) * tiles.size());
    std::memcpy(hI, init.data(), 8 * (size_t)count);
    std::memcpy(hQ, &hq, sizeof(hq));

#define BK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);   \
            return ACCSINK_ERR_CUDA;                                    \
        }                                                               \
    } while (0)

    if (pl.R > 0) BK(prepare_batch_form_tc(&tcl.sms));
    // The launch sequence of the batch: record upload, cost formation, queue
    // set-up, the persistent solve and the result download. It is captured
    // into a CUDA graph on the workspace's own stream and replayed on s as one
    // launch (the previous batch's executable graph is updated in place when
    // the sequence has the same shape); ACCSINK_BATCH_GRAPH=0 issues it
    // directly on s.
    const bool graph = batch_graph_enabled();
    if (graph && !ws.cap) BK(cudaStreamCreateWithFlags(&ws.cap, cudaStreamNonBlocking));
    cudaStream_t cs = graph ? ws.cap : s;
    const char *failed = nullptr;
    auto sequence = [&]() -> cudaError_t {
        cudaError_t e;
#define SQ(call)                                   \
    do {                                           \
        e = (call);                                \
        if (e != cudaSuccess) { failed = #call; return e; } \
    } while (0)
        auto rec = [&](cudaEvent_t ev) {
            return graph ? cudaEventRecordWithFlags(ev, cs, cudaEventRecordExternal)
                         : cudaEventRecord(ev, cs);
        };
        SQ(rec(env.ev0));
        SQ(cudaMemcpyAsync(dP, hP, sizeof(BatchProb) * count, cudaMemcpyHostToDevice, cs));
        if (!tiles.empty())
            SQ(cudaMemcpyAsync(dT, hT, sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice, cs));
        SQ(cudaMemcpyAsync(dInit, hI, 8 * (size_t)count, cudaMemcpyHostToDevice, cs));
        SQ(cudaMemcpyAsync(dQ, hQ, sizeof(BatchQueue), cudaMemcpyHostToDevice, cs));
        if (ntc) {
            SQ(cudaMemcpyAsync(dTcp, hTcp, 4 * ntc, cudaMemcpyHostToDevice, cs));
            SQ(cudaMemcpyAsync(dTcs, hTcs, 8 * ntc, cudaMemcpyHostToDevice, cs));
        }
        SQ(launch_batch_form(dP, dT, pl.nform, 0, cs));
        if (pl.R > 0) SQ(launch_batch_form_tc(dP, tcl, cs));
        SQ(launch_batch_scale(dP, dT + pl.nform, pl.nscale, cs));
        SQ(launch_queue_init(dQ, dInit, count, cap, cs));
        SQ(rec(env.ev_mid));
        SQ(launch_batch_solve(dP, dQ, dR, grid, cs));
        SQ(rec(env.ev1));
        SQ(cudaMemcpyAsync(hR, dR, sizeof(BatchResult) * count, cudaMemcpyDeviceToHost, cs));
        SQ(cudaMemcpyAsync(hQ, dQ, sizeof(BatchQueue), cudaMemcpyDeviceToHost, cs));
#undef SQ
        return cudaSuccess;
    };
    if (!graph) {
        const cudaError_t e = sequence();
        if (e != cudaSuccess) {
            err = std::string(failed) + ": " + cudaGetErrorString(e);
            return ACCSINK_ERR_CUDA;
        }
    } else {
        BK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const cudaError_t e = sequence();
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            err = e != cudaSuccess ? std::string(failed) + " (captured): " + cudaGetErrorString(e)
                                   : std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ec);
            return ACCSINK_ERR_CUDA;
        }
        bool updated = false;
        if (ws.exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(ws.exec, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(ws.exec);
                ws.exec = nullptr;
            }
        }
        cudaError_t ei = cudaSuccess;
        if (!updated) ei = cudaGraphInstantiate(&ws.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            ws.exec = nullptr;
            err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
            return ACCSINK_ERR_CUDA;
        }
        BK(cudaGraphLaunch(ws.exec, s));
    }
    if (env.on_done && env.early_host && env.flag_host) {
        // hand back each problem as soon as the kernel has finished it
        std::vector<char> seen(count, 0);
        int left = count;
        for (;;) {
            const bool finished = cudaStreamQuery(s) != cudaErrorNotReady;
            for (int k = 0; k < count && left > 0; ++k) {
                if (seen[k] || *(volatile int32_t *)&env.flag_host[k] == 0) continue;
                std::atomic_thread_fence(std::memory_order_acquire);
                accsink_result o;
                to_result(env.early_host[k], 0.0f, o);
                seen[k] = 1;
                --left;
                env.on_done(k, o);
            }
            if (finished || left == 0) break;
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    BK(cudaStreamSynchronize(s));
    float ms_all = 0.0f, ms_form = 0.0f;
    cudaEventElapsedTime(&ms_all, env.ev0, env.ev1);
    cudaEventElapsedTime(&ms_form, env.ev0, env.ev_mid);
    if (timing) {
        timing->total_ms = ms_all;
        timing->form_ms = ms_form;
        timing->solve_ms = ms_all - ms_form;
        timing->grid = grid;
    }
#undef BK
    if (hQ->error) {
        err = "a batch queue wait ran out of time";
        for (int k = 0; k < count; ++k) {
            std::memset(&res[k], 0, sizeof(res[k]));
            res[k].status = ACCSINK_ERR_TIMEOUT;
        }
        return ACCSINK_ERR_TIMEOUT;
    }
    int rc = ACCSINK_OK;
    for (int k = 0; k < count; ++k) {
        const BatchResult &r = hR[k];
        accsink_result &o = res[k];
        to_result(r, ms_all, o);
        if (r.status != ACCSINK_OK) {
            if (rc == ACCSINK_OK || (rc == ACCSINK_ERR_MAXITER && r.status != ACCSINK_ERR_MAXITER))
                rc = r.status;
        }
    }
    if (rc == ACCSINK_ERR_MAXITER) err = "some problems did not converge within max_sinkhorn_steps";
    else if (rc != ACCSINK_OK) err = "some problems stopped with an error status (see res[k].status)";
    return rc;
}

}  // namespace accsink

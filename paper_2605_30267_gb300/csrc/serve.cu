// Request server: a native loop that admits submitted solves by a device-
// memory budget and runs each admitted group through the batched solver,
// keeping every solve's potentials resident on the device until the client
// releases its ticket.
//
// Threads: client calls (submit, poll, wait, release, ...) take the server
// mutex; one worker thread owns the CUDA stream, the batch workspace and all
// device allocations. A request moves QUEUED -> RUNNING -> DONE (or FAILED)
// -> released. Admission is FIFO: the worker takes queued requests in order
// while inputs, outputs and the batch workspace fit in the budget next to the
// potentials that are still held, and while the group's cost entries stay
// within its limit; a request that cannot fit even alone fails with
// ACCSINK_ERR_BUDGET.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "accsink.h"
#include "accsink_internal.cuh"
#include "batch_host.h"
#include "batch_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    accsink_problem prob{};       // host pointers as submitted
    accsink_params params{};
    int32_t state = ACCSINK_REQ_QUEUED;
    accsink_result res{};
    double *f_dev = nullptr, *g_dev = nullptr;   // resident outputs
    size_t out_bytes = 0;
    Clock::time_point t_submit, t_start, t_done;
};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

size_t input_bytes(const accsink_problem &p)
{
    size_t b = up256((size_t)p.n * 8) + up256((size_t)p.m * 8);
    if (p.cost_kind == ACCSINK_COST_DENSE)
        b += up256((size_t)p.n * (size_t)(p.ldc ? p.ldc : p.m) * 4);
    else
        b += up256((size_t)p.n * p.d * 4) + up256((size_t)p.m * p.d * 4);
    return b;
}

size_t output_bytes(const accsink_problem &p)
{
    return up256((size_t)p.n * 8) + up256((size_t)p.m * 8);
}

// Default admission limit of a group, in cost entries: none. Measured on the
// serving workload at 2000 offered requests/s (15-s windows), the sustained
// rate fell with smaller limits (2^27: 160/s, 2^28: 194/s, 2^29: 254/s,
// none: 306/s), since a large group keeps every SM busy with many problems
// while its slowest ones finish; a limit only shortens the wait of requests
// queued behind a running group.
constexpr int64_t kDefaultGroupEntries = 0;

}  // namespace

struct accsink_server {
    int device = 0;
    size_t budget = 0;
    int num_sms = 1, occ = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread worker;
    // owned by the worker thread
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev_mid = nullptr, ev1 = nullptr;
    accsink::BatchWorkspace ws;
    accsink::BatchTuning tuning;
    cudaMemPool_t pool = nullptr;   // server-owned pool for inputs and outputs
    // host-mapped result records and done flags of the running batch, so a
    // request finishes when its own problem does, not when the whole batch
    // does (capacity in problems; grown by the worker)
    accsink::BatchResult *early = nullptr;
    int32_t *early_flag = nullptr;
    int early_cap = 0;
    // admission limit: cost entries (sum of n m) of one admitted group; a
    // request larger than the limit still runs, alone (0: no limit)
    int64_t max_group_entries = kDefaultGroupEntries;
    // accounting (under mu)
    size_t resident = 0;          // outputs held for DONE tickets
    size_t peak_in_use = 0;
    int64_t batches = 0, solved = 0, failed = 0;
    double busy_ms = 0.0;
    std::string err;
};

namespace {

void worker_loop(accsink_server *S)
{
    cudaSetDevice(S->device);
    std::vector<uint64_t> group;
    std::vector<accsink_problem> probs;
    std::vector<accsink_params> params;
    std::vector<double *> fo, go;
    std::vector<accsink_result> res;
    std::vector<void *> inputs;
    for (;;) {
        group.clear();
        size_t in_total = 0, out_total = 0;
        accsink::BatchTuning tuning;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            tuning = S->tuning;
            S->cv_work.wait(lk, [&] { return S->stopping || !S->queue.empty(); });
            if (S->stopping && S->queue.empty()) return;
            // FIFO admission against the budget and the group limit; the
            // group's batch workspace grows by one request at a time (O(1)
            // per request, no re-planning of the group)
            accsink::BatchSizer sizer(tuning);
            int64_t entries = 0;
            while (!S->queue.empty()) {
                const uint64_t t = S->queue.front();
                Request &r = S->reqs[t];
                const int64_t nm = (int64_t)r.prob.n * r.prob.m;
                if (!group.empty() && S->max_group_entries > 0 &&
                    entries + nm > S->max_group_entries)
                    break;
                accsink::BatchSizer next = sizer;
                next.add(r.prob);
                const size_t ws_need = next.bytes();
                const size_t in_b = input_bytes(r.prob), out_b = output_bytes(r.prob);
                const size_t total = S->resident + in_total + out_total + in_b + out_b + ws_need;
                if (total > S->budget) {
                    if (group.empty()) {
                        // cannot run even alone next to the held potentials
                        accsink::BatchSizer one(tuning);
                        one.add(r.prob);
                        const size_t alone = in_b + out_b + one.bytes();
                        if (alone > S->budget) {
                            r.state = ACCSINK_REQ_FAILED;
                            r.res.status = ACCSINK_ERR_BUDGET;
                            r.t_done = Clock::now();
                            S->queue.pop_front();
                            ++S->failed;
                            S->cv_done.notify_all();
                            continue;
                        }
                        // wait for releases, then try again
                        S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                    }
                    break;
                }
                sizer = next;
                entries += nm;
                in_total += in_b;
                out_total += out_b;
                group.push_back(t);
                S->queue.pop_front();
                r.state = ACCSINK_REQ_RUNNING;
                r.t_start = Clock::now();
            }
            if (group.empty()) continue;
            S->peak_in_use = std::max(S->peak_in_use,
                                      S->resident + in_total + out_total + sizer.bytes());
        }
        // ---- stage inputs, allocate outputs (stream-ordered)
        const int k = (int)group.size();
        probs.assign(k, accsink_problem{});
        params.assign(k, accsink_params{});
        fo.assign(k, nullptr);
        go.assign(k, nullptr);
        res.assign(k, accsink_result{});
        inputs.clear();
        bool cuda_ok = true;
        std::string cerr;
        auto alloc = [&](size_t bytes) -> void * {
            void *p = nullptr;
            if (cudaMallocFromPoolAsync(&p, bytes, S->pool, S->stream) != cudaSuccess) {
                cudaGetLastError();
                cuda_ok = false;
                cerr = "cudaMallocAsync failed";
                return nullptr;
            }
            return p;
        };
        for (int i = 0; i < k; ++i) {
            accsink_problem hp;
            accsink_params pp;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                hp = S->reqs[group[i]].prob;
                pp = S->reqs[group[i]].params;
            }
            accsink_problem dp = hp;
            const int64_t ldc = hp.ldc ? hp.ldc : hp.m;
            if (hp.cost_kind == ACCSINK_COST_DENSE) {
                float *C = (float *)alloc((size_t)hp.n * ldc * 4);
                if (C) cudaMemcpyAsync(C, hp.C, (size_t)hp.n * ldc * 4, cudaMemcpyHostToDevice, S->stream);
                inputs.push_back(C);
                dp.C = C;
                dp.ldc = ldc;
            } else {
                float *X = (float *)alloc((size_t)hp.n * hp.d * 4);
                float *Y = (float *)alloc((size_t)hp.m * hp.d * 4);
                if (X) cudaMemcpyAsync(X, hp.X, (size_t)hp.n * hp.d * 4, cudaMemcpyHostToDevice, S->stream);
                if (Y) cudaMemcpyAsync(Y, hp.Y, (size_t)hp.m * hp.d * 4, cudaMemcpyHostToDevice, S->stream);
                inputs.push_back(X);
                inputs.push_back(Y);
                dp.X = X;
                dp.Y = Y;
            }
            double *a = (double *)alloc((size_t)hp.n * 8), *b = (double *)alloc((size_t)hp.m * 8);
            if (a) cudaMemcpyAsync(a, hp.a, (size_t)hp.n * 8, cudaMemcpyHostToDevice, S->stream);
            if (b) cudaMemcpyAsync(b, hp.b, (size_t)hp.m * 8, cudaMemcpyHostToDevice, S->stream);
            inputs.push_back(a);
            inputs.push_back(b);
            dp.a = a;
            dp.b = b;
            fo[i] = (double *)alloc((size_t)hp.n * 8);
            go[i] = (double *)alloc((size_t)hp.m * 8);
            probs[i] = dp;
            params[i] = pp;
        }
        int rc = ACCSINK_ERR_CUDA;
        std::string berr = cerr;
        accsink::BatchTiming tm;
        if (cuda_ok && k > S->early_cap) {
            const int cap = std::max(k, 2 * S->early_cap);
            if (S->early) cudaFreeHost(S->early);
            if (S->early_flag) cudaFreeHost(S->early_flag);
            S->early = nullptr;
            S->early_flag = nullptr;
            S->early_cap = 0;
            if (cudaHostAlloc((void **)&S->early, sizeof(accsink::BatchResult) * cap,
                              cudaHostAllocMapped) == cudaSuccess &&
                cudaHostAlloc((void **)&S->early_flag, sizeof(int32_t) * cap,
                              cudaHostAllocMapped) == cudaSuccess) {
                S->early_cap = cap;
            } else {
                cudaGetLastError();   // no early completion; the batch still runs
            }
        }
        if (cuda_ok) {
            accsink::BatchEnv env;
            env.num_sms = S->num_sms;
            env.occ_solve = S->occ;
            env.budget_left = 0;
            env.ev0 = S->ev0;
            env.ev_mid = S->ev_mid;
            env.ev1 = S->ev1;
            if (S->early_cap >= k) {
                std::memset(S->early_flag, 0, sizeof(int32_t) * k);
                env.early_host = S->early;
                env.flag_host = S->early_flag;
                if (cudaHostGetDevicePointer((void **)&env.early_dev, S->early, 0) != cudaSuccess ||
                    cudaHostGetDevicePointer((void **)&env.flag_dev, S->early_flag, 0) !=
                        cudaSuccess) {
                    cudaGetLastError();
                    env.early_host = nullptr;
                    env.flag_host = nullptr;
                } else {
                    // a converged (or step-limited) problem is DONE at once;
                    // anything else is settled with the batch below
                    env.on_done = [&](int i, const accsink_result &r) {
                        if (r.status != ACCSINK_OK && r.status != ACCSINK_ERR_MAXITER) return;
                        {
                            std::lock_guard<std::mutex> lk(S->mu);
                            auto it = S->reqs.find(group[i]);
                            if (it == S->reqs.end()) return;
                            Request &q = it->second;
                            q.t_done = Clock::now();
                            q.res = r;
                            q.f_dev = fo[i];
                            q.g_dev = go[i];
                            q.out_bytes = output_bytes(q.prob);
                            S->resident += q.out_bytes;
                            q.state = ACCSINK_REQ_DONE;
                            ++S->solved;
                        }
                        S->cv_done.notify_all();
                    };
                }
            }
            rc = accsink::batch_run(env, S->ws, tuning, k, probs.data(), params.data(),
                                    fo.data(), go.data(), res.data(), S->stream, berr, &tm);
        }
        for (void *p : inputs)
            if (p) cudaFreeAsync(p, S->stream);
        cudaStreamSynchronize(S->stream);
        const Clock::time_point now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            ++S->batches;
            S->busy_ms += tm.total_ms;
            // the engine ran when it returned OK or a per-problem status
            const bool ran = cuda_ok && (rc == ACCSINK_OK || rc == ACCSINK_ERR_MAXITER ||
                                         rc == ACCSINK_ERR_NONFINITE ||
                                         rc == ACCSINK_ERR_NONPOSITIVE_MARGINAL ||
                                         rc == ACCSINK_ERR_INVALID_ARG);
            for (int i = 0; i < k; ++i) {
                // a ticket handed back early may already be released
                auto it = S->reqs.find(group[i]);
                if (it == S->reqs.end()) continue;
                Request &r = it->second;
                if (r.state == ACCSINK_REQ_DONE) {
                    r.res.gpu_ms = res[i].gpu_ms;   // handed back early; batch time only
                    continue;
                }
                r.t_done = now;
                if (ran && (res[i].status == ACCSINK_OK || res[i].status == ACCSINK_ERR_MAXITER)) {
                    r.res = res[i];
                    r.f_dev = fo[i];
                    r.g_dev = go[i];
                    r.out_bytes = output_bytes(r.prob);
                    S->resident += r.out_bytes;
                    r.state = ACCSINK_REQ_DONE;
                    ++S->solved;
                } else {
                    r.res = ran ? res[i] : accsink_result{};
                    if (!ran) r.res.status = rc == ACCSINK_OK ? ACCSINK_ERR_CUDA : rc;
                    r.state = ACCSINK_REQ_FAILED;
                    if (fo[i]) cudaFreeAsync(fo[i], S->stream);
                    if (go[i]) cudaFreeAsync(go[i], S->stream);
                    ++S->failed;
                    if (!ran) S->err = berr;
                }
            }
        }
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int accsink_server_create(int device, size_t mem_budget_bytes, accsink_server **out)
{
    if (!out) return ACCSINK_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return ACCSINK_ERR_INVALID_ARG;
    }
    if (mem_budget_bytes == 0) return ACCSINK_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return ACCSINK_ERR_CUDA;
    accsink_server *S = new accsink_server();
    S->device = device;
    S->budget = mem_budget_bytes;
    cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, device);
    S->occ = accsink::occupancy_batch_solve();
    S->tuning = accsink::batch_default_tuning(S->num_sms);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return ACCSINK_ERR_CUDA;
    }
    // keep freed blocks in the pool (no return to the driver between batches)
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&S->ev0) != cudaSuccess || cudaEventCreate(&S->ev_mid) != cudaSuccess ||
        cudaEventCreate(&S->ev1) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return ACCSINK_ERR_CUDA;
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return ACCSINK_OK;
}

void accsink_server_destroy(accsink_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        // queued requests are dropped
        for (uint64_t t : S->queue) {
            Request &r = S->reqs[t];
            r.state = ACCSINK_REQ_FAILED;
            r.res.status = ACCSINK_ERR_INVALID_ARG;
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (auto &kv : S->reqs) {
        if (kv.second.f_dev) cudaFreeAsync(kv.second.f_dev, S->stream);
        if (kv.second.g_dev) cudaFreeAsync(kv.second.g_dev, S->stream);
    }
    cudaStreamSynchronize(S->stream);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    accsink::batch_workspace_free(S->ws);
    if (S->early) cudaFreeHost(S->early);
    if (S->early_flag) cudaFreeHost(S->early_flag);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->ev0) cudaEventDestroy(S->ev0);
    if (S->ev_mid) cudaEventDestroy(S->ev_mid);
    if (S->ev1) cudaEventDestroy(S->ev1);
    delete S;
}

const char *accsink_server_last_error(accsink_server *S)
{
    if (!S) return "NULL server";
    std::lock_guard<std::mutex> lk(S->mu);
    return S->err.c_str();
}

int accsink_server_submit(accsink_server *S, const accsink_problem *prob_host,
                          const accsink_params *params, accsink_ticket *ticket)
{
    if (!S || !prob_host || !params || !ticket) return ACCSINK_ERR_INVALID_ARG;
    const accsink_problem &p = *prob_host;
    if (p.n < 1 || p.m < 1 || !p.a || !p.b) return ACCSINK_ERR_INVALID_ARG;
    if (p.cost_kind == ACCSINK_COST_DENSE) {
        if (!p.C || (p.ldc && p.ldc < p.m)) return ACCSINK_ERR_INVALID_ARG;
    } else if (p.cost_kind == ACCSINK_COST_SQEUCLID || p.cost_kind == ACCSINK_COST_COSINE) {
        if (!p.X || !p.Y || p.d < 1 || p.d > 4096) return ACCSINK_ERR_INVALID_ARG;
    } else {
        return ACCSINK_ERR_INVALID_ARG;
    }
    if (p.cost_scale != ACCSINK_SCALE_NONE && p.cost_scale != ACCSINK_SCALE_MAX_TO_ONE)
        return ACCSINK_ERR_INVALID_ARG;
    const accsink_params &q = *params;
    if (!(q.eps > 0.0) || !(q.tol > 0.0) || q.max_sinkhorn_steps < 1 ||
        (q.method != ACCSINK_PLAIN && q.method != ACCSINK_ACC) ||
        (q.method == ACCSINK_ACC && (!(q.mu0 > 0.0 && q.mu0 < 1.0) || q.m0 < 1)) ||
        q.stability < 0 || q.stability > 3 ||
        (q.carry != ACCSINK_CARRY_Y && q.carry != ACCSINK_CARRY_W) ||
        q.precision < ACCSINK_PRECISION_AUTO || q.precision > ACCSINK_PRECISION_DF32)
        return ACCSINK_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) return ACCSINK_ERR_INVALID_ARG;
        const uint64_t t = S->next_ticket++;
        Request &r = S->reqs[t];
        r.prob = p;
        r.params = q;
        r.t_submit = Clock::now();
        S->queue.push_back(t);
        *ticket = t;
    }
    S->cv_work.notify_one();
    return ACCSINK_OK;
}

int accsink_server_poll(accsink_server *S, accsink_ticket t, int32_t *state)
{
    if (!S || !state) return ACCSINK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(t);
    if (it == S->reqs.end()) return ACCSINK_ERR_INVALID_ARG;
    *state = it->second.state;
    return ACCSINK_OK;
}

int accsink_server_wait(accsink_server *S, accsink_ticket t, int32_t timeout_ms,
                        accsink_result *res, double *latency_ms)
{
    if (!S) return ACCSINK_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(t);
    if (it == S->reqs.end()) return ACCSINK_ERR_INVALID_ARG;
    auto finished = [&] {
        const int st = S->reqs[t].state;
        return st == ACCSINK_REQ_DONE || st == ACCSINK_REQ_FAILED;
    };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, finished);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
        return ACCSINK_ERR_TIMEOUT;
    }
    Request &r = S->reqs[t];
    if (res) *res = r.res;
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    return r.state == ACCSINK_REQ_DONE ? r.res.status : r.res.status ? r.res.status : ACCSINK_ERR_CUDA;
}

int accsink_server_potentials(accsink_server *S, accsink_ticket t, const double **f_dev,
                              const double **g_dev)
{
    if (!S) return ACCSINK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(t);
    if (it == S->reqs.end() || it->second.state != ACCSINK_REQ_DONE) return ACCSINK_ERR_INVALID_ARG;
    if (f_dev) *f_dev = it->second.f_dev;
    if (g_dev) *g_dev = it->second.g_dev;
    return ACCSINK_OK;
}

int accsink_server_copy_potentials(accsink_server *S, accsink_ticket t, double *f_host,
                                   double *g_host)
{
    if (!S) return ACCSINK_ERR_INVALID_ARG;
    const double *f = nullptr, *g = nullptr;
    int n = 0, m = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(t);
        if (it == S->reqs.end() || it->second.state != ACCSINK_REQ_DONE)
            return ACCSINK_ERR_INVALID_ARG;
        f = it->second.f_dev;
        g = it->second.g_dev;
        n = it->second.prob.n;
        m = it->second.prob.m;
    }
    // the ticket stays DONE until released by this client, so f and g stay valid
    cudaSetDevice(S->device);
    if (f_host && cudaMemcpy(f_host, f, (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ACCSINK_ERR_CUDA;
    if (g_host && cudaMemcpy(g_host, g, (size_t)m * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ACCSINK_ERR_CUDA;
    return ACCSINK_OK;
}

int accsink_server_release(accsink_server *S, accsink_ticket t)
{
    if (!S) return ACCSINK_ERR_INVALID_ARG;
    double *f = nullptr, *g = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(t);
        if (it == S->reqs.end()) return ACCSINK_ERR_INVALID_ARG;
        const int st = it->second.state;
        if (st != ACCSINK_REQ_DONE && st != ACCSINK_REQ_FAILED) return ACCSINK_ERR_INVALID_ARG;
        f = it->second.f_dev;
        g = it->second.g_dev;
        S->resident -= it->second.out_bytes;
        S->reqs.erase(it);
    }
    cudaSetDevice(S->device);
    if (f) cudaFreeAsync(f, S->stream);
    if (g) cudaFreeAsync(g, S->stream);
    S->cv_work.notify_one();
    return ACCSINK_OK;
}

int accsink_server_get_stats(accsink_server *S, accsink_server_stats *out)
{
    if (!S || !out) return ACCSINK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->queued = (int64_t)S->queue.size();
    out->solved = S->solved;
    out->failed = S->failed;
    out->batches = S->batches;
    out->resident_bytes = (int64_t)S->resident;
    out->peak_bytes = (int64_t)S->peak_in_use;
    out->budget_bytes = (int64_t)S->budget;
    out->busy_ms = S->busy_ms;
    return ACCSINK_OK;
}

int accsink_server_set_limits(accsink_server *S, int64_t max_group_entries)
{
    if (!S || max_group_entries < 0) return ACCSINK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->max_group_entries = max_group_entries;
    return ACCSINK_OK;
}

int accsink_server_set_config(accsink_server *S, const accsink_batch_config *cfg)
{
    if (!S) return ACCSINK_ERR_INVALID_ARG;
    accsink::BatchTuning t = accsink::batch_default_tuning(S->num_sms);
    if (cfg) {
        if (cfg->small_max_nm < 0 || cfg->row_tile_elems < 0 || cfg->ctas_per_sm < 0)
            return ACCSINK_ERR_INVALID_ARG;
        if (cfg->small_max_nm) t.small_max_nm = cfg->small_max_nm;
        if (cfg->row_tile_elems) t.row_tile_elems = cfg->row_tile_elems;
        t.ctas_per_sm = cfg->ctas_per_sm;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->tuning = t;
    return ACCSINK_OK;
}

}  // extern "C"

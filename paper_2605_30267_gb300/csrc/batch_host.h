// Host-side interface of the batched solver (used by the C-ABI layer).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>

#include "accsink.h"

namespace accsink {

// Device workspace of a context's batches (grow-only) and its pinned staging.
// Device and pinned host workspace of batched launches, and the CUDA graph
// their launch sequence is replayed from (captured on `cap`).
struct BatchWorkspace {
    void *dev = nullptr;
    size_t bytes = 0;
    void *host = nullptr;
    size_t host_bytes = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Frees everything a BatchWorkspace holds.
void batch_workspace_free(BatchWorkspace &ws);

// Work split of a batch. small_max_nm: problems with n m at most this are
// solved whole by one CTA; row_tile_elems: cost entries per row-pass item of
// the larger ones; ctas_per_sm: persistent CTAs per SM (0: occupancy);
// dense_solo_min_nm: dense problems with n m at least this (and a batch's
// only problem, when it is dense) are solved one at a time by the
// single-solve path instead of the batched launch (negative: never). The
// batched launch itself (batch_run) takes every problem it is given.
struct BatchTuning {
    int small_max_nm = 1 << 16;
    int row_tile_elems = 1 << 16;
    int ctas_per_sm = 0;
    int dense_solo_min_nm = 1 << 24;
};

struct BatchResult;

struct BatchEnv {
    int num_sms = 1;
    int occ_solve = 1;
    size_t budget_left = 0;      // 0: no cap
    cudaEvent_t ev0 = nullptr, ev_mid = nullptr, ev1 = nullptr;
    // Early completion (optional): host-mapped arrays of at least `count`
    // results and flags (flags zero at the call) and their device addresses.
    // While the launch runs, batch_run polls the flags and calls on_done(k, r)
    // once for every problem k the kernel has finished, in finishing order.
    BatchResult *early_host = nullptr, *early_dev = nullptr;
    int32_t *flag_host = nullptr, *flag_dev = nullptr;
    std::function<void(int, const accsink_result &)> on_done;
};

struct BatchTiming {
    float total_ms = 0, form_ms = 0, solve_ms = 0;
    float solo_ms = 0;      // the dense problems solved one at a time (in total and solve)
    int grid = 0;
};

BatchTuning batch_default_tuning(int num_sms);

// Device workspace bytes batch_run needs for these problems.
size_t batch_workspace_bytes(const BatchTuning &tn, int count, const accsink_problem *probs);
// The same number from the full plan (every formation tile listed); for
// checks of the incremental sizer below.
size_t batch_workspace_bytes_planned(const BatchTuning &tn, int count,
                                     const accsink_problem *probs);

// Workspace bytes of a batch that grows one problem at a time, in O(1) per
// problem (the plan's sizes without its tile lists): the server's admission
// adds queued requests one by one against its memory budget.
class BatchSizer {
public:
    explicit BatchSizer(const BatchTuning &tn);
    void add(const accsink_problem &q);
    size_t bytes() const;
    int count() const { return count_; }

private:
    BatchTuning tn_;
    bool tc_on_;
    size_t data_ = 0, outstanding_ = 0;
    int64_t tiles_ = 0, R_ = 0;
    int dpad_ = 0, ntc_ = 0, count_ = 0;
};

// Plans, launches and waits for one batch on stream s. Returns an ACCSINK_*
// code; res[k] receives each problem's record; err the message on failure.
int batch_run(const BatchEnv &env, BatchWorkspace &ws, const BatchTuning &tn, int count,
              const accsink_problem *probs, const accsink_params *params, double *const *f_out,
              double *const *g_out, accsink_result *res, cudaStream_t s, std::string &err,
              BatchTiming *timing);

}  // namespace accsink

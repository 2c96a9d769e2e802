// Internal declarations of the batched solver (many independent problems in
// one persistent launch).
//
// Each problem's cost is formed once into the workspace as a double-float
// pair (Kh + Kl = k C, k = log2(e) / eps_c, so that the passes work in log2
// units), then a persistent kernel solves every problem. Its CTAs pull work
// items from a device queue: a whole solve for a small problem, or one
// phase tile (rows of the row pass, columns of the column pass, rows of the
// final pass) of a large one. The last CTA to finish a phase of a problem
// (per-problem arrival counter) runs the step of Algorithm 1 for it and
// queues the next phase, so no CTA ever waits for another to make progress;
// a CTA only waits, bounded, for the next item to be published.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace accsink {

// One problem of a batch (device-resident). Inputs are the caller's device
// pointers; the rest points into the batch workspace.
struct BatchProb {
    // ---- inputs
    const float *C, *X, *Y;
    const double *a_in, *b_in;
    double *f_out, *g_out;
    int64_t ldc;
    int32_t n, m, d, kind, scale;
    int32_t method, stability, carry, max_steps, m0, evaluate;
    int32_t pad_in;
    double eps, tol, mu0;
    // ---- workspace
    float *Kh, *Kl;          // n x ldm, k C as (hi, lo); C before scaling
    int64_t ldm;             // m rounded up to 4
    float *KTh, *KTl;        // m x ldn, the transpose (large problems only, else null)
    int64_t ldn;             // n rounded up to 4
    double *a, *loga, *u;    // n
    float *Fh, *Fl;          // n (padded): k (eps_c u + shift_f) as (hi, lo)
    double *b, *logb, *x, *x_prev, *w, *w1, *p_prev, *D_prev, *raw, *D1, *del, *ell;  // m
    float *Gh, *Gl;          // m (padded): k (eps_c x + shift_g) as (hi, lo)
    double *rowpart;         // row tiles x 2 (sum a u, sum cost)
    double *colrec;          // column tiles x kBatchColRec (step P1 sums and bounds)
    double *p2rec;           // step items x 3 (P2 sum, min w1, max w1), large problems
    // ---- schedule
    int32_t small;           // 1: the whole solve is one work item
    int32_t row_tiles, rows_per_tile, col_tiles;
    int32_t col_items, cols_per_item;   // column-phase work items (over K^T when present)
    int32_t arrive;          // arrival counter of the phase in flight
    int32_t tc;              // 1: cost formed on the tensor cores (batch_form_tc.cu)
    int32_t tc_xoff, tc_yoff;   // first slice rows of X and Y (tensor-core problems)
    int32_t step_items, step_cols;   // > 0: the step's column loops as work items
    int32_t pad_s;
    // ---- cost statistics from the formation (ordered encodings of FP64)
    unsigned long long cmax_enc, cmin_enc, cabs_enc;
    uint32_t nonfinite;      // bit 0: a non-finite input or cost; bit 1: a formation wait ran out
    uint32_t pad_c;
    // ---- solver state (written by the CTA that owns the current phase)
    double k2, eps_c, inv_eps, cost_div, cmax, cmin, cabs, min_loga, log_m;
    double shift_g, shift_f, mu, kl_prev, err, dual, cost;
    int32_t steps, stages, m_stage, j_in_stage, failures, first, status, done;
    // ---- a step split into work items: P1 totals, then the update's scalars
    double s_v[6], s_lo3[3], s_hi3[3], s_err, s_rbar, s_dual;
    double u_alpha, u_ratio, u_inv1pa;
    int32_t u_wupd, u_gate;
};

// Result record of one problem (device, copied back to the host).
struct BatchResult {
    int32_t status, steps, stages, failures;
    double marginal_l1, transport_cost, dual, cost_max;
};

// Work queue: a ring of 64-bit items with a per-slot sequence word
// (published when seq == pos + 1, free for position pos when seq == pos).
struct BatchQueue {
    unsigned long long head, tail;
    unsigned long long *items;
    unsigned long long *seq;
    unsigned long long cap;      // power of two
    int32_t count;               // problems in the batch
    // optional (a serving loop): host-mapped copies of each problem's result
    // and a flag set once the problem's potentials are written, so the host
    // can hand finished problems back while the launch still runs
    BatchResult *early;
    int32_t *early_flag;
    int32_t done_count;
    int32_t all_done;
    int32_t error;               // ACCSINK_ERR_TIMEOUT on a wait that ran out
};

// Work item kinds.
enum BatchItem {
    BI_SMALL = 0, BI_INIT = 1, BI_ROW = 2, BI_COL = 3, BI_FINAL = 4,
    BI_P2 = 5,    // a column range of the step's P2 sums (large problems)
    BI_UPD = 6    // a column range of the step's update of x, w and G' (large problems)
};

// Large problems (tiled, m >= kBatchStepSplitMin) run the step's per-column
// loops as items of kBatchStepCols columns instead of in one CTA.
constexpr int kBatchStepSplitMin = 4096;
constexpr int kBatchStepCols = 1024;

__host__ __device__ inline unsigned long long batch_item(int kind, int prob, int tile)
{
    return ((unsigned long long)(uint32_t)prob << 32) | ((unsigned long long)kind << 28) |
           (unsigned long long)(uint32_t)tile;
}

// A 64 x 64 tile of one problem's cost for the formation kernels.
struct BatchTile {
    int32_t prob, row0, col0, pad;
};

// Tensor-core formation of cosine costs: 128 x 64 tiles, 32 contraction
// elements per stage, six 7-bit slices per vector; exact class sums need
// d 2^15 < 2^24, i.e. d <= 480 (d padded to a multiple of 32).
constexpr int kBatchTcRows = 128, kBatchTcCols = 64, kBatchTcK = 32, kBatchTcLevels = 6;
constexpr int kBatchTcMinD = 32, kBatchTcMaxD = 480;

// Arguments of the tensor-core formation (device pointers into the workspace).
struct BatchTcLaunch {
    const BatchTile *tiles;      // 128 x 64 tiles of the tensor-core problems
    int ntiles;
    const int32_t *tcp;          // the tensor-core problems
    const int64_t *tcs;          // first slice row of each (X rows, then Y rows)
    int ntc;
    int dpad;                    // contraction length padded to kBatchTcK
    int64_t R;                   // slice rows
    void *SL;                    // FP16 slices [kBatchTcLevels][R][dpad]
    int32_t *expo;               // exponent of each slice row
    int sms;                     // persistent CTAs (one per SM), from prepare_batch_form_tc
};

// Order-preserving map of doubles to unsigned 64-bit integers (for atomic
// min / max of FP64 values).
__device__ __forceinline__ unsigned long long enc_d(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double dec_d(unsigned long long e)
{
    const unsigned long long b = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    return __longlong_as_double((long long)b);
}

constexpr int kBatchThreads = 256;
constexpr int kBatchColTile = 128;     // columns per column-pass item (32 lanes x 4)
constexpr int kBatchFormTile = 64;     // formation tile edge
constexpr int kBatchColWarps = kBatchColTile / 32;   // warps that finish a column tile
constexpr int64_t kBatchTransposeMin = 1 << 20;      // n m from which K^T is also stored
// per 128-column group: for each finishing warp 6 sums, 3 minima, 3 maxima
constexpr int kBatchColRec = 12 * kBatchColWarps;

cudaError_t launch_batch_form(const BatchProb *P, const BatchTile *tiles, int ntiles,
                              int dmax, cudaStream_t s);
bool batch_tc_available();
size_t batch_tc_slice_bytes(int64_t R, int dpad);
// Sets the formation kernel's shared-memory attribute and returns the current
// device's SM count in *sms (host calls only, made before a graph capture).
cudaError_t prepare_batch_form_tc(int *sms);
cudaError_t launch_batch_form_tc(BatchProb *P, const BatchTcLaunch &t, cudaStream_t s);
cudaError_t launch_batch_scale(BatchProb *P, const BatchTile *tiles, int ntiles, cudaStream_t s);
cudaError_t launch_batch_solve(BatchProb *P, BatchQueue *q, BatchResult *res, int grid,
                               cudaStream_t s);
int occupancy_batch_solve();
cudaError_t launch_queue_init(BatchQueue *q, const unsigned long long *items0, int count,
                              unsigned long long cap, cudaStream_t s);

}  // namespace accsink

// Internal declarations of the sm_103a Acc-Sinkhorn solver.
//
// Units. Kernels work with the cost exactly as stored (FP32) and the
// effective regulariser eps_c = eps * cost_div (cost_div = max C when the
// caller asked for MAX_TO_ONE scaling, else 1). The iterate x and the row
// variable u are the paper's dimensionless variables (Sec. 2: cost divided by
// eps); potentials in cost units are f = eps_c u, g = eps_c x.
//
// Precision. The exponent (g_j - C_ij)/eps_c must be accurate to ~1e-7 in
// absolute terms for the l1 marginal error to reach 1e-6 at eps = 1e-3, far
// beyond what a plain FP32 subtraction of O(1) numbers gives (6e-8/eps).
// Each operand is therefore held as an unevaluated FP32 pair
//   G_j + gamma_j = g_j + shift_g   (shift_g makes G_j >= max|C|),
// the difference G_j - C_ij is formed exactly by Fast2Sum (valid because
// |G_j| >= |C_ij|), the per-row reference R_i (a running max of G_j - C_ij)
// is subtracted exactly-relative, and only then is the small remainder
// scaled by log2(e)/eps_c, itself carried as a (hi, lo) FP32 pair. All
// remaining roundings are relative to the shifted exponent, whose size is
// O(10) for every term that matters, so each term's exponent is accurate to
// ~1e-7. Sums use short FP32 chunks folded into Kahan-compensated partials;
// cross-thread merges and every per-row / per-column finish are FP64.
// A product whose rounded value enters an error-free transformation (its
// error recovered by an FMA, a TwoSum or a Kahan update) is written
// __fmul_rn, which the compiler never fuses into a neighbouring add: a fused
// multiply-add there would silently break the exactness (the register
// allocation of a build decides where nvcc contracts a plain a * b + c).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace accsink {

constexpr double kLog2e = 1.44269504088896340736;
constexpr double kLn2 = 0.69314718055994530942;
constexpr int kColStrip = 128;      // columns per column-pass CTA (32 lanes x 4)
constexpr int kPartStride = 16;     // doubles per block partial in the step kernel
constexpr int kMaxStages = 160;     // homotopy stages tabulated (alpha ~ 1e-24 at the last)
constexpr int kStageSlots = 8;      // alpha, 1/alpha, 1/(1+alpha), alpha^2-2, kappa1,
                                    // alpha^1.5, alpha_next/alpha, 1/(1+alpha_next)

// Guard band of the stopping test (Sec. 5 eq. l1tol). The test runs on the
// FP64 sum of the column errors that the FP32 passes give, which misses the
// FP64 truth of ||P1 - a||_1 + ||P'1 - b||_1 by the row marginal's FP32 floor
// (the row pass's u is exact only to FP32 rounding: 3e-8 to 1.2e-7 measured)
// and the column sums' own error (up to 3e-8 measured). A solve therefore
// stops once that estimate is below tol - 2^-22 (2.4e-7), so that the FP64
// truth of the whole eq. l1tol sum stays below tol.
constexpr double kStopGuard = 0x1p-22;
inline double stop_threshold(double tol) { return tol - kStopGuard; }

// Device-resident solver state. Written only by the init kernel, by block 0
// of the step kernel (after its last grid barrier) and by the host before a
// launch; read by every kernel.
struct DevState {
    // problem constants
    double eps_c;        // regulariser in stored-cost units (eps * cost_div)
    double inv_eps_c;
    double eps_user;     // eps as given (potentials are returned as eps_user * x)
    double cost_div;     // 1 or max C
    double tol;
    double cmax, cmin, cabs;   // max C, min C, max |C|
    double min_loga;
    double log_m;
    double sum_a, sum_b;
    // double-float operand constants
    double shift_g, shift_f;
    float k_hi, k_lo;          // log2(e)/eps_c = k_hi + k_lo
    double k2;                 // log2(e)/eps_c in FP64 (point-cloud operands)
    // Algorithm 1/2 state
    double mu;
    double kl_prev;            // D_phi*(0, grad f(x_k)) of the previous iterate
    double err;                // marginal L1 at the last evaluated iterate
    double dual;               // dual objective there (cost units, scaled)
    double last_cond[4];
    int32_t method, stability, carry, max_steps;
    int32_t m_stage, j_in_stage, steps, stages, failures;
    int32_t first, done, status, use_cond;
    int32_t hist_cap, row_grid, col_splits, nonfinite;
    int32_t mode;              // step-kernel mode (solve / single map)
    int32_t col_mode;          // 0: column partials (strip pass); 1: ell from C^T
    uint32_t barrier;          // grid-barrier arrival counter (reset by the row pass)
    int32_t pad[1];
};

enum StepMode { STEP_SOLVE = 0, STEP_MAP = 1 };

// Workspace pointers shared by the kernels (all device memory).
struct Work {
    // marginals
    double *a, *b, *loga, *logb;
    // iterate state (m)
    double *x, *x_prev, *w, *p_prev, *D_prev;
    // per-column scratch of the step kernel (m)
    double *raw, *D1, *del, *w1;
    // row pass output (n)
    double *u;
    // double-float operands
    float *G, *Gk;            // m (row pass)
    float2 *FF;               // n (column pass): (F_hi, F_lo * k_hi)
    float *Fh, *Fk;           // n: the same pair as two arrays (transposed column pass)
    double *ell;              // m: column log-sum-exp (transposed column pass)
    // partials
    float2 *colpart;          // splits x m : (R, S) per column per row split
    double *rowpart;          // row-grid x 2 : (sum a_i u_i, sum cost) per CTA
    double *steppart;         // kPartStride doubles per block of the O(n + m) kernels
                              // (block-major; the step kernel stores them slot-major)
    double *statpart;         // cost-stats grid x 4
    // per-stage constants of Algorithm 1/2 (kStageSlots doubles per stage)
    const double *stage_table;
    // history (hist_cap each)
    double *h_err, *h_dual, *h_mu, *h_cond;
    int32_t *h_stab;
    DevState *st;
    // point-cloud costs (NULL for a dense cost): Bx = s||x||^2 (or 0), By =
    // s||y||^2 (or s) in FP64 and as pairs; scaled points in SoA pairs
    double *Bx64, *By64;
    float *Bxh, *Bxl, *Byh, *Byl;
    float *PXh, *PXl, *PYh, *PYl;
    int64_t ldx, ldy;         // SoA row strides (n, m rounded up to 4)
    double *rowmax;           // n: row maxima of the cost (scaling)
    // rows split into column parts (warp-per-row pass): per part its
    // (R, hi, lo) record and cost pair; per row an arrival counter, zero
    // between passes
    float4 *prec;
    float2 *pcrec;
    uint32_t *pcnt;
    // inputs of the single-pass entry points
    const double *b_src;      // column marginal to copy (may be NULL)
    const double *f_given;    // row potentials weighting the cost sum (may be NULL)
    int32_t nstat;            // number of cost-statistics partials
    int32_t ignore_done;      // row pass runs even when the solve has stopped
};

// One pass over a point-cloud cost: rows of P (AoS, nr x d) against columns
// whose scaled points are Qh/Ql (SoA, d x ldq); A (per column) and B (per
// row) are the expansion terms as pairs; Ch (per column, hi) serves the
// transport-cost sum.
// One point-cloud pass: rows r of P (nr x d, row-major FP32) against the
// columns c of Q (d x ldq SoA, (hi, lo) FP32 pairs, pre-scaled to log2
// units), with the per-column operand A (pairs) and the rows' FP64 norm term
// B64 (applied in the finish). Pc (the columns' points, nc x d) and scal
// ({max C, s}) are only read when the transport cost is accumulated, which
// forms each C_ij directly from the points.
struct PointView {
    const float *P, *Pc;
    const float *Ah, *Al, *Qh, *Ql;
    const double *B64, *scal;
    int64_t ldq;
    int32_t nr, nc, d, kind;
    int32_t prune;   // 1: points sorted along a space-filling curve; far slots skipped
    int32_t fp32;    // 1: x.Q in plain FP32 (no low parts)
    // pruned passes: per group of four rows, the slot of the column nearest to
    // the group's first row (-1: none); may be NULL
    const int32_t *hint;
    // pruned passes: log2 of the ratio below a row's largest term under which
    // a term is skipped (see points.cu)
    float skip;
    // pruned passes, per block of 64 columns (kBoxSlots float4 slots) of the
    // whole chunks: qbox[2 b], qbox[2 b + 1] = the minimum and maximum of each of
    // the block's Q coordinates (d <= 4), fixed for the solve; abox[b] = the
    // maximum of the block's A and of |A| (high parts), set before every
    // pass by launch_points_pass. NULL: no block test.
    const float4 *qbox;
    float2 *abox;
    // pruned passes without the cost sum: row groups are taken from this
    // counter (zeroed by the block-record kernel before every pass) instead of
    // dealt round-robin, so warps whose rows prune well take more of them.
    // NULL: round-robin.
    unsigned int *next_group;
};

struct CostView {
    const float *C;
    int64_t ldc;
    int32_t n, m;
    int32_t vec;   // 1: ldc % 4 == 0 and C 16-byte aligned
};

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2^((d) * k) with k = kh + kl, d small: both products rounded once.
__device__ __forceinline__ float exp2_scaled(float d, float kh, float kl)
{
    return ex2_approx(fmaf(d, kh, d * kl));
}

__device__ __forceinline__ float4 ld_stream4(const float *p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ float ld_stream1(const float *p)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Running log2-sum-exp accumulator of one lane: sum = (S - K) 2^R (Kahan
// pair S, K about the running maximum R).
struct Lse2 {
    float R, S, K;
};

__device__ __forceinline__ void lse2_kahan(Lse2 &a, float x)
{
    const float y = x - a.K;
    const float t = a.S + y;
    a.K = (t - a.S) - y;
    a.S = t;
}

// Knuth's TwoSum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Folds one slot's terms 2^(h + l - R) into a row accumulator; raises R to
// the slot maximum first (rare after the first slots).
template <bool WC>
__device__ __forceinline__ void slot_accumulate(Lse2 &acc, Lse2 &cacc, const float h[4],
                                                const float l[4], const float cst[4])
{
    const float m4 = fmaxf(fmaxf(h[0], h[1]), fmaxf(h[2], h[3]));
    if (m4 > acc.R) {
        const float f = ex2_approx(acc.R - m4);
        acc.S = __fmul_rn(acc.S, f);
        acc.K = __fmul_rn(acc.K, f);
        if (WC) { cacc.S = __fmul_rn(cacc.S, f); cacc.K = __fmul_rn(cacc.K, f); }
        acc.R = m4;
    }
    float s = 0.0f, cs = 0.0f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float t = ex2_approx((h[e] - acc.R) + l[e]);   // h - R exact (Sterbenz)
        s += t;
        if (WC) cs = fmaf(cst[e], t, cs);
    }
    lse2_kahan(acc, s);
    if (WC) lse2_kahan(cacc, cs);
}

// Grid-wide barrier for cooperatively launched kernels (all blocks resident).
// `target` is the arrival count to wait for (k * gridDim for the k-th
// barrier of a launch; the counter is zeroed by the kernel that runs before).
// The wait is bounded by `limit_ns` of global time; on expiry the barrier
// records ACCSINK_ERR_TIMEOUT in the state, stops the solve and returns false.
__device__ __forceinline__ bool grid_barrier(DevState *st, uint32_t target, uint64_t limit_ns)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(&st->barrier, 1u);
        uint64_t t0 = globaltimer_ns();
        for (;;) {
            uint32_t v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&st->barrier));
            if (v >= target) break;
            if (globaltimer_ns() - t0 > limit_ns) {
                ok = 0;
                atomicExch(&st->status, 6 /* ACCSINK_ERR_TIMEOUT */);
                atomicExch(&st->done, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// ---------------------------------------------------------------- launches --

struct LaunchCfg {
    int num_sms;
    int row_grid;      // row-pass CTAs
    int col_splits;    // column-pass row splits
    int step_grid;     // step-kernel CTAs (cooperative)
    int stat_grid;
};

cudaError_t launch_cost_stats(const CostView &cv, const Work &w, int grid, cudaStream_t s);
// Work split of the warp-per-row pass: `grid` CTAs; rows [0, nfull) whole,
// the rows after them in `parts` column parts of part4 float4 slots each.
struct RowSplit {
    int grid = 1, nfull = 0, parts = 1, part4 = 0;
};
cudaError_t launch_row_pass(const CostView &cv, const Work &w, int grid, const RowSplit &sp,
                            bool with_cost, cudaStream_t s);
cudaError_t launch_col_pass(const CostView &cv, const Work &w, int splits, cudaStream_t s);
// How a solve starts (k_init): at zero, or at a given iterate.
//   x: the iterate (multiplied by mul: a resume at a new eps), or, when
//      div > 0, a potential g0 with x = g0 / div (a warm start);
//   w: the momentum (times mul); NULL gives w = sqrt(2 mu) x for the Acc
//      method (y = x) and 0 for plain Sinkhorn;
//   perm: the solve's columns are a permutation of the caller's (sorted
//      point clouds);
//   keep_shifts: reuse the operand shifts below when the cost statistics
//      and eps_c they were derived for equal this solve's.
struct InitState {
    const double *x = nullptr, *w = nullptr;
    const int *perm = nullptr;   // column j of the solve reads x[perm[j]], w[perm[j]]
    double mul = 1.0, div = 0.0;
    int32_t keep_shifts = 0;
    double shift_g = 0.0, shift_f = 0.0, cabs = 0.0, cmin = 0.0, eps_c = 0.0;
};
cudaError_t launch_init(const CostView &cv, const Work &w, int grid, const double *a_in,
                        const double *b_in, int scale_max, const InitState &is,
                        cudaStream_t s);
cudaError_t launch_barrier_selftest(DevState *st, int grid, uint64_t limit_ns, cudaStream_t s);
cudaError_t launch_step(const CostView &cv, const Work &w, int grid,
                        cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_step_map(const CostView &cv, const Work &w, int grid, double *c_out,
                            double *s_out, cudaStream_t s);
cudaError_t launch_prep_g(const CostView &cv, const Work &w, int grid, const double *g,
                          const double *a_in, double eps, int scale_max, cudaStream_t s);
cudaError_t launch_prep_f(const CostView &cv, const Work &w, int grid, const double *f,
                          double eps, int scale_max, cudaStream_t s);
cudaError_t launch_scale_out(const double *src, double scale, double *dst, int n,
                             cudaStream_t s);
cudaError_t launch_col_finish_lse(const Work &w, int m, double *ell_out, cudaStream_t s);
int occupancy_row_pass(int vec);
cudaError_t launch_row_pass_tma(const CostView &cv, const Work &w, int grid, bool with_cost,
                                cudaStream_t s);
cudaError_t setup_row_pass_tma();
int row_pass_tma_smem_bytes();
RowSplit plan_row_split(int rows, int cols, int64_t max_warps);
// Part records a split pass needs (0 without a split).
int64_t row_split_records(const RowSplit &r, int rows);
cudaError_t launch_row_pass_warp(const CostView &cv, const Work &w, int grid,
                                 const RowSplit &sp, bool with_cost, cudaStream_t s);
int occupancy_row_pass_warp();
cudaError_t launch_col_pass_transposed(const float *CT, int64_t ldct, int n, int m,
                                       const Work &w, int grid, const RowSplit &sp,
                                       cudaStream_t s);
cudaError_t launch_transpose(const CostView &cv, float *CT, int64_t ldct, cudaStream_t s);
// The transposed copy and the cost statistics of k_cost_stats in one read of
// C (cv.vec only): `grid` CTAs, each writing its partial to
// w.statpart[part0 + blockIdx.x]; only rows [r0, r1) of C (r0 a multiple of
// 64, r1 a multiple of 64 or n; r1 = -1: n).
cudaError_t launch_transpose_stats(const CostView &cv, float *CT, int64_t ldct, const Work &w,
                                   int grid, cudaStream_t s, int r0 = 0, int r1 = -1,
                                   int part0 = 0);
// Which kernel serves 128-bit-aligned row passes: 0 warp-per-row, 1 TMA.
int row_kernel_choice();
int occupancy_col_pass(int vec);
cudaError_t launch_points_pass(const PointView &pv, const Work &w, int grid, int mode,
                               bool with_cost, cudaStream_t s);
int occupancy_points_pass();
// CTAs per SM of the pruned pass kernel for dimension d <= 4.
int occupancy_points_pruned(int d);
// Spatial sort of one point cloud: buffers in the solve's point workspace.
// P (n x d) and a (n) receive the cloud and its marginal in Hilbert-curve order;
// perm[i] is the original index of sorted point i.
struct PointSort {
    uint32_t *box, *code, *code2;
    int *idx, *perm;
    void *temp;
    size_t temp_bytes;
    float *P;
    double *a;
};
size_t points_sort_temp_bytes(int count);
// Slot hints of the pruned passes over rows of P against columns of Q (d <= 4).
cudaError_t launch_points_hint(const float *P, int nr, const float *Q, int nc, int d, int kind,
                               int32_t *hint, int grid, cudaStream_t s);
cudaError_t launch_points_sort(const float *P, const double *a, int n, int d, const PointSort &ps,
                               cudaStream_t s);
// dst[perm[i]] = scale * src[i]
cudaError_t launch_scatter_scaled(const double *src, double scale, const int *perm, int n,
                                  double *dst, cudaStream_t s);
cudaError_t launch_points_rowmax(const float *X, const float *Y, int n, int m, int d, int kind,
                                 double *rowmax, int grid, cudaStream_t s);
cudaError_t launch_points_setup(const float *X, const float *Y, int n, int m, int d, int kind,
                                int scale_max, double eps, const Work &w, double *scal,
                                double *blockmax, int nblk, cudaStream_t s);
int points_rows_per_warp(int d);
// Block records of the pruned passes cover kBoxSlots float4 slots (64
// columns) each; the whole 32-slot chunks of nc columns hold
// points_blocks(nc) of them.
constexpr int kBoxSlots = 16;
inline int points_blocks(int nc) { return ((nc >> 2) & ~31) / kBoxSlots; }
// The per-block coordinate boxes of Q (nc x d SoA with leading dimension
// ldq, d <= 4) for the block test of the pruned passes.
cudaError_t launch_points_qbox(const float *Qh, int64_t ldq, int nc, int d, float4 *qbox,
                               cudaStream_t s);
// log2 threshold of the pruned passes for rows of nc terms: every skipped
// term is below 2^-(skip + 1) of its row's largest, so all of a row's
// skipped terms together stay below 2^-30 of its sum.
inline float points_skip_log2(int nc)
{
    int l = 0;
    while ((1ll << l) < (long long)nc) ++l;
    return (float)(29 + l);
}
void setup_col_pass();

}  // namespace accsink

// O(n + m) kernels around the two streaming passes: problem set-up, the fused
// per-iteration step of Algorithm 1/2, and operand preparation for the
// single-pass entry points. They are cooperative launches (every block is
// resident) that separate their phases with the bounded grid barrier of
// accsink_internal.cuh; every block reduces the block partials itself in the
// same fixed order, so all blocks agree bit-for-bit on every scalar and the
// whole solve is deterministic. FP64 is used for the marginal-error and
// dual-objective sums and for the Theorem 4 stability test.
#include <float.h>

#include "accsink_internal.cuh"

namespace accsink {

// Two warps per block: every FP64 instruction of a warp holds the SM's narrow
// FP64 pipe (about 2 operations per clock on GB300) for ~16 cycles, and the
// block reductions cost the same FP64 instructions per warp whatever the
// column count, so more warps per block made the step slower (measured).
constexpr int kVecNT = 64;
constexpr uint64_t kBarrierLimitNs = 2000000000ull;   // 2 s per barrier

// Sum K per-thread doubles over the block; thread k < K writes the k-th sum
// to out[k]. Deterministic (fixed shuffle tree, fixed warp order).
template <int K>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double *out)
{
    __shared__ double sh[K][kVecNT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int q = 0; q < kVecNT / 32; ++q) s += sh[threadIdx.x][q];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double warp_min_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block min/max of one double each; thread 0 writes (min, max) to out[0..1].
__device__ __forceinline__ void block_minmax_store(double mn, double mx, double *out)
{
    __shared__ double sh[2][kVecNT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    mn = warp_min_d(mn);
    mx = warp_max_d(mx);
    if (lane == 0) { sh[0][wid] = mn; sh[1][wid] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kVecNT / 32; ++q) { mn = fmin(mn, sh[0][q]); mx = fmax(mx, sh[1][q]); }
        out[0] = mn;
        out[1] = mx;
    }
    __syncthreads();
}

// Reduces K values held by every thread over the whole block (op per value:
// 0 sum, 1 min, 2 max) and returns the totals to every thread. Fixed
// shuffle tree and fixed warp order, so the result is deterministic.
template <int K>
__device__ __forceinline__ void block_allreduce(double (&v)[K], const int (&op)[K])
{
    __shared__ double sh[K][kVecNT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (op[k] == 0) ? x + y : (op[k] == 1 ? fmin(x, y) : fmax(x, y));
        }
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = sh[k][0];
        for (int q = 1; q < kVecNT / 32; ++q)
            x = (op[k] == 0) ? x + sh[k][q] : (op[k] == 1 ? fmin(x, sh[k][q]) : fmax(x, sh[k][q]));
        v[k] = x;
    }
    __syncthreads();
}

// Totals of K consecutive slots of every block's partial record (stride
// kPartStride), computed identically by every block: thread t reads the
// records t, t + blockDim, ... (bypassing L1, they were written by other
// blocks) and the block reduces them in a fixed order.
template <int K>
__device__ __forceinline__ void grid_totals(const double *part, int nblocks, int slot0,
                                            const int (&op)[K], double (&tot)[K])
{
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = (op[k] == 0) ? 0.0 : (op[k] == 1 ? DBL_MAX : -DBL_MAX);
    for (int b = threadIdx.x; b < nblocks; b += kVecNT) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double x = __ldcg(&part[(int64_t)b * kPartStride + slot0 + k]);
            tot[k] = (op[k] == 0) ? tot[k] + x : (op[k] == 1 ? fmin(tot[k], x) : fmax(tot[k], x));
        }
    }
    block_allreduce<K>(tot, op);
}

// Reduction of the cost-statistics partials (max C, min C, max|C|, #bad).
__device__ __forceinline__ void cost_totals(const double *statpart, int nstat, double &cmax,
                                            double &cmin, double &cabs, double &bad)
{
    double v[4] = {-DBL_MAX, DBL_MAX, 0.0, 0.0};
    const int op[4] = {2, 1, 2, 0};
    for (int b = threadIdx.x; b < nstat; b += kVecNT) {
        v[0] = fmax(v[0], __ldcg(&statpart[4 * b + 0]));
        v[1] = fmin(v[1], __ldcg(&statpart[4 * b + 1]));
        v[2] = fmax(v[2], __ldcg(&statpart[4 * b + 2]));
        v[3] += __ldcg(&statpart[4 * b + 3]);
    }
    block_allreduce<4>(v, op);
    cmax = v[0]; cmin = v[1]; cabs = v[2]; bad = v[3];
}

// Writes the row-pass operand for column j from g_j + shift_g: for a dense
// cost the pair (hi, lo k_hi) of G_j; for a point-cloud cost the pair
// (hi, lo) of A_j = k (G_j - By_j) in log2 units (k = log2(e)/eps_c, the
// expansion term of points.cu).
__device__ __forceinline__ void write_G(const Work &w, int j, double gshift, float kh, double k)
{
    if (w.By64) {
        const double a = k * (gshift - w.By64[j]);
        const float hi = (float)a;
        w.G[j] = hi;
        w.Gk[j] = (float)(a - (double)hi);
        return;
    }
    const float hi = (float)gshift;
    const float lo = (float)(gshift - (double)hi);
    w.G[j] = hi;
    w.Gk[j] = lo * kh;
}

// ------------------------------------------------------------------------
// Set-up of a solve. The host has written eps_user, tol, mu, method, the
// homotopy position, ... into the state (barrier = 0). Validates and
// normalises the marginals, derives eps_c and the operand shifts, and writes
// x_0, w_0 (zero, or the start `is` gives) and G for x_0.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecNT) k_init(Work w, int n, int m, int nstat,
                                                 const double *a_in, const double *b_in,
                                                 int scale_max, InitState is)
{
    DevState *st = w.st;
    const int tid = blockIdx.x * kVecNT + threadIdx.x;
    const int nthr = gridDim.x * kVecNT;
    const uint32_t nb = gridDim.x;

    double cmax, cmin, cabs, bad;
    cost_totals(w.statpart, nstat, cmax, cmin, cabs, bad);

    // phase A: sums and validity of a, b
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // sum a, sum b, #a<=0, #b<=0, #nonfinite
    for (int i = tid; i < n; i += nthr) {
        const double ai = a_in[i];
        v[0] += ai;
        if (!(ai > 0.0)) v[2] += 1.0;
        if (!isfinite(ai)) v[4] += 1.0;
    }
    for (int j = tid; j < m; j += nthr) {
        const double bj = b_in[j];
        v[1] += bj;
        if (!(bj > 0.0)) v[3] += 1.0;
        if (!isfinite(bj)) v[4] += 1.0;
    }
    block_sum_store<6>(v, w.steppart + (int64_t)blockIdx.x * kPartStride);
    if (!grid_barrier(st, nb, kBarrierLimitNs)) return;
    double t[6];
    const int ops6[6] = {0, 0, 0, 0, 0, 0};
    grid_totals<6>(w.steppart, nb, 0, ops6, t);
    int status = 0;
    if (bad > 0.0 || t[4] > 0.0) status = 3;           // ACCSINK_ERR_NONFINITE
    else if (t[2] > 0.0 || t[3] > 0.0) status = 2;     // ACCSINK_ERR_NONPOSITIVE_MARGINAL
    else if (scale_max && !(cmax > 0.0)) status = 1;   // cannot scale by max C <= 0
    if (status != 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->status = status;
            st->done = 1;
            st->cmax = cmax;
        }
        return;
    }
    const double sa = t[0], sb = t[1];
    const double cost_div = scale_max ? cmax : 1.0;
    const double eps_c = st->eps_user * cost_div;
    const double k = kLog2e / eps_c;
    const float kh = (float)k;
    const float kl = (float)(k - (double)kh);

    // phase B: normalised marginals, logs, the starting iterate
    const double alpha0 = st->method == 1 ? sqrt(2.0 * st->mu) : 0.0;
    double mnla = DBL_MAX, xlo = DBL_MAX, xhi = -DBL_MAX;
    for (int i = tid; i < n; i += nthr) {
        const double ai = a_in[i] / sa;
        w.a[i] = ai;
        w.loga[i] = log(ai);
        mnla = fmin(mnla, w.loga[i]);
    }
    for (int j = tid; j < m; j += nthr) {
        const double bj = b_in[j] / sb;
        w.b[j] = bj;
        w.logb[j] = log(bj);
        double xj = 0.0, wj = 0.0;
        if (is.x) {
            const int jj = is.perm ? is.perm[j] : j;
            xj = is.div > 0.0 ? is.x[jj] / is.div : is.x[jj] * is.mul;
            wj = is.w ? is.w[jj] * is.mul : alpha0 * xj;
        }
        w.x[j] = xj;
        w.x_prev[j] = xj;
        w.w[j] = wj;
        w.p_prev[j] = 0.0;
        w.D_prev[j] = bj;
        xlo = fmin(xlo, xj);
        xhi = fmax(xhi, xj);
    }
    // block min of log a and bounds of x_0 into slots 6..8 (slots 0..5 are
    // still being read)
    {
        double v3[3] = {mnla, xlo, xhi};
        const int ops3[3] = {1, 1, 2};
        block_allreduce<3>(v3, ops3);
        if (threadIdx.x == 0) {
            double *r = w.steppart + (int64_t)blockIdx.x * kPartStride;
            r[6] = v3[0];
            r[7] = v3[1];
            r[8] = v3[2];
        }
    }
    if (!grid_barrier(st, 2 * nb, kBarrierLimitNs)) return;
    double t3[3];
    const int ops3[3] = {1, 1, 2};
    grid_totals<3>(w.steppart, nb, 6, ops3, t3);
    const double min_loga = t3[0];
    const double log_m = log((double)m);
    // G = eps_c x + shift_g with shift_g = max|C| - eps_c min x makes
    // G >= |C|; F_i >= max|C| follows from
    // eps_c u_i >= eps_c min log a - eps_c max x + min C - eps_c log m.
    // At x_0 = 0 that is shift_g = max|C|; a given x_0 has exact bounds,
    // widened by a relative margin for the rounding of eps_c x + shift.
    double shift_g, shift_f;
    if (is.keep_shifts && is.cabs == cabs && is.cmin == cmin && is.eps_c == eps_c) {
        shift_g = is.shift_g;
        shift_f = is.shift_f;
    } else if (is.x) {
        const double lo = t3[1] - 1e-12 * (1.0 + fabs(t3[1]));
        const double hi = t3[2] + 1e-12 * (1.0 + fabs(t3[2]));
        shift_g = cabs - eps_c * lo;
        shift_f = cabs - (eps_c * min_loga - eps_c * hi + cmin - eps_c * log_m);
    } else {
        shift_g = cabs;
        shift_f = cabs - (eps_c * min_loga - 0.0 + cmin - eps_c * log_m);
    }
    if (is.x) {
        for (int j = tid; j < m; j += nthr) write_G(w, j, eps_c * w.x[j] + shift_g, kh, k);
    } else {
        for (int j = tid; j < m; j += nthr) write_G(w, j, shift_g, kh, k);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->eps_c = eps_c;
        st->inv_eps_c = 1.0 / eps_c;
        st->cost_div = cost_div;
        st->cmax = cmax; st->cmin = cmin; st->cabs = cabs;
        st->sum_a = sa; st->sum_b = sb;
        st->min_loga = min_loga;
        st->log_m = log_m;
        st->shift_g = shift_g;
        st->shift_f = shift_f;
        st->k_hi = kh;
        st->k_lo = kl;
        st->k2 = k;
        // (the homotopy position mu, m_stage, j_in_stage, stages is the host's)
        st->steps = 0; st->failures = 0;
        st->first = 1; st->done = 0; st->status = 0;
        st->err = INFINITY; st->dual = 0.0; st->kl_prev = 0.0;
        st->mode = STEP_SOLVE;
    }
}

cudaError_t launch_init(const CostView &cv, const Work &w, int grid, const double *a_in,
                        const double *b_in, int scale_max, const InitState &is,
                        cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kVecNT);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_init, w, cv.n, cv.m, (int)w.nstat, a_in, b_in, scale_max,
                              is);
}

// ------------------------------------------------------------------------
// The per-iteration step, run after the row and column passes at x (the
// iterate being evaluated, x_{k+1} in Algorithm 1's indexing):
//   P1  ell_j (merged column partials, or read from the transposed column
//       pass), p_j = log(c_j/b_j) = x_j + ell_j - log b_j, raw_j = x_j - p_j
//       (v-update), c_j - b_j = b_j expm1(p_j), D_j = (c_j - b_j)/p_j
//       (eq. D), KL term b_j (e^p - 1 - p); block partials of the L1 error,
//       sum raw, KL, <b, x>, Cond 1 lhs and Cond 2 lhs (Theorem 4), and FP32
//       outward-rounded bounds of raw, x, w.
//   P2  S(x) = raw - mean(raw) (Sec. 3); Algorithm 1 w-update
//       w+ = (w + (alpha^2 - 2) x + 2 S(x)) / (1 + alpha); Cond 2 rhs and
//       bounds of w+.
//   P3  stop test (Sec. 5 eq. l1tol), stability verdict and gate, homotopy
//       (Algorithm 2), next x = (w+ + S(x)) / (1 + alpha_next) (or S(x) for
//       plain Sinkhorn) and its operand G. The operand shifts only need
//       bounds of the next x, which the P1/P2 bounds give, so no third grid
//       barrier is needed. Block 0 records the scalars, the history entry and
//       the graph loop condition.
// ------------------------------------------------------------------------
namespace {

// Record slots of a block: sums (FP64) then FP32 bounds stored as doubles.
enum {
    R_ERR = 0, R_RAW, R_KL, R_XB, R_C1, R_C2L, R_AU,    // P1 sums
    R_RAWLO, R_RAWHI, R_XLO, R_XHI, R_WLO, R_WHI,       // P1 bounds
    R_C2R, R_W1LO, R_W1HI,                              // P2
    R_NSLOTS
};
static_assert(R_NSLOTS <= kPartStride, "step-kernel record too long");
// records a thread loads at once in the step's reductions (152 blocks of 64
// threads: three each)
constexpr int kRecPerThread = 4;

__device__ __forceinline__ float lo_f(double v) { return __double2float_rd(v); }
__device__ __forceinline__ float hi_f(double v) { return __double2float_ru(v); }

// Block min and max of floats (exact; ALU pipe).
__device__ __forceinline__ void block_minmax_f(float (&lo)[3], float (&hi)[3])
{
    __shared__ float sh[6][kVecNT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
        if (lane == 0) { sh[k][wid] = lo[k]; sh[3 + k][wid] = hi[k]; }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float a = sh[k][0], b = sh[3 + k][0];
        for (int q = 1; q < kVecNT / 32; ++q) { a = fminf(a, sh[k][q]); b = fmaxf(b, sh[3 + k][q]); }
        lo[k] = a;
        hi[k] = b;
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(kVecNT) k_step(Work w, int n, int m,
                                                 cudaGraphConditionalHandle h,
                                                 double *c_out, double *s_out)
{
    DevState *st = w.st;
    // Any early exit must end the graph's while loop, or it would spin on
    // no-op launches: block 0 clears the condition before returning.
    auto bail = [&]() {
        if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) cudaGraphSetConditional(h, 0u);
    };
    if (*(volatile int32_t *)&st->done) { bail(); return; }
    const int tid = blockIdx.x * kVecNT + threadIdx.x;
    const int nthr = gridDim.x * kVecNT;
    const uint32_t nb = gridDim.x;
    // this block's record, slot k at rec[k * nb]: the records are stored
    // slot-major (slot k of every block contiguous), so the reads of all
    // records by every block are coalesced
    double *rec = w.steppart + blockIdx.x;

    const int method = st->method, first = st->first, stab = st->stability;
    const int mode = st->mode, splits = st->col_splits;
    const double mu = st->mu;
    // alpha-dependent constants of the current stage, tabulated on the host
    // (FP64 transcendentals are slow on this part; every warp would
    // recompute them)
    const bool acc_solve = (method == 1) && (mode == STEP_SOLVE);
    const int stage = min(st->stages, kMaxStages - 1);
    const double one[kStageSlots] = {1.0, 1.0, 0.5, -1.0, 0.0, 1.0, 1.0, 0.5};
    const double *T = acc_solve ? w.stage_table + stage * kStageSlots : one;
    const double alpha = T[0];
    const double inv_alpha = T[1];
    const double inv_1pa = T[2];
    const double inv_eps = st->inv_eps_c;
    const double shift_f = st->shift_f;
    const float kh = st->k_hi, kl = st->k_lo;
    const bool is_acc = acc_solve;
    const bool check = is_acc && !first && stab != 0;
    const bool wupd = is_acc && !first;

    // ---- P1
    double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // err, raw, kl, <b,x>, c1, c2l, <a,u>
    // the first two row terms of <a, u>, loaded with the column loads
    double a0 = 0.0, u0 = 0.0, a1 = 0.0, u1 = 0.0;
    if (tid < n) { a0 = w.a[tid]; u0 = w.u[tid]; }
    if (tid + nthr < n) { a1 = w.a[tid + nthr]; u1 = w.u[tid + nthr]; }
    float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int col_mode = st->col_mode;
    // A thread's columns two at a time: both columns' inputs are loaded
    // before either is used (the stores in between would otherwise keep the
    // compiler from issuing the second column's loads early); the sums take
    // the columns in the same order as one at a time.
    for (int j0 = tid; j0 < m; j0 += 2 * nthr) {
        double ell[2], xj[2], bj[2], wj[2], lb[2], p0[2], xp[2], Dp[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = j0 + u * nthr;
            if (j >= m) continue;
            if (col_mode == 1) {
                ell[u] = w.ell[j];
            } else {
                float R = w.colpart[j].x;
                for (int q = 1; q < splits; ++q) R = fmaxf(R, w.colpart[(int64_t)q * m + j].x);
                double S = 0.0;
                for (int q = 0; q < splits; ++q) {
                    const float2 pr = w.colpart[(int64_t)q * m + j];
                    S += (double)pr.y * (double)exp2_scaled(pr.x - R, kh, kl);
                }
                ell[u] = log(S) + ((double)R - shift_f) * inv_eps;
            }
            xj[u] = w.x[j];
            bj[u] = w.b[j];
            wj[u] = w.w[j];
            lb[u] = w.logb[j];
            if (check) {
                p0[u] = w.p_prev[j];
                xp[u] = w.x_prev[j];
                Dp[u] = w.D_prev[j];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = j0 + u * nthr;
            if (j >= m) continue;
            const double del = xj[u] + ell[u] - lb[u];
            const double raw = xj[u] - del;
            // p = log(c/b) is formed in FP64; e^p - 1, D(p)/b = (e^p - 1)/p
            // and e^p - 1 - p are then needed to ~1e-7 relative, which FP32
            // gives (series for the last one at small p, where the
            // difference cancels).
            double xi, D1, klt;
            const float dl = (float)del;
            if (fabsf(dl) <= 80.0f) {
                const float e = expm1f(dl);
                float km;   // e^p - 1 - p
                if (fabsf(dl) < 0.0625f) {
                    km = dl * dl * fmaf(dl, fmaf(dl, fmaf(dl, fmaf(dl, 1.0f / 720.0f, 1.0f / 120.0f),
                                                         1.0f / 24.0f), 1.0f / 6.0f), 0.5f);
                } else {
                    km = e - dl;
                }
                const float dr = (dl != 0.0f) ? e / dl : 1.0f;
                xi = bj[u] * (double)e;
                D1 = bj[u] * (double)dr;
                klt = bj[u] * (double)km;
            } else {
                const double e = expm1(del);
                xi = bj[u] * e;
                D1 = xi / del;
                klt = bj[u] * (e - del);
            }
            v[0] += fabs(xi);
            v[1] += raw;
            v[2] += klt;
            v[3] += bj[u] * xj[u];
            if (check) {
                const double v0 = wj[u] * inv_alpha - xp[u];
                v[4] += p0[u] * p0[u] * D1;
                v[5] += v0 * v0 * (D1 - Dp[u]);
            }
            blo[0] = fminf(blo[0], lo_f(raw));   bhi[0] = fmaxf(bhi[0], hi_f(raw));
            blo[1] = fminf(blo[1], lo_f(xj[u])); bhi[1] = fmaxf(bhi[1], hi_f(xj[u]));
            blo[2] = fminf(blo[2], lo_f(wj[u])); bhi[2] = fmaxf(bhi[2], hi_f(wj[u]));
            w.raw[j] = raw;
            w.D1[j] = D1;
            w.del[j] = del;
            if (c_out) c_out[j] = bj[u] * exp(del);
        }
    }
    // <a, u> of the dual (Sec. 5), from the row pass's u in a fixed order
    v[6] = a0 * u0;
    if (tid + nthr < n) v[6] += a1 * u1;
    for (int i = tid + 2 * nthr; i < n; i += nthr) v[6] += w.a[i] * w.u[i];
    {
        __shared__ double shs[7];
        block_sum_store<7>(v, shs);
        block_minmax_f(blo, bhi);
        if (threadIdx.x < 7) rec[(R_ERR + threadIdx.x) * nb] = shs[threadIdx.x];
        if (threadIdx.x == 0) {
            rec[R_RAWLO * nb] = blo[0]; rec[R_RAWHI * nb] = bhi[0];
            rec[R_XLO * nb] = blo[1];   rec[R_XHI * nb] = bhi[1];
            rec[R_WLO * nb] = blo[2];   rec[R_WHI * nb] = bhi[2];
        }
    }
    if (!grid_barrier(st, nb, kBarrierLimitNs)) { bail(); return; }

    // ---- P2
    double t[R_WHI + 1];
    {
        // one read of every block's record: the P1 sums and bounds. A
        // thread's records are all loaded before any is added (in the same
        // order as one at a time), so their L2 round trips overlap: the
        // records were written by blocks on every SM, half of them on the
        // other die.
        double t6[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const int ops6[7] = {0, 0, 0, 0, 0, 0, 0};
        float blo2[3] = {INFINITY, INFINITY, INFINITY}, bhi2[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int b0 = threadIdx.x; b0 < (int)nb; b0 += kRecPerThread * kVecNT) {
            double rv[kRecPerThread][R_WHI + 1];
#pragma unroll
            for (int q = 0; q < kRecPerThread; ++q) {
                const int b = b0 + q * kVecNT;
                if (b < (int)nb) {
#pragma unroll
                    for (int k = 0; k <= R_WHI; ++k) rv[q][k] = __ldcg(&w.steppart[k * nb + b]);
                }
            }
#pragma unroll
            for (int q = 0; q < kRecPerThread; ++q) {
                if (b0 + q * kVecNT < (int)nb) {
#pragma unroll
                    for (int k = 0; k < 7; ++k) t6[k] += rv[q][R_ERR + k];
                    blo2[0] = fminf(blo2[0], (float)rv[q][R_RAWLO]);
                    bhi2[0] = fmaxf(bhi2[0], (float)rv[q][R_RAWHI]);
                    blo2[1] = fminf(blo2[1], (float)rv[q][R_XLO]);
                    bhi2[1] = fmaxf(bhi2[1], (float)rv[q][R_XHI]);
                    blo2[2] = fminf(blo2[2], (float)rv[q][R_WLO]);
                    bhi2[2] = fmaxf(bhi2[2], (float)rv[q][R_WHI]);
                }
            }
        }
        block_allreduce<7>(t6, ops6);
        block_minmax_f(blo2, bhi2);
        for (int k = 0; k < 7; ++k) t[k] = t6[k];
        t[R_RAWLO] = blo2[0]; t[R_RAWHI] = bhi2[0];
        t[R_XLO] = blo2[1];   t[R_XHI] = bhi2[1];
        t[R_WLO] = blo2[2];   t[R_WHI] = bhi2[2];
    }
    const double err = t[R_ERR];
    const double rbar = t[R_RAW] / (double)m;
    const double sum_au = t[R_AU];
    const double dual = st->eps_user * (sum_au + t[R_XB] - 1.0);
    if (mode == STEP_MAP) {
        for (int j = tid; j < m; j += nthr) s_out[j] = st->eps_user * (w.raw[j] - rbar);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->err = err;
            st->dual = dual;
            st->done = 1;
        }
        return;
    }
    double v2[1] = {0.0};
    float wlo[3] = {INFINITY, INFINITY, INFINITY}, whi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (wupd) {
        const double a2 = T[3];
        for (int j = tid; j < m; j += nthr) {
            const double s = w.raw[j] - rbar;
            const double xj = w.x[j];
            const double w1 = (w.w[j] + a2 * xj + 2.0 * s) * inv_1pa;
            w.w1[j] = w1;
            const double v1 = w1 * inv_alpha - xj;
            v2[0] += v1 * v1 * w.D1[j];
            wlo[0] = fminf(wlo[0], lo_f(w1));
            whi[0] = fmaxf(whi[0], hi_f(w1));
        }
    }
    {
        __shared__ double shv[1];
        block_sum_store<1>(v2, shv);
        block_minmax_f(wlo, whi);
        if (threadIdx.x == 0) {
            rec[R_C2R * nb] = shv[0];
            rec[R_W1LO * nb] = wlo[0];
            rec[R_W1HI * nb] = whi[0];
        }
    }
    if (!grid_barrier(st, 2 * nb, kBarrierLimitNs)) { bail(); return; }

    // ---- P3
    double t2[3];
    {
        // one read of every block's record: the P2 sum and bounds (loaded
        // before use, as in P2)
        double c2[1] = {0.0};
        const int op1[1] = {0};
        float wl[3] = {INFINITY, INFINITY, INFINITY}, wh[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int b0 = threadIdx.x; b0 < (int)nb; b0 += kRecPerThread * kVecNT) {
            double rv[kRecPerThread][3];
#pragma unroll
            for (int q = 0; q < kRecPerThread; ++q) {
                const int b = b0 + q * kVecNT;
                if (b < (int)nb) {
                    rv[q][0] = __ldcg(&w.steppart[R_C2R * nb + b]);
                    rv[q][1] = __ldcg(&w.steppart[R_W1LO * nb + b]);
                    rv[q][2] = __ldcg(&w.steppart[R_W1HI * nb + b]);
                }
            }
#pragma unroll
            for (int q = 0; q < kRecPerThread; ++q) {
                if (b0 + q * kVecNT < (int)nb) {
                    c2[0] += rv[q][0];
                    wl[0] = fminf(wl[0], (float)rv[q][1]);
                    wh[0] = fmaxf(wh[0], (float)rv[q][2]);
                }
            }
        }
        block_allreduce<1>(c2, op1);
        block_minmax_f(wl, wh);
        t2[0] = c2[0];
        t2[1] = wl[0];
        t2[2] = wh[0];
    }
    const double c1 = t[R_C1], c2l = t[R_C2L], c2r_sum = t2[0];
    const double kappa1 = T[4];
    const double c1r = kappa1 * st->kl_prev;
    const double c2r = T[5] * c2r_sum;
    int stab_bits = 0;
    if (check) stab_bits = (c1 <= c1r ? 0 : 1) | (c2l <= c2r ? 0 : 2);
    const bool gate = (stab == 2) && (stab_bits != 0);
    const int steps_new = st->steps + 1;
    const bool nonfinite = !isfinite(err);
    const bool converged = err < st->tol;
    const bool stop = converged || nonfinite || steps_new >= st->max_steps;

    double mu_new = mu;
    int ms = st->m_stage, jst = st->j_in_stage, stages = st->stages;
    bool stage_end = false;
    if (wupd) {
        jst += 1;
        // BACKTRACK: a failed stability test ends the stage at once
        if (jst == ms || (stab == 3 && stab_bits != 0)) {
            stage_end = true;
            mu_new = mu / 2.0;
            ms = (int)floor(sqrt(2.0) * (double)ms) + 1;
            jst = 0;
            stages += 1;
        }
    }
    // the next iterate uses the next stage's alpha after a stage change
    const double inv_1pa_new = stage_end ? T[7] : inv_1pa;
    const double ratio = (stage_end && st->carry == 0) ? T[6] : 1.0;
    // bounds of the next iterate from the P1/P2 bounds (all factors > 0)
    const double slo = t[R_RAWLO] - rbar, shi = t[R_RAWHI] - rbar;
    double xlo, xhi;
    if (is_acc) {
        double w1lo, w1hi;
        if (!wupd) { w1lo = t[R_WLO]; w1hi = t[R_WHI]; }
        else if (gate) { w1lo = alpha * t[R_XLO]; w1hi = alpha * t[R_XHI]; }
        else { w1lo = t2[1]; w1hi = t2[2]; }
        xlo = (w1lo * ratio + slo) * inv_1pa_new;
        xhi = (w1hi * ratio + shi) * inv_1pa_new;
    } else {
        xlo = slo;
        xhi = shi;
    }
    // widen by a relative margin that covers the FP64 rounding of the bounds
    xlo -= 1e-12 * (1.0 + fabs(xlo));
    xhi += 1e-12 * (1.0 + fabs(xhi));
    const double eps_c = st->eps_c;
    const double shift_g = st->cabs - eps_c * xlo;
    const double shift_fn = st->cabs - (eps_c * st->min_loga - eps_c * xhi + st->cmin -
                                        eps_c * st->log_m);
    if (!stop) {
        const double k2 = st->k2;
        // two columns at a time, inputs loaded first (as in P1)
        for (int j0 = tid; j0 < m; j0 += 2 * nthr) {
            double rw[2], xj[2], wv[2], dl[2], d1[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j = j0 + u * nthr;
                if (j >= m) continue;
                rw[u] = w.raw[j];
                xj[u] = w.x[j];
                wv[u] = (is_acc && !(wupd && gate)) ? (wupd ? w.w1[j] : w.w[j]) : 0.0;
                dl[u] = w.del[j];
                d1[u] = w.D1[j];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j = j0 + u * nthr;
                if (j >= m) continue;
                const double s = rw[u] - rbar;
                double xn;
                if (is_acc) {
                    double w1 = (wupd && gate) ? alpha * xj[u] : wv[u];
                    w1 *= ratio;
                    xn = (w1 + s) * inv_1pa_new;
                    w.w[j] = w1;
                } else {
                    xn = s;
                }
                w.x_prev[j] = xj[u];
                w.x[j] = xn;
                w.p_prev[j] = dl[u];
                w.D_prev[j] = d1[u];
                write_G(w, j, eps_c * xn + shift_g, kh, k2);
            }
        }
    } else if (is_acc) {
        // stopped at x: keep the momentum after this step's update (gate and
        // stage hand-over applied), the w a continued iteration would use
        for (int j = tid; j < m; j += nthr) {
            const double w1 = wupd ? (gate ? alpha * w.x[j] : w.w1[j]) : w.w[j];
            w.w1[j] = w1 * ratio;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int e = st->steps;
        if (e < st->hist_cap) {
            w.h_err[e] = err;
            w.h_dual[e] = dual;
            w.h_mu[e] = (is_acc && !first) ? mu : 0.0;
            w.h_stab[e] = stab_bits;
            w.h_cond[4 * e + 0] = check ? c1 : 0.0;
            w.h_cond[4 * e + 1] = check ? c1r : 0.0;
            w.h_cond[4 * e + 2] = check ? c2l : 0.0;
            w.h_cond[4 * e + 3] = check ? c2r : 0.0;
        }
        st->last_cond[0] = c1; st->last_cond[1] = c1r;
        st->last_cond[2] = c2l; st->last_cond[3] = c2r;
        st->steps = steps_new;
        st->err = err;
        st->dual = dual;
        st->kl_prev = t[R_KL];
        st->first = 0;
        if (stab_bits) st->failures += 1;
        if (wupd) {
            st->mu = mu_new;
            st->m_stage = ms;
            st->j_in_stage = jst;
            st->stages = stages;
        }
        if (stop) {
            st->done = 1;
            st->status = nonfinite ? 3 : (converged ? 0 : 7);
        } else {
            st->shift_g = shift_g;
            st->shift_f = shift_fn;
        }
        if (st->use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
    }
}

// Failure-path self test of the bounded grid barrier: block 0 never
// arrives (a flag nothing sets), so every other block's wait runs out after
// limit_ns, records ACCSINK_ERR_TIMEOUT in the state and returns; block 0
// returns at once. Used by a test to check the timeout path without a fault.
__global__ void __launch_bounds__(kVecNT) k_barrier_selftest(DevState *st, uint64_t limit_ns)
{
    if (blockIdx.x == 0) return;
    grid_barrier(st, gridDim.x, limit_ns);
}

cudaError_t launch_barrier_selftest(DevState *st, int grid, uint64_t limit_ns, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kVecNT);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_barrier_selftest, st, limit_ns);
}

cudaError_t launch_step(const CostView &cv, const Work &w, int grid, cudaGraphConditionalHandle h,
                        cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kVecNT);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    double *nul = nullptr;
    return cudaLaunchKernelEx(&cfg, k_step, w, cv.n, cv.m, h, nul, nul);
}

cudaError_t launch_step_map(const CostView &cv, const Work &w, int grid, double *c_out,
                            double *s_out, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kVecNT);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaGraphConditionalHandle h = 0;
    return cudaLaunchKernelEx(&cfg, k_step, w, cv.n, cv.m, h, c_out, s_out);
}

// ------------------------------------------------------------------------
// Operand preparation for the single-pass entry points (no normalisation,
// no solve state). prep_g: given g (cost units) and a (and optionally b),
// writes x = g/eps, log a, the shifts and G. prep_f: given f, writes F.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecNT) k_prep_g(Work w, int n, int m, int nstat,
                                                   const double *g, const double *a_in,
                                                   const double *b_in, double eps,
                                                   int scale_max)
{
    DevState *st = w.st;
    const int tid = blockIdx.x * kVecNT + threadIdx.x;
    const int nthr = gridDim.x * kVecNT;
    const uint32_t nb = gridDim.x;
    double cmax, cmin, cabs, bad;
    cost_totals(w.statpart, nstat, cmax, cmin, cabs, bad);
    double gmn = DBL_MAX, gmx = -DBL_MAX, lmn = DBL_MAX;
    for (int j = tid; j < m; j += nthr) {
        const double gj = g[j];
        gmn = fmin(gmn, gj);
        gmx = fmax(gmx, gj);
        w.x[j] = gj / eps;
        if (b_in) {
            w.b[j] = b_in[j];
            w.logb[j] = log(b_in[j]);
        }
    }
    for (int i = tid; i < n; i += nthr) {
        const double ai = a_in ? a_in[i] : 1.0;
        w.a[i] = ai;
        w.loga[i] = log(ai);
        lmn = fmin(lmn, w.loga[i]);
    }
    {
        __shared__ double sh[2];
        block_minmax_store(gmn, gmx, sh);
        double dummy = -DBL_MAX;
        __shared__ double sh2[2];
        block_minmax_store(lmn, dummy, sh2);
        if (threadIdx.x == 0) {
            w.steppart[(int64_t)blockIdx.x * kPartStride + 0] = sh[0];
            w.steppart[(int64_t)blockIdx.x * kPartStride + 1] = sh[1];
            w.steppart[(int64_t)blockIdx.x * kPartStride + 2] = sh2[0];
        }
    }
    if (!grid_barrier(st, nb, kBarrierLimitNs)) return;
    double t[3];
    const int ops[3] = {1, 2, 1};
    grid_totals<3>(w.steppart, nb, 0, ops, t);
    // g is in units of the (possibly scaled) cost; the kernels work in units
    // of the stored cost, i.e. with eps_c = eps * cost_div and G = cost_div g.
    const double cost_div = (scale_max && cmax > 0.0) ? cmax : 1.0;
    const double eps_c = eps * cost_div;
    const double k = kLog2e / eps_c;
    const float kh = (float)k;
    const float kl = (float)(k - (double)kh);
    const double shift_g = cabs - cost_div * t[0];
    const double shift_f =
        cabs - (eps_c * t[2] - cost_div * t[1] + cmin - eps_c * log((double)m));
    for (int j = tid; j < m; j += nthr) write_G(w, j, cost_div * g[j] + shift_g, kh, k);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->eps_c = eps_c;
        st->inv_eps_c = 1.0 / eps_c;
        st->eps_user = eps;
        st->cost_div = cost_div;
        st->cmax = cmax; st->cmin = cmin; st->cabs = cabs;
        st->nonfinite = (bad > 0.0) ? 1 : 0;
        st->shift_g = shift_g;
        st->shift_f = shift_f;
        st->k_hi = kh;
        st->k_lo = kl;
        st->k2 = k;
        st->done = 0;
        st->status = 0;
        st->first = 1;
        st->mode = STEP_MAP;
    }
}

cudaError_t launch_prep_g(const CostView &cv, const Work &w, int grid, const double *g,
                          const double *a_in, double eps, int scale_max, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kVecNT);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const double *b_in = w.b_src;
    return cudaLaunchKernelEx(&cfg, k_prep_g, w, cv.n, cv.m, (int)w.nstat, g, a_in, b_in, eps,
                              scale_max);
}

__global__ void __launch_bounds__(kVecNT) k_prep_f(Work w, int n, int m, int nstat,
                                                   const double *f, double eps, int scale_max)
{
    DevState *st = w.st;
    const int tid = blockIdx.x * kVecNT + threadIdx.x;
    const int nthr = gridDim.x * kVecNT;
    const uint32_t nb = gridDim.x;
    double cmax, cmin, cabs, bad;
    cost_totals(w.statpart, nstat, cmax, cmin, cabs, bad);
    double fmn = DBL_MAX, fmx = -DBL_MAX;
    for (int i = tid; i < n; i += nthr) {
        fmn = fmin(fmn, f[i]);
        fmx = fmax(fmx, f[i]);
    }
    {
        __shared__ double sh[2];
        block_minmax_store(fmn, fmx, sh);
        if (threadIdx.x == 0) {
            w.steppart[(int64_t)blockIdx.x * kPartStride + 0] = sh[0];
            w.steppart[(int64_t)blockIdx.x * kPartStride + 1] = sh[1];
        }
    }
    if (!grid_barrier(st, nb, kBarrierLimitNs)) return;
    double t[1];
    const int ops[1] = {1};
    grid_totals<1>(w.steppart, nb, 0, ops, t);
    const double cost_div = (scale_max && cmax > 0.0) ? cmax : 1.0;
    const double eps_c = eps * cost_div;
    const double k = kLog2e / eps_c;
    const float kh = (float)k;
    const float kl = (float)(k - (double)kh);
    const double shift_f = cabs - cost_div * t[0];
    for (int i = tid; i < n; i += nthr) {
        const double F = cost_div * f[i] + shift_f;
        if (w.Bx64) {
            // point-cloud column operand A'_i = k (F_i - Bx_i) as (hi, lo)
            const double A2 = k * (F - w.Bx64[i]);
            const float Ah = (float)A2;
            w.Fh[i] = Ah;
            w.Fk[i] = (float)(A2 - (double)Ah);
        } else {
            const float Fh = (float)F;
            const float Fl = (float)(F - (double)Fh);
            w.FF[i] = make_float2(Fh, Fl * kh);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->eps_c = eps_c;
        st->inv_eps_c = 1.0 / eps_c;
        st->eps_user = eps;
        st->cost_div = cost_div;
        st->cmax = cmax; st->cmin = cmin; st->cabs = cabs;
        st->nonfinite = (bad > 0.0) ? 1 : 0;
        st->shift_f = shift_f;
        st->k_hi = kh;
        st->k_lo = kl;
        st->k2 = k;
        st->done = 0;
        st->status = 0;
    }
}

cudaError_t launch_prep_f(const CostView &cv, const Work &w, int grid, const double *f,
                          double eps, int scale_max, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kVecNT);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_prep_f, w, cv.n, cv.m, (int)w.nstat, f, eps, scale_max);
}

__global__ void k_scale_out(const double *src, double scale, double *dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] * scale;
}

cudaError_t launch_scale_out(const double *src, double scale, double *dst, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_scale_out<<<(n + 255) / 256, 256, 0, s>>>(src, scale, dst, n);
    return cudaGetLastError();
}

// ell_j = log S_j + (R_j - shift_f) / eps from the column-pass partials.
// When the operand preparation stopped early (its bounded grid barrier ran
// out, so the column pass did not run), the partials are not this call's:
// every ell_j is then NaN.
__global__ void k_col_finish_lse(Work w, int m, double *ell_out)
{
    const DevState *st = w.st;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    if (*(volatile int32_t *)&st->status != 0) {
        ell_out[j] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int splits = st->col_splits;
    const float kh = st->k_hi, kl = st->k_lo;
    float R = w.colpart[j].x;
    for (int q = 1; q < splits; ++q) R = fmaxf(R, w.colpart[(int64_t)q * m + j].x);
    double S = 0.0;
    for (int q = 0; q < splits; ++q) {
        const float2 pr = w.colpart[(int64_t)q * m + j];
        S += (double)pr.y * (double)exp2_scaled(pr.x - R, kh, kl);
    }
    ell_out[j] = log(S) + ((double)R - st->shift_f) * st->inv_eps_c;
}

cudaError_t launch_col_finish_lse(const Work &w, int m, double *ell_out, cudaStream_t s)
{
    k_col_finish_lse<<<(m + 255) / 256, 256, 0, s>>>(w, m, ell_out);
    return cudaGetLastError();
}

}  // namespace accsink

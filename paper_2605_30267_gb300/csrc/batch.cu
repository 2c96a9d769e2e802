// Batched solver kernels: cost formation, scaling and the persistent solve.
//
// The arithmetic of a pass is the single-problem path's, in log2 units on a
// stored double-float cost: with G'_j = k (eps_c x_j + shift_g) and
// K_ij = k C_ij as (hi, lo) pairs, the exponent G'_j - K_ij is formed
// exactly (Fast2Sum on the hi parts, valid because the shift makes
// G' >= k max|C|, plus the lo parts), each row keeps a running maximum R and
// a Kahan pair, lanes merge in double-float and each row finishes in FP64:
//   LSE_j(x_j - C_ij / eps_c) = (R + log2 S) ln 2 - shift_g / eps_c.
// The step is Algorithm 1 + 2 with Theorem 4's test, as in the single-problem
// step kernel, reduced over one CTA.
#include <float.h>

#include "accsink_internal.cuh"
#include "batch_internal.cuh"

namespace accsink {

namespace {

constexpr int kBW = kBatchThreads / 32;            // warps per CTA
constexpr uint64_t kQueueWaitNs = 20000000000ull;  // 20 s for one queue wait

// ---------------------------------------------------------------- helpers --

// Polling load: no ordering (so it does not invalidate this SM's L1 on every
// poll); the waiter issues one acquire fence once the value it waits for
// is seen.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acquire_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int32_t *p)
{
    return *(const volatile int32_t *)p;
}

// The scale k = log2(e) / eps_c of a problem, from its formation statistics.
__device__ __forceinline__ double batch_cost_div(const BatchProb *P)
{
    const double cmax = dec_d(P->cmax_enc);
    return (P->scale && cmax > 0.0) ? cmax : 1.0;
}

__device__ __forceinline__ double batch_k(const BatchProb *P)
{
    return kLog2e / (P->eps * batch_cost_div(P));
}

// CTA-wide sums of N doubles (fixed order); every thread gets the totals.
template <int N>
__device__ __forceinline__ void cta_sum(double (&v)[N])
{
    __shared__ double sh[N][kBW];
    __shared__ double tot[N];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int q = 0; q < kBW; ++q) s += sh[threadIdx.x][q];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = tot[k];
    __syncthreads();
}

// CTA-wide min (lo) and max (hi) of N doubles each.
template <int N>
__device__ __forceinline__ void cta_minmax(double (&lo)[N], double (&hi)[N])
{
    __shared__ double sl[N][kBW], shh[N][kBW];
    __shared__ double tl[N], th[N];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double a = lo[k], b = hi[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { sl[k][wid] = a; shh[k][wid] = b; }
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double a = sl[threadIdx.x][0], b = shh[threadIdx.x][0];
        for (int q = 1; q < kBW; ++q) { a = fmin(a, sl[threadIdx.x][q]); b = fmax(b, shh[threadIdx.x][q]); }
        tl[threadIdx.x] = a;
        th[threadIdx.x] = b;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) { lo[k] = tl[k]; hi[k] = th[k]; }
    __syncthreads();
}

// Writes a double-float (hi, lo) of v.
__device__ __forceinline__ void put_df(float *hp, float *lp, int64_t i, double v)
{
    const float h = (float)v;
    hp[i] = h;
    lp[i] = (float)(v - (double)h);
}

// Loads of per-problem data written during the solve. When another CTA may
// have written it (tiled problems) the load goes to L2 (ld.cg); when this
// CTA owns the whole problem (LOCAL) every write came from this SM, so the
// L1-cached load is coherent and much faster.
template <bool LOCAL, class T>
__device__ __forceinline__ T ldv(const T *p)
{
    if constexpr (LOCAL) return *p;
    else return __ldcg(p);
}

// Lane-tree merge of (R, S, K) accumulators over each aligned segment of L
// lanes (L a power of two; L = 32 is the whole warp) into one double-float
// sum about the segment maximum; every lane of a segment gets (Rw, hi, lo).
__device__ __forceinline__ void seg_merge(const Lse2 &a, int L, float &Rw, float &hi, float &lo)
{
    Rw = a.R;
    for (int o = L >> 1; o > 0; o >>= 1) Rw = fmaxf(Rw, __shfl_xor_sync(0xffffffffu, Rw, o));
    const float sc = (a.R == -INFINITY) ? 0.0f : ex2_approx(a.R - Rw);
    two_sum_f(__fmul_rn(a.S, sc), -__fmul_rn(a.K, sc), hi, lo);
    for (int o = L >> 1; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float s2, e2;
        two_sum_f(hi, ohi, s2, e2);
        lo = lo + olo + e2;
        two_sum_f(s2, lo, hi, lo);
    }
}

// The same double-float tree for a second sum `a` kept about the lane's
// reference R of the first one (Ra) and merged about its segment maximum Rw.
__device__ __forceinline__ void seg_merge_same_r(const Lse2 &a, float Ra, float Rw, int L,
                                                 float &hi, float &lo)
{
    const float sc = (Ra == -INFINITY) ? 0.0f : ex2_approx(Ra - Rw);
    two_sum_f(__fmul_rn(a.S, sc), -__fmul_rn(a.K, sc), hi, lo);
    for (int o = L >> 1; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float s2, e2;
        two_sum_f(hi, ohi, s2, e2);
        lo = lo + olo + e2;
        two_sum_f(s2, lo, hi, lo);
    }
}

// Lanes per row: the smallest power of two covering the row's float4 slots
// (at most 32), so a warp works on 32 / L short rows at once.
__device__ __forceinline__ int seg_lanes(int slots)
{
    int L = 1;
    while (L < slots && L < 32) L <<= 1;
    return L;
}

// ---------------------------------------------------------------- passes --

// Row pass over rows [r0, r1) of problem P: u_i, the column operand F'_i and
// the CTA's partials (sum a u, and with WC the transport cost in K units).
// Scratch of the pass functions (row pass, column tiles, column pass over
// K^T): one buffer for all of them, since a CTA runs one at a time and each
// ends with a CTA barrier after its last read. Per-function arrays would
// take 45 KB per CTA (one set per template instance) and cap residency.
__shared__ __align__(16) float s_pass[3 * kBW * kBatchColTile];
static_assert(5 * kBatchThreads <= 3 * kBW * kBatchColTile, "row-pass scratch does not fit");

// Each warp takes four rows at a time (one operand load serves four rows and
// four rows' loads are in flight); rows go in chunks of one row per thread:
// the warps reduce each row to (R, hi, lo) in shared memory, then every
// thread finishes one row in FP64 (so the slow FP64 pipe works on 32 rows
// per warp instruction).
template <bool WC, bool LOCAL>
__device__ void cta_rows(BatchProb *P, int r0, int r1, double *part2)
{
    constexpr int RW = 4;
    float *sR = s_pass, *sH = s_pass + kBatchThreads, *sL = s_pass + 2 * kBatchThreads;
    float *sCH = s_pass + 3 * kBatchThreads, *sCL = s_pass + 4 * kBatchThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int m = P->m;
    const int64_t ldm = P->ldm;
    const int m4 = (m + 3) >> 2, mfull = m >> 2;
    const double k2 = ldv<LOCAL>(&P->k2), eps_c = ldv<LOCAL>(&P->eps_c);
    const double shift_g = ldv<LOCAL>(&P->shift_g), shift_f = ldv<LOCAL>(&P->shift_f);
    const double inv_eps = ldv<LOCAL>(&P->inv_eps);
    const float4 *G4h = reinterpret_cast<const float4 *>(P->Gh);
    const float4 *G4l = reinterpret_cast<const float4 *>(P->Gl);
    const int L = seg_lanes(m4), sub = lane / L, li = lane % L;
    const int nvw = kBW * (32 / L), vw = wid * (32 / L) + sub;
    double my_dual = 0.0, my_cost = 0.0;
    for (int base = r0; base < r1; base += kBatchThreads) {
        const int rend = min(r1, base + kBatchThreads);
        // Each row is worked by an aligned segment of L lanes; a warp holds
        // 32 / L segments ("virtual warps"), and virtual warp vw takes rows
        // rb + vw + nvw q, q < RW (interleaved, so short tiles still give
        // every warp a row).
        for (int rb = base; rb < rend; rb += RW * nvw) {
            int rq[RW];
            bool ok[RW];
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                rq[q] = rb + vw + nvw * q;
                ok[q] = rq[q] < rend;
            }
            Lse2 acc[RW], cacc[RW];
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                acc[q] = {-INFINITY, 0.0f, 0.0f};
                cacc[q] = {0.0f, 0.0f, 0.0f};
            }
            for (int v = li; v < m4; v += L) {
                const float4 gh = ldv<LOCAL>(G4h + v), gl = ldv<LOCAL>(G4l + v);
                const float ga[4] = {gh.x, gh.y, gh.z, gh.w}, gb[4] = {gl.x, gl.y, gl.z, gl.w};
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                    if (ok[q]) {
                        const int64_t off = (int64_t)rq[q] * ldm;
                        const float4 kh = __ldg(reinterpret_cast<const float4 *>(P->Kh + off) + v);
                        const float4 kl = __ldg(reinterpret_cast<const float4 *>(P->Kl + off) + v);
                        const float ka[4] = {kh.x, kh.y, kh.z, kh.w}, kb[4] = {kl.x, kl.y, kl.z, kl.w};
                        float h[4], l[4], cst[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float hn = ga[e] - ka[e];        // Fast2Sum: |G'| >= |K|
                            const float z = hn - ga[e];
                            l[e] = (gb[e] - kb[e]) + (-ka[e] - z);
                            h[e] = hn;
                            if (WC) cst[e] = ka[e] + kb[e];
                        }
                        if (v >= mfull) {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (4 * v + e >= m) {
                                    h[e] = -INFINITY;
                                    l[e] = 0.0f;
                                    if (WC) cst[e] = 0.0f;
                                }
                        }
                        slot_accumulate<WC>(acc[q], cacc[q], h, l, cst);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                float Rw, hi, lo;
                seg_merge(acc[q], L, Rw, hi, lo);
                float chi = 0.0f, clo = 0.0f;
                if (WC) seg_merge_same_r(cacc[q], acc[q].R, Rw, L, chi, clo);
                if (li == 0 && ok[q]) {
                    const int t = rq[q] - base;
                    sR[t] = Rw;
                    sH[t] = hi;
                    sL[t] = lo;
                    if (WC) { sCH[t] = chi; sCL[t] = clo; }
                }
            }
        }
        __syncthreads();
        const int r = base + threadIdx.x;
        if (r < rend) {
            const int t = threadIdx.x;
            const double S = (double)sH[t] + (double)sL[t];
            const double lse = (double)sR[t] * kLn2 + log(S) - shift_g * inv_eps;
            const double ui = ldv<LOCAL>(&P->loga[r]) - lse;
            P->u[r] = ui;
            put_df(P->Fh, P->Fl, r, k2 * (eps_c * ui + shift_f));
            const double ar = ldv<LOCAL>(&P->a[r]);
            my_dual += ar * ui;
            if (WC) my_cost += ar * (((double)sCH[t] + (double)sCL[t]) / S);
        }
        __syncthreads();
    }
    double v[2] = {my_dual, my_cost};
    cta_sum<2>(v);
    part2[0] = v[0];
    part2[1] = v[1];
}

// Algorithm 1's stage constants for the current mu (see the single-problem
// step kernel's table): alpha = sqrt(2 mu) and its functions.
struct StageK {
    double alpha, inv_alpha, inv_1pa, a2, kappa1, c2f, ratio_next, inv_1pa_next;
};

__device__ __forceinline__ StageK stage_constants(bool is_acc, double mu)
{
    StageK k = {1.0, 1.0, 0.5, -1.0, 0.0, 1.0, 1.0, 0.5};
    if (is_acc) {
        const double alpha = sqrt(2.0 * mu);
        const double an = sqrt(mu);             // alpha of the next stage (mu / 2)
        k.alpha = alpha;
        k.inv_alpha = 1.0 / alpha;
        k.inv_1pa = 1.0 / (1.0 + alpha);
        k.a2 = alpha * alpha - 2.0;
        k.kappa1 = (4.0 - alpha * alpha - 2.0 * sqrt(alpha)) /
                   (2.0 * alpha * (1.0 + alpha) * (1.0 + alpha));
        k.c2f = alpha * sqrt(alpha);
        k.ratio_next = an / alpha;
        k.inv_1pa_next = 1.0 / (1.0 + an);
    }
    return k;
}

// The stage constants computed once by thread 0 and shared with the CTA (FP64
// square roots and divisions are slow on this part; every thread computing
// them costs more than a whole small row pass).
__device__ __forceinline__ StageK cta_stage_constants(bool is_acc, double mu)
{
    __shared__ StageK ks;
    if (threadIdx.x == 0) ks = stage_constants(is_acc, mu);
    __syncthreads();
    const StageK k = ks;
    __syncthreads();
    return k;
}

// Step phase P1 for column j, given ell_j from the column pass: p = log(c/b),
// raw_j = x_j - p (the v-update), c_j - b_j, D_j, the KL term and Theorem 4's
// Cond 1 / Cond 2 left-hand terms; adds to the sums v and the bounds.
template <bool LOCAL>
__device__ __forceinline__ void p1_column(BatchProb *P, int j, double ell, double inv_alpha,
                                          bool check, double (&v)[6], double (&lo3)[3],
                                          double (&hi3)[3])
{
    const double xj = ldv<LOCAL>(&P->x[j]);
    const double bj = ldv<LOCAL>(&P->b[j]);
    const double wj = ldv<LOCAL>(&P->w[j]);
    const double del = xj + ell - ldv<LOCAL>(&P->logb[j]);
    const double raw = xj - del;
    double xi, D1, klt;
    const float dl = (float)del;
    if (fabsf(dl) <= 80.0f) {
        const float e = expm1f(dl);
        float km;
        if (fabsf(dl) < 0.0625f) {
            km = dl * dl * fmaf(dl, fmaf(dl, fmaf(dl, fmaf(dl, 1.0f / 720.0f, 1.0f / 120.0f),
                                                 1.0f / 24.0f), 1.0f / 6.0f), 0.5f);
        } else {
            km = e - dl;
        }
        const float dr = (dl != 0.0f) ? e / dl : 1.0f;
        xi = bj * (double)e;
        D1 = bj * (double)dr;
        klt = bj * (double)km;
    } else {
        const double e = expm1(del);
        xi = bj * e;
        D1 = xi / del;
        klt = bj * (e - del);
    }
    v[0] += fabs(xi);
    v[1] += raw;
    v[2] += klt;
    v[3] += bj * xj;
    if (check) {
        const double p0 = ldv<LOCAL>(&P->p_prev[j]);
        const double v0 = wj * inv_alpha - ldv<LOCAL>(&P->x_prev[j]);
        v[4] += p0 * p0 * D1;
        v[5] += v0 * v0 * (D1 - ldv<LOCAL>(&P->D_prev[j]));
    }
    lo3[0] = fmin(lo3[0], raw); hi3[0] = fmax(hi3[0], raw);
    lo3[1] = fmin(lo3[1], xj);  hi3[1] = fmax(hi3[1], xj);
    lo3[2] = fmin(lo3[2], wj);  hi3[2] = fmax(hi3[2], wj);
    P->raw[j] = raw;
    P->D1[j] = D1;
    P->del[j] = del;
}

// Column pass over columns [c0, c0 + 128) of problem P: ell_j. Each lane owns
// four columns, warps split the rows in groups of four, and the warps'
// accumulators are merged per column in a fixed order.
template <bool LOCAL>
__device__ void cta_cols(BatchProb *P, int tile, const StageK &K, bool check, double (&wsum)[6],
                         double (&lo3)[3], double (&hi3)[3])
{
    const int c0 = tile * kBatchColTile;
    float(*sR)[kBatchColTile] = reinterpret_cast<float(*)[kBatchColTile]>(s_pass);
    float(*sH)[kBatchColTile] = reinterpret_cast<float(*)[kBatchColTile]>(s_pass + kBW * kBatchColTile);
    float(*sL)[kBatchColTile] =
        reinterpret_cast<float(*)[kBatchColTile]>(s_pass + 2 * kBW * kBatchColTile);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n = P->n, m = P->m;
    const int64_t ldm = P->ldm;
    const int cb = c0 + 4 * lane;
    const bool any = cb < m;
    Lse2 acc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] = {-INFINITY, 0.0f, 0.0f};
    if (any) {
        for (int rg = 4 * wid; rg < n; rg += 4 * kBW) {
            float h[4][4], l[4][4];     // [column][row]
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rg + q;
                if (r < n) {
                    const float4 kh = __ldg(reinterpret_cast<const float4 *>(P->Kh + (int64_t)r * ldm + cb));
                    const float4 kl = __ldg(reinterpret_cast<const float4 *>(P->Kl + (int64_t)r * ldm + cb));
                    const float fh = ldv<LOCAL>(P->Fh + r), fl = ldv<LOCAL>(P->Fl + r);
                    const float ka[4] = {kh.x, kh.y, kh.z, kh.w}, kb[4] = {kl.x, kl.y, kl.z, kl.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float hn = fh - ka[e];
                        const float z = hn - fh;
                        l[e][q] = (fl - kb[e]) + (-ka[e] - z);
                        h[e][q] = hn;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) { h[e][q] = -INFINITY; l[e][q] = 0.0f; }
                }
            }
            float dummy[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                Lse2 none;
                slot_accumulate<false>(acc[e], none, h[e], l[e], dummy);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float hi, lo;
        two_sum_f(acc[e].S, -acc[e].K, hi, lo);
        sR[wid][4 * lane + e] = acc[e].R;
        sH[wid][4 * lane + e] = hi;
        sL[wid][4 * lane + e] = lo;
    }
    __syncthreads();
    // per column: merge the warps, finish ell_j and run step phase P1 on it
    // here, so the step's per-column FP64 work is spread over the tiles. The
    // P1 sums of the columns a warp finished are reduced over its lanes (fixed
    // tree) and added to that warp's running sums `wsum`; the bounds stay
    // per thread (the caller reduces them).
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (threadIdx.x < kBatchColTile) {
        const int t = threadIdx.x, c = c0 + t;
        if (c < m) {
            float R = -INFINITY;
            for (int q = 0; q < kBW; ++q) R = fmaxf(R, sR[q][t]);
            double S = 0.0;
            for (int q = 0; q < kBW; ++q) {
                if (sR[q][t] == -INFINITY) continue;
                const double f = (double)ex2_approx(sR[q][t] - R);
                S += ((double)sH[q][t] + (double)sL[q][t]) * f;
            }
            const double shift_f = ldv<LOCAL>(&P->shift_f), inv_eps = ldv<LOCAL>(&P->inv_eps);
            const double ell = (double)R * kLn2 + log(S) - shift_f * inv_eps;
            P->ell[c] = ell;
            p1_column<LOCAL>(P, c, ell, K.inv_alpha, check, v, lo3, hi3);
        }
    }
    if (threadIdx.x < kBatchColTile) {
#pragma unroll
        for (int q = 0; q < 6; ++q) wsum[q] += warp_sum(v[q]);
    }
    __syncthreads();
}

// Column pass over K^T rows [j0, j1) (columns of K) of a large problem: the
// same warp-per-row log-sum-exp as the row pass with F' as the operand, then
// per thread one column's ell_j and step phase P1. Each warp's 32 columns are
// summed over lanes (the tree of the strip column pass) and written, with
// their bounds, to that warp's slot of its 128-column group's record. j0 is a
// multiple of 32.
__device__ void cta_colsT(BatchProb *P, int j0, int j1, const StageK &K, bool check)
{
    constexpr int RW = 4;
    float *sR = s_pass, *sH = s_pass + kBatchThreads, *sL = s_pass + 2 * kBatchThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n = P->n;
    const int64_t ldn = P->ldn;
    const int n4 = (n + 3) >> 2, nfull = n >> 2;
    const double shift_f = __ldcg(&P->shift_f), inv_eps = __ldcg(&P->inv_eps);
    const float4 *F4h = reinterpret_cast<const float4 *>(P->Fh);
    const float4 *F4l = reinterpret_cast<const float4 *>(P->Fl);
    const int L = seg_lanes(n4), sub = lane / L, li = lane % L;
    const int nvw = kBW * (32 / L), vw = wid * (32 / L) + sub;
    for (int base = j0; base < j1; base += kBatchThreads) {
        const int jend = min(j1, base + kBatchThreads);
        for (int jb = base; jb < jend; jb += RW * nvw) {
            int jq[RW];
            bool ok[RW];
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                jq[q] = jb + vw + nvw * q;
                ok[q] = jq[q] < jend;
            }
            Lse2 acc[RW];
#pragma unroll
            for (int q = 0; q < RW; ++q) acc[q] = {-INFINITY, 0.0f, 0.0f};
            for (int v = li; v < n4; v += L) {
                const float4 fh = __ldcg(F4h + v), fl = __ldcg(F4l + v);
                const float fa[4] = {fh.x, fh.y, fh.z, fh.w}, fb[4] = {fl.x, fl.y, fl.z, fl.w};
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                    if (ok[q]) {
                        const int64_t off = (int64_t)jq[q] * ldn;
                        const float4 kh = __ldg(reinterpret_cast<const float4 *>(P->KTh + off) + v);
                        const float4 kl = __ldg(reinterpret_cast<const float4 *>(P->KTl + off) + v);
                        const float ka[4] = {kh.x, kh.y, kh.z, kh.w}, kb[4] = {kl.x, kl.y, kl.z, kl.w};
                        float h[4], l[4], dummy[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float hn = fa[e] - ka[e];        // Fast2Sum: |F'| >= |K|
                            const float z = hn - fa[e];
                            l[e] = (fb[e] - kb[e]) + (-ka[e] - z);
                            h[e] = hn;
                        }
                        if (v >= nfull) {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (4 * v + e >= n) { h[e] = -INFINITY; l[e] = 0.0f; }
                        }
                        Lse2 none;
                        slot_accumulate<false>(acc[q], none, h, l, dummy);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                float Rw, hi, lo;
                seg_merge(acc[q], L, Rw, hi, lo);
                if (li == 0 && ok[q]) {
                    const int t = jq[q] - base;
                    sR[t] = Rw;
                    sH[t] = hi;
                    sL[t] = lo;
                }
            }
        }
        __syncthreads();
        // finish one column per thread, then per-warp P1 sums and bounds
        double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double lo3[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi3[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
        const int c = base + threadIdx.x;
        if (c < jend) {
            const int t = threadIdx.x;
            const double S = (double)sH[t] + (double)sL[t];
            const double ell = (double)sR[t] * kLn2 + log(S) - shift_f * inv_eps;
            P->ell[c] = ell;
            p1_column<false>(P, c, ell, K.inv_alpha, check, v, lo3, hi3);
        }
        double ws[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) ws[q] = warp_sum(v[q]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            double a = lo3[q], b = hi3[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
                b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
            }
            lo3[q] = a;
            hi3[q] = b;
        }
        // this warp's 32 columns lie in one 128-column group (items start on
        // multiples of 32); write its slot of that group's record if the
        // columns are this item's
        const int c0w = base + 32 * wid;
        if (lane == 0 && c0w < jend) {
            const int group = c0w / kBatchColTile, slot = (c0w % kBatchColTile) / 32;
            double *r = P->colrec + (int64_t)group * kBatchColRec + 12 * slot;
            for (int q = 0; q < 6; ++q) r[q] = ws[q];
            for (int q = 0; q < 3; ++q) { r[6 + q] = lo3[q]; r[9 + q] = hi3[q]; }
        }
        __syncthreads();
    }
}

// Writes record `rec`: each finishing warp's P1 sums and bounds (the bounds
// reduced over the warp's lanes).
__device__ void cta_colrec(BatchProb *P, int rec, const double (&wsum)[6], double (&lo3)[3],
                           double (&hi3)[3])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double a = lo3[q], b = hi3[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        lo3[q] = a;
        hi3[q] = b;
    }
    if (lane == 0 && wid < kBatchColWarps) {
        double *r = P->colrec + (int64_t)rec * kBatchColRec + 12 * wid;
        for (int q = 0; q < 6; ++q) r[q] = wsum[q];
        for (int q = 0; q < 3; ++q) { r[6 + q] = lo3[q]; r[9 + q] = hi3[q]; }
    }
    __syncthreads();
}

// ------------------------------------------------------------ init, step --

// Validates and normalises the marginals, derives eps_c, k and the operand
// shifts, and writes x_0 = w_0 = 0 with its operand G'. Returns false (and
// records the status) for invalid inputs.
__device__ bool cta_init(BatchProb *P)
{
    __shared__ int st_s;
    const int n = P->n, m = P->m;
    const double cmax = dec_d(P->cmax_enc), cmin = dec_d(P->cmin_enc), cabs = dec_d(P->cabs_enc);
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // sum a, sum b, #a<=0, #b<=0, #nonfinite
    for (int i = threadIdx.x; i < n; i += kBatchThreads) {
        const double ai = P->a_in[i];
        v[0] += ai;
        if (!(ai > 0.0)) v[2] += 1.0;
        if (!isfinite(ai)) v[4] += 1.0;
    }
    for (int j = threadIdx.x; j < m; j += kBatchThreads) {
        const double bj = P->b_in[j];
        v[1] += bj;
        if (!(bj > 0.0)) v[3] += 1.0;
        if (!isfinite(bj)) v[4] += 1.0;
    }
    cta_sum<5>(v);
    if (threadIdx.x == 0) {
        int status = 0;
        if (P->nonfinite & 2u) status = 6;    // ACCSINK_ERR_TIMEOUT in the formation
        else if (P->nonfinite || v[4] > 0.0 || !isfinite(cmax) || !isfinite(cmin)) status = 3;
        else if (v[2] > 0.0 || v[3] > 0.0) status = 2;
        else if (P->scale && !(cmax > 0.0)) status = 1;
        st_s = status;
        if (status) { P->status = status; P->cmax = cmax; }
    }
    __syncthreads();
    if (st_s != 0) return false;
    const double sa = v[0], sb = v[1];
    const double cost_div = batch_cost_div(P);
    const double eps_c = P->eps * cost_div;
    const double k2 = batch_k(P);
    double mn[1] = {DBL_MAX}, mx[1] = {-DBL_MAX};
    for (int i = threadIdx.x; i < n; i += kBatchThreads) {
        const double ai = P->a_in[i] / sa;
        const double la = log(ai);
        P->a[i] = ai;
        P->loga[i] = la;
        mn[0] = fmin(mn[0], la);
    }
    cta_minmax<1>(mn, mx);
    const double min_loga = mn[0];
    const double log_m = log((double)m);
    const double shift_g = cabs;
    const double shift_f = cabs - (eps_c * min_loga + cmin - eps_c * log_m);
    // record slots of the last 128-column group that no column reaches (the
    // transposed column pass never writes them): neutral sums and bounds
    if (P->KTh && threadIdx.x < kBatchColWarps) {
        const int w = threadIdx.x, g = P->col_tiles - 1;
        if (g * kBatchColTile + 32 * w >= m) {
            double *r = P->colrec + (int64_t)g * kBatchColRec + 12 * w;
            for (int q = 0; q < 6; ++q) r[q] = 0.0;
            for (int q = 0; q < 3; ++q) { r[6 + q] = DBL_MAX; r[9 + q] = -DBL_MAX; }
        }
    }
    for (int j = threadIdx.x; j < m; j += kBatchThreads) {
        const double bj = P->b_in[j] / sb;
        P->b[j] = bj;
        P->logb[j] = log(bj);
        P->x[j] = 0.0;
        P->x_prev[j] = 0.0;
        P->w[j] = 0.0;
        P->p_prev[j] = 0.0;
        P->D_prev[j] = bj;
        put_df(P->Gh, P->Gl, j, k2 * shift_g);
    }
    if (threadIdx.x == 0) {
        P->k2 = k2;
        P->eps_c = eps_c;
        P->inv_eps = 1.0 / eps_c;
        P->cost_div = cost_div;
        P->cmax = cmax; P->cmin = cmin; P->cabs = cabs;
        P->min_loga = min_loga;
        P->log_m = log_m;
        P->shift_g = shift_g;
        P->shift_f = shift_f;
        P->mu = P->mu0;
        P->m_stage = P->m0;
        P->j_in_stage = 0;
        P->steps = 0; P->stages = 0; P->failures = 0;
        P->first = 1; P->status = 0; P->done = 0;
        P->err = INFINITY; P->dual = 0.0; P->kl_prev = 0.0; P->cost = NAN;
    }
    __syncthreads();
    return true;
}

// One step after the row and column passes at x (see the single-problem step
// kernel for the phases P1-P3; P1 ran in the column tiles, which left `nrec`
// records of sums and bounds). Returns true when the solve stops.
// ---- the step of Algorithm 1, in pieces: cta_step runs them all in one CTA;
// large problems run the per-column loops (P2, the update) as work items.

// P1 totals from the column records (per finishing warp in record order, then
// over the warps: the same order for every work split) and the dual.
struct StepP1 {
    double v[6];                 // err, raw, kl, <b,x>, c1, c2l
    double lo3[3], hi3[3];       // bounds of raw, x, w
    double err, rbar, dual;
};

template <bool LOCAL>
__device__ void step_p1(BatchProb *P, int nrec, StepP1 &o)
{
    const int m = P->m;
    {
        __shared__ double tot_s[12];
        if (threadIdx.x < 12) {
            const int q = threadIdx.x;
            double a;
            if (q < 6) {
                a = 0.0;
                for (int w = 0; w < kBatchColWarps; ++w) {
                    double aw = 0.0;
                    for (int t = 0; t < nrec; ++t)
                        aw += ldv<LOCAL>(&P->colrec[(int64_t)t * kBatchColRec + 12 * w + q]);
                    a += aw;
                }
            } else {
                const bool mn = q < 9;
                a = mn ? DBL_MAX : -DBL_MAX;
                for (int t = 0; t < nrec; ++t)
                    for (int w = 0; w < kBatchColWarps; ++w) {
                        const double r = ldv<LOCAL>(&P->colrec[(int64_t)t * kBatchColRec + 12 * w + q]);
                        a = mn ? fmin(a, r) : fmax(a, r);
                    }
            }
            tot_s[q] = a;
        }
        __syncthreads();
        for (int q = 0; q < 6; ++q) o.v[q] = tot_s[q];
        for (int q = 0; q < 3; ++q) { o.lo3[q] = tot_s[6 + q]; o.hi3[q] = tot_s[9 + q]; }
        __syncthreads();
    }
    o.err = o.v[0];
    o.rbar = o.v[1] / (double)m;
    double au[1] = {0.0};
    {
        const int rt = P->row_tiles;
        for (int t = threadIdx.x; t < rt; t += kBatchThreads) au[0] += ldv<LOCAL>(&P->rowpart[2 * t]);
        cta_sum<1>(au);
    }
    o.dual = P->eps * (au[0] + o.v[3] - 1.0);
}

// P2 over columns [j0, j1): w1 = (w + (alpha^2 - 2) x + 2 s) / (1 + alpha),
// Theorem 4's sum_j v1_j^2 D1_j and the bounds of w1 (CTA totals).
template <bool LOCAL>
__device__ void step_p2(BatchProb *P, int j0, int j1, double rbar, const StageK &K, double &v2,
                        double &wl, double &wh)
{
    double v2a[1] = {0.0};
    double wla[1] = {DBL_MAX}, wha[1] = {-DBL_MAX};
    for (int j = j0 + threadIdx.x; j < j1; j += kBatchThreads) {
        const double s = ldv<LOCAL>(&P->raw[j]) - rbar;
        const double xj = ldv<LOCAL>(&P->x[j]);
        const double w1 = (ldv<LOCAL>(&P->w[j]) + K.a2 * xj + 2.0 * s) * K.inv_1pa;
        P->w1[j] = w1;
        const double v1 = w1 * K.inv_alpha - xj;
        v2a[0] += v1 * v1 * ldv<LOCAL>(&P->D1[j]);
        wla[0] = fmin(wla[0], w1);
        wha[0] = fmax(wha[0], w1);
    }
    cta_sum<1>(v2a);
    cta_minmax<1>(wla, wha);
    v2 = v2a[0];
    wl = wla[0];
    wh = wha[0];
}

// P3: the scalar decisions (stop, gate, stage hand-over, operand shifts).
struct P3 {
    double inv_1pa_new, ratio, shift_g, shift_fn, mu_new;
    int stab_bits, gate, stop, steps_new, ms, jst, stages, status;
};

template <bool LOCAL>
__device__ P3 step_p3(BatchProb *P, const StepP1 &o, const StageK &K, double mu, bool is_acc,
                      bool wupd, bool check, double v2, double wl, double wh)
{
    __shared__ P3 p3s;
    const int stab = P->stability;
    if (threadIdx.x == 0) {
        P3 r;
        const double c1 = o.v[4], c2l = o.v[5];
        const double c1r = K.kappa1 * ldv<LOCAL>(&P->kl_prev);
        const double c2r = K.c2f * v2;
        r.stab_bits = 0;
        if (check) r.stab_bits = (c1 <= c1r ? 0 : 1) | (c2l <= c2r ? 0 : 2);
        r.gate = (stab == 2) && (r.stab_bits != 0);
        r.steps_new = ldv<LOCAL>(&P->steps) + 1;
        const bool nonfinite = !isfinite(o.err);
        const bool converged = o.err < P->tol;
        r.stop = converged || nonfinite || r.steps_new >= P->max_steps;
        r.status = nonfinite ? 3 : (converged ? 0 : 7);
        r.mu_new = mu;
        r.ms = ldv<LOCAL>(&P->m_stage);
        r.jst = ldv<LOCAL>(&P->j_in_stage);
        r.stages = ldv<LOCAL>(&P->stages);
        bool stage_end = false;
        if (wupd) {
            r.jst += 1;
            // BACKTRACK: a failed stability test ends the stage at once
            if (r.jst == r.ms || (stab == 3 && r.stab_bits != 0)) {
                stage_end = true;
                r.mu_new = mu / 2.0;
                r.ms = (int)floor(sqrt(2.0) * (double)r.ms) + 1;
                r.jst = 0;
                r.stages += 1;
            }
        }
        r.inv_1pa_new = stage_end ? K.inv_1pa_next : K.inv_1pa;
        r.ratio = (stage_end && P->carry == 0) ? K.ratio_next : 1.0;
        const double slo = o.lo3[0] - o.rbar, shi = o.hi3[0] - o.rbar;
        double xlo, xhi;
        if (is_acc) {
            double w1lo, w1hi;
            if (!wupd) { w1lo = o.lo3[2]; w1hi = o.hi3[2]; }
            else if (r.gate) { w1lo = K.alpha * o.lo3[1]; w1hi = K.alpha * o.hi3[1]; }
            else { w1lo = wl; w1hi = wh; }
            xlo = (w1lo * r.ratio + slo) * r.inv_1pa_new;
            xhi = (w1hi * r.ratio + shi) * r.inv_1pa_new;
        } else {
            xlo = slo;
            xhi = shi;
        }
        // widen by a relative margin that covers the FP64 rounding of the bounds
        xlo -= 1e-12 * (1.0 + fabs(xlo));
        xhi += 1e-12 * (1.0 + fabs(xhi));
        const double eps_c = P->eps_c;
        r.shift_g = P->cabs - eps_c * xlo;
        r.shift_fn = P->cabs - (eps_c * P->min_loga - eps_c * xhi + P->cmin - eps_c * P->log_m);
        p3s = r;
    }
    __syncthreads();
    const P3 r = p3s;
    __syncthreads();
    return r;
}

// The update over columns [j0, j1): x+, w+ (Algorithm 1), the previous
// iterate's records for Theorem 4, and the row-pass operand G'.
template <bool LOCAL>
__device__ void step_update(BatchProb *P, int j0, int j1, bool is_acc, bool wupd, bool gate,
                            double alpha, double ratio, double inv_1pa_new, double rbar,
                            double shift_g)
{
    const double eps_c = P->eps_c, k2 = P->k2;
    for (int j = j0 + threadIdx.x; j < j1; j += kBatchThreads) {
        const double s = ldv<LOCAL>(&P->raw[j]) - rbar;
        const double xj = ldv<LOCAL>(&P->x[j]);
        double xn;
        if (is_acc) {
            double w1 = wupd ? (gate ? alpha * xj : ldv<LOCAL>(&P->w1[j])) : ldv<LOCAL>(&P->w[j]);
            w1 *= ratio;
            xn = (w1 + s) * inv_1pa_new;
            P->w[j] = w1;
        } else {
            xn = s;
        }
        P->x_prev[j] = xj;
        P->x[j] = xn;
        P->p_prev[j] = ldv<LOCAL>(&P->del[j]);
        P->D_prev[j] = ldv<LOCAL>(&P->D1[j]);
        put_df(P->Gh, P->Gl, j, k2 * (eps_c * xn + shift_g));
    }
}

// The per-problem state after a step (thread 0); returns the stop flag to the CTA.
__device__ bool step_tail(BatchProb *P, const P3 &r, const StepP1 &o, bool wupd)
{
    __shared__ int stop_s;
    if (threadIdx.x == 0) {
        P->steps = r.steps_new;
        P->err = o.err;
        P->dual = o.dual;
        P->kl_prev = o.v[2];
        P->first = 0;
        if (r.stab_bits) P->failures += 1;
        if (wupd) {
            P->mu = r.mu_new;
            P->m_stage = r.ms;
            P->j_in_stage = r.jst;
            P->stages = r.stages;
        }
        if (r.stop) {
            P->status = r.status;
        } else {
            P->shift_g = r.shift_g;
            P->shift_f = r.shift_fn;
        }
        stop_s = r.stop ? 1 : 0;
    }
    __syncthreads();
    return stop_s != 0;
}

template <bool LOCAL>
__device__ bool cta_step(BatchProb *P, int nrec)
{
    const int m = P->m;
    const int first = ldv<LOCAL>(&P->first);
    const double mu = ldv<LOCAL>(&P->mu);
    const bool is_acc = P->method == 1;
    const StageK K = cta_stage_constants(is_acc, mu);
    const bool check = is_acc && !first && P->stability != 0;
    const bool wupd = is_acc && !first;
    StepP1 o;
    step_p1<LOCAL>(P, nrec, o);
    double v2 = 0.0, wl = DBL_MAX, wh = -DBL_MAX;
    if (wupd) step_p2<LOCAL>(P, 0, m, o.rbar, K, v2, wl, wh);
    const P3 r = step_p3<LOCAL>(P, o, K, mu, is_acc, wupd, check, v2, wl, wh);
    if (!r.stop)
        step_update<LOCAL>(P, 0, m, is_acc, wupd, r.gate, K.alpha, r.ratio, r.inv_1pa_new, o.rbar,
                           r.shift_g);
    __syncthreads();
    return step_tail(P, r, o, wupd);
}

// ---- a large problem's step as work items (every read of data another CTA
// wrote goes to L2: LOCAL = false)

// After the last column item: the P1 totals, kept in the problem record for
// the CTA that finishes the P2 items. Returns true when P2 items follow.
__device__ bool split_step_begin(BatchProb *P)
{
    StepP1 o;
    step_p1<false>(P, P->col_tiles, o);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 6; ++q) P->s_v[q] = o.v[q];
        for (int q = 0; q < 3; ++q) { P->s_lo3[q] = o.lo3[q]; P->s_hi3[q] = o.hi3[q]; }
        P->s_err = o.err;
        P->s_rbar = o.rbar;
        P->s_dual = o.dual;
    }
    __syncthreads();
    return P->method == 1 && !__ldcg(&P->first);
}

// One P2 item: its columns' w1 and its record (v2, min w1, max w1).
__device__ void split_step_p2(BatchProb *P, int item)
{
    const double mu = __ldcg(&P->mu);
    const StageK K = cta_stage_constants(true, mu);
    const int j0 = item * P->step_cols, j1 = min(P->m, j0 + P->step_cols);
    double v2, wl, wh;
    step_p2<false>(P, j0, j1, __ldcg(&P->s_rbar), K, v2, wl, wh);
    if (threadIdx.x == 0) {
        P->p2rec[3 * item] = v2;
        P->p2rec[3 * item + 1] = wl;
        P->p2rec[3 * item + 2] = wh;
    }
}

// After the P2 items (or at once when the step has none): the P2 totals in
// item order, the scalar decisions and the new state; the update's scalars
// go to the problem record for the update items. Returns the stop flag.
__device__ bool split_step_decide(BatchProb *P, bool wupd)
{
    StepP1 o;
    for (int q = 0; q < 6; ++q) o.v[q] = __ldcg(&P->s_v[q]);
    for (int q = 0; q < 3; ++q) { o.lo3[q] = __ldcg(&P->s_lo3[q]); o.hi3[q] = __ldcg(&P->s_hi3[q]); }
    o.err = __ldcg(&P->s_err);
    o.rbar = __ldcg(&P->s_rbar);
    o.dual = __ldcg(&P->s_dual);
    const double mu = __ldcg(&P->mu);
    const bool is_acc = P->method == 1;
    const StageK K = cta_stage_constants(is_acc, mu);
    const bool check = wupd && P->stability != 0;
    double v2 = 0.0, wl = DBL_MAX, wh = -DBL_MAX;
    if (wupd) {
        for (int t = 0; t < P->step_items; ++t) {
            v2 += __ldcg(&P->p2rec[3 * t]);
            wl = fmin(wl, __ldcg(&P->p2rec[3 * t + 1]));
            wh = fmax(wh, __ldcg(&P->p2rec[3 * t + 2]));
        }
    }
    const P3 r = step_p3<false>(P, o, K, mu, is_acc, wupd, check, v2, wl, wh);
    if (threadIdx.x == 0) {
        P->u_alpha = K.alpha;
        P->u_ratio = r.ratio;
        P->u_inv1pa = r.inv_1pa_new;
        P->u_wupd = wupd ? 1 : 0;
        P->u_gate = r.gate;
    }
    return step_tail(P, r, o, wupd);
}

// One update item: x, w and G' for its columns.
__device__ void split_step_update(BatchProb *P, int item)
{
    const int j0 = item * P->step_cols, j1 = min(P->m, j0 + P->step_cols);
    step_update<false>(P, j0, j1, P->method == 1, __ldcg(&P->u_wupd) != 0, __ldcg(&P->u_gate) != 0,
                       __ldcg(&P->u_alpha), __ldcg(&P->u_ratio), __ldcg(&P->u_inv1pa),
                       __ldcg(&P->s_rbar), __ldcg(&P->shift_g));
}

// Outputs of a finished problem: f = eps u, g = eps x, the result record.
template <bool LOCAL>
__device__ void cta_finish(BatchProb *P, BatchResult *R, bool ok)
{
    const int n = P->n, m = P->m;
    const double eps = P->eps;
    if (ok) {
        for (int i = threadIdx.x; i < n; i += kBatchThreads) P->f_out[i] = eps * ldv<LOCAL>(&P->u[i]);
        for (int j = threadIdx.x; j < m; j += kBatchThreads) P->g_out[j] = eps * ldv<LOCAL>(&P->x[j]);
    }
    double c[1] = {0.0};
    if (ok && P->evaluate) {
        for (int t = threadIdx.x; t < P->row_tiles; t += kBatchThreads)
            c[0] += ldv<LOCAL>(&P->rowpart[2 * t + 1]);
    }
    cta_sum<1>(c);
    if (threadIdx.x == 0) {
        R->status = P->status;
        R->steps = ok ? P->steps : 0;
        R->stages = ok ? P->stages : 0;
        R->failures = ok ? P->failures : 0;
        R->marginal_l1 = ok ? P->err : NAN;
        R->transport_cost = (ok && P->evaluate) ? c[0] / (P->k2 * P->cost_div) : NAN;
        R->dual = ok ? P->dual : NAN;
        R->cost_max = P->cmax;
        P->done = 1;
    }
    __syncthreads();
}

// Publishes a finished problem's result to the host-mapped copy (when the
// launch has one): every thread's output writes are made visible first, then
// thread 0 writes the record and, after a system-scope fence, the flag.
__device__ void publish_early(BatchQueue *q, int p, const BatchResult *R)
{
    if (!q->early) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        q->early[p] = *R;
        __threadfence_system();
        *(volatile int32_t *)&q->early_flag[p] = 1;
    }
    __syncthreads();
}

// ----------------------------------------------------------------- queue --

// Pops one item (thread 0). Returns false when the batch is finished or a
// wait ran out.
__device__ bool q_pop(BatchQueue *q, unsigned long long &item)
{
    const unsigned long long pos = atomicAdd(&q->head, 1ull);
    const unsigned long long slot = pos & (q->cap - 1);
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        const unsigned long long s = ld_relaxed_u64(&q->seq[slot]);
        if (s == pos + 1) break;
        if (ld_volatile_i32(&q->all_done)) return false;
        if (globaltimer_ns() - t0 > kQueueWaitNs) {
            atomicExch(&q->error, 6 /* ACCSINK_ERR_TIMEOUT */);
            atomicExch(&q->all_done, 1);
            return false;
        }
        __nanosleep(200);
    }
    fence_acquire_gpu();
    item = *(volatile unsigned long long *)&q->items[slot];
    st_release_u64(&q->seq[slot], pos + q->cap);
    return true;
}

// Pushes k items (all threads of the CTA call it; item(t) gives item t).
template <class F>
__device__ void q_push(BatchQueue *q, int k, F item)
{
    __shared__ unsigned long long base_s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) base_s = atomicAdd(&q->tail, (unsigned long long)k);
    __syncthreads();
    const unsigned long long base = base_s;
    for (int t = threadIdx.x; t < k; t += kBatchThreads) {
        const unsigned long long pos = base + t;
        const unsigned long long slot = pos & (q->cap - 1);
        const uint64_t t0 = globaltimer_ns();
        bool ok = true;
        while (ld_relaxed_u64(&q->seq[slot]) != pos) {
            if (globaltimer_ns() - t0 > kQueueWaitNs || ld_volatile_i32(&q->all_done)) {
                atomicExch(&q->error, 6);
                atomicExch(&q->all_done, 1);
                ok = false;
                break;
            }
            __nanosleep(200);
        }
        if (!ok) continue;
        *(volatile unsigned long long *)&q->items[slot] = item(t);
        st_release_u64(&q->seq[slot], pos + 1);
    }
    __syncthreads();
}

// Arrival at the end of a phase tile; true for the last of `ntiles`.
__device__ bool arrive_last(BatchProb *P, int ntiles)
{
    __shared__ int last_s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int old = atomicAdd(&P->arrive, 1);
        const bool last = old == ntiles - 1;
        if (last) {
            P->arrive = 0;
            __threadfence();
        }
        last_s = last ? 1 : 0;
    }
    __syncthreads();
    return last_s != 0;
}

__device__ void problem_done(BatchQueue *q)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int d = atomicAdd(&q->done_count, 1) + 1;
        if (d == q->count) atomicExch(&q->all_done, 1);
    }
    __syncthreads();
}

}  // namespace

// ------------------------------------------------------- cost formation --

// Lexicographic max / min of normalised double-float pairs (numeric order).
__device__ __forceinline__ void df_max(float &mh, float &ml, float h, float l)
{
    if (h > mh || (h == mh && l > ml)) { mh = h; ml = l; }
}

__device__ __forceinline__ void df_min(float &mh, float &ml, float h, float l)
{
    if (h < mh || (h == mh && l < ml)) { mh = h; ml = l; }
}

// (hi, lo) = k (h + l) for a double-float k = kh + kl: Dekker's product with
// FMA, renormalised (~2^-47 relative).
__device__ __forceinline__ void df_scale(float kh, float kl, float h, float l, float &oh, float &ol)
{
    const float p = __fmul_rn(kh, h);   // never fused: pe is its error
    const float pe = fmaf(kh, l, fmaf(kl, h, fmaf(kh, h, -p)));
    two_sum_f(p, pe, oh, ol);
}

// One 64 x 64 tile of C_ij for one problem, unscaled, as (hi, lo): squared
// Euclidean sum_k (x_k - y_k)^2 and cosine 1 - <x, y> accumulated exactly
// (TwoSum on each exact product or square) and rounded once; dense costs are
// copied. Per-problem min / max / max|C| and non-finite entries are folded
// in with atomics. Problems without scaling get k C directly. The
// per-entry arithmetic is FP32 double-float (GB300's FP64 pipe is narrow);
// K is written with 16-byte stores and K^T through a shared-memory
// transpose, both coalesced.
__global__ void __launch_bounds__(256) k_batch_form(BatchProb *Pall, const BatchTile *tiles)
{
    constexpr int T = kBatchFormTile, KC = 32;
    __shared__ float Xs[T][KC + 1], Ys[T][KC + 1];
    __shared__ float Th[T][T + 1], Tl[T][T + 1];
    const BatchTile tl = tiles[blockIdx.x];
    BatchProb *P = Pall + tl.prob;
    const int n = P->n, m = P->m, d = P->d, kind = P->kind;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const int rb = tl.row0 + 4 * ty, cb = tl.col0 + 4 * tx;
    float vh[4][4], vl[4][4];
    if (kind == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int r = rb + a, c = cb + b;
                vh[a][b] = (r < n && c < m) ? P->C[(int64_t)r * P->ldc + c] : 0.0f;
                vl[a][b] = 0.0f;
            }
    } else {
        // Cosine: every partial sum of <x, y> lies within +-|x||y|, so a
        // running sum started at off = 2 |x||y| (rounded up) never drops
        // below |x||y| >= |x_k y_k|: each step can use Fast2Sum (3 ops, exact)
        // instead of TwoSum (6), and the offset comes off exactly at the end
        // (Sterbenz). The tile's row norms come from a first sweep over d.
        __shared__ float sN[2 * T];
        float off[4][4];
        if (kind == 2) {
            if (threadIdx.x < 2 * T) {
                const int rr = threadIdx.x % T;
                const bool isx = threadIdx.x < T;
                const int g = (isx ? tl.row0 : tl.col0) + rr;
                const float *row = isx ? P->X + (int64_t)g * d : P->Y + (int64_t)g * d;
                float nn = 0.0f;
                if (g < (isx ? n : m))
                    for (int k = 0; k < d; ++k) nn = fmaf(row[k], row[k], nn);
                sN[threadIdx.x] = sqrtf(nn) * (1.0f + 0x1p-10f) + 0x1p-100f;
            }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    off[a][b] = 2.0f * sN[4 * ty + a] * sN[T + 4 * tx + b] * (1.0f + 0x1p-10f);
        }
        float sacc[4][4], e[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) { sacc[a][b] = (kind == 2) ? off[a][b] : 0.0f; e[a][b] = 0.0f; }
        for (int k0 = 0; k0 < d; k0 += KC) {
            for (int t = threadIdx.x; t < T * KC; t += 256) {
                const int rr = t / KC, kk = t % KC;
                const int gx = tl.row0 + rr, gy = tl.col0 + rr, k = k0 + kk;
                Xs[rr][kk] = (gx < n && k < d) ? P->X[(int64_t)gx * d + k] : 0.0f;
                Ys[rr][kk] = (gy < m && k < d) ? P->Y[(int64_t)gy * d + k] : 0.0f;
            }
            __syncthreads();
            const int kn = min(KC, d - k0);
            for (int kk = 0; kk < kn; ++kk) {
                float xa[4], yb[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) xa[a] = Xs[4 * ty + a][kk];
#pragma unroll
                for (int b = 0; b < 4; ++b) yb[b] = Ys[4 * tx + b][kk];
                if (kind == 1) {
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            float dh, de;
                            two_sum_f(xa[a], -yb[b], dh, de);       // exact difference
                            const float p = __fmul_rn(dh, dh);
                            const float pe = fmaf(dh, dh, -p) + 2.0f * dh * de;  // + de^2 (negligible)
                            float t, te;
                            two_sum_f(sacc[a][b], p, t, te);
                            sacc[a][b] = t;
                            e[a][b] += te + pe;
                        }
                } else {
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const float p = __fmul_rn(xa[a], yb[b]);
                            const float pe = fmaf(xa[a], yb[b], -p);  // exact product error
                            const float t = sacc[a][b] + p;           // Fast2Sum: |s| >= |p|
                            const float z = t - sacc[a][b];
                            e[a][b] += (p - z) + pe;
                            sacc[a][b] = t;
                        }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (kind == 1) {
                    two_sum_f(sacc[a][b], e[a][b], vh[a][b], vl[a][b]);
                } else {
                    const float dot_hi = sacc[a][b] - off[a][b];     // exact (Sterbenz)
                    float ch, t;
                    two_sum_f(1.0f, -dot_hi, ch, t);
                    two_sum_f(ch, t - e[a][b], vh[a][b], vl[a][b]);
                }
            }
    }
    // statistics (double-float, FP64 once per thread), then k C
    const bool direct = !P->scale;
    const double kd = direct ? kLog2e / P->eps : 1.0;
    const float kh = (float)kd, kl = (float)(kd - (double)kh);
    float mxh = -INFINITY, mxl = 0.0f, mnh = INFINITY, mnl = 0.0f;
    int bad = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const bool valid = rb + a < n && cb + b < m;
            if (valid) {
                if (!isfinite(vh[a][b])) bad = 1;
                df_max(mxh, mxl, vh[a][b], vl[a][b]);
                df_min(mnh, mnl, vh[a][b], vl[a][b]);
            }
            float oh, ol;
            df_scale(kh, kl, vh[a][b], vl[a][b], oh, ol);
            vh[a][b] = valid ? oh : 0.0f;
            vl[a][b] = valid ? ol : 0.0f;
        }
    }
    // K: one 16-byte store per row and thread (columns [m, ldm) get zeros)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = rb + a;
        if (r < n && cb < P->ldm) {
            const int64_t i = (int64_t)r * P->ldm + cb;
            *reinterpret_cast<float4 *>(P->Kh + i) = make_float4(vh[a][0], vh[a][1], vh[a][2], vh[a][3]);
            *reinterpret_cast<float4 *>(P->Kl + i) = make_float4(vl[a][0], vl[a][1], vl[a][2], vl[a][3]);
        }
    }
    if (P->KTh) {
        // K^T through shared memory: row c of K^T, columns r (rows [n, ldn) get zeros)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                Th[4 * tx + b][4 * ty + a] = vh[a][b];
                Tl[4 * tx + b][4 * ty + a] = vl[a][b];
            }
        __syncthreads();
        for (int t = threadIdx.x; t < T * (T / 4); t += 256) {
            const int cc = t / (T / 4), r4 = 4 * (t % (T / 4));
            const int c = tl.col0 + cc, r = tl.row0 + r4;
            if (c < m && r < P->ldn) {
                const int64_t i = (int64_t)c * P->ldn + r;
                *reinterpret_cast<float4 *>(P->KTh + i) =
                    make_float4(Th[cc][r4], Th[cc][r4 + 1], Th[cc][r4 + 2], Th[cc][r4 + 3]);
                *reinterpret_cast<float4 *>(P->KTl + i) =
                    make_float4(Tl[cc][r4], Tl[cc][r4 + 1], Tl[cc][r4 + 2], Tl[cc][r4 + 3]);
            }
        }
    }
    double mx = mxh == -INFINITY ? -DBL_MAX : (double)mxh + (double)mxl;
    double mn = mnh == INFINITY ? DBL_MAX : (double)mnh + (double)mnl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx != -DBL_MAX) {
            atomicMax(&P->cmax_enc, enc_d(mx));
            atomicMin(&P->cmin_enc, enc_d(mn));
            atomicMax(&P->cabs_enc, enc_d(fmax(fabs(mx), fabs(mn))));
        }
        if (bad) atomicOr(&P->nonfinite, 1u);
    }
}

// k C in place for problems scaled by their maximum (k needs max C): a
// double-float product per entry, K and K^T each swept with coalesced
// 16-byte accesses (padding entries hold zeros and stay zero).
__global__ void __launch_bounds__(256) k_batch_scale(BatchProb *Pall, const BatchTile *tiles)
{
    const BatchTile tl = tiles[blockIdx.x];
    BatchProb *P = Pall + tl.prob;
    if (!P->scale) return;
    const double k = batch_k(P);
    const float kh = (float)k, kl = (float)(k - (double)kh);
    constexpr int T = kBatchFormTile, V = kBatchFormTile / 4;
    auto scale4 = [&](float *H, float *L, int64_t i) {
        float4 h = *reinterpret_cast<float4 *>(H + i), l = *reinterpret_cast<float4 *>(L + i);
        float4 oh, ol;
        df_scale(kh, kl, h.x, l.x, oh.x, ol.x);
        df_scale(kh, kl, h.y, l.y, oh.y, ol.y);
        df_scale(kh, kl, h.z, l.z, oh.z, ol.z);
        df_scale(kh, kl, h.w, l.w, oh.w, ol.w);
        *reinterpret_cast<float4 *>(H + i) = oh;
        *reinterpret_cast<float4 *>(L + i) = ol;
    };
    for (int t = threadIdx.x; t < T * V; t += 256) {
        const int r = tl.row0 + t / V, c4 = tl.col0 + 4 * (t % V);
        if (r < P->n && c4 < P->m) scale4(P->Kh, P->Kl, (int64_t)r * P->ldm + c4);
    }
    if (P->KTh) {
        for (int t = threadIdx.x; t < T * V; t += 256) {
            const int c = tl.col0 + t / V, r4 = tl.row0 + 4 * (t % V);
            if (c < P->m && r4 < P->n) scale4(P->KTh, P->KTl, (int64_t)c * P->ldn + r4);
        }
    }
}

// ---------------------------------------------------------- the solver --

// What follows a large problem's step: the next row phase (through the update
// items when the step was split), the final evaluation pass, or the result.
__device__ void step_continue(BatchQueue *q, BatchProb *P, BatchResult *R, int p, bool stop,
                              bool split)
{
    if (!stop) {
        if (split) q_push(q, P->step_items, [&](int t) { return batch_item(BI_UPD, p, t); });
        else q_push(q, P->row_tiles, [&](int t) { return batch_item(BI_ROW, p, t); });
    } else if (P->evaluate) {
        q_push(q, P->row_tiles, [&](int t) { return batch_item(BI_FINAL, p, t); });
    } else {
        cta_finish<false>(P, R, true);
        publish_early(q, p, R);
        problem_done(q);
    }
}

__global__ void __launch_bounds__(kBatchThreads, 4) k_batch_solve(BatchProb *Pall, BatchQueue *q,
                                                               BatchResult *res)
{
    __shared__ unsigned long long item_s;
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned long long it;
            item_s = q_pop(q, it) ? it : ~0ull;
        }
        __syncthreads();
        const unsigned long long item = item_s;
        __syncthreads();
        if (item == ~0ull) break;
        const int p = (int)(item >> 32);
        const int kind = (int)((item >> 28) & 0xf);
        const int tile = (int)(item & 0x0fffffffu);
        BatchProb *P = Pall + p;
        BatchResult *R = res + p;
        if (kind == BI_SMALL) {
            // the whole solve in this CTA (every read of the problem's data
            // is of this CTA's own writes: L1 loads, CTA barriers)
            bool ok = cta_init(P);
            if (ok) {
                const bool is_acc = P->method == 1;
                for (;;) {
                    __syncthreads();
                    double part[2];
                    cta_rows<false, true>(P, 0, P->n, part);
                    if (threadIdx.x == 0) { P->rowpart[0] = part[0]; P->rowpart[1] = part[1]; }
                    __syncthreads();
                    const StageK K = cta_stage_constants(is_acc, P->mu);
                    const bool check = is_acc && !P->first && P->stability != 0;
                    double ws[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                    double lo3[3] = {DBL_MAX, DBL_MAX, DBL_MAX};
                    double hi3[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
                    for (int t = 0; t < P->col_tiles; ++t) cta_cols<true>(P, t, K, check, ws, lo3, hi3);
                    cta_colrec(P, 0, ws, lo3, hi3);
                    if (cta_step<true>(P, 1)) break;
                }
                __syncthreads();
                if (P->evaluate) {
                    double part[2];
                    cta_rows<true, true>(P, 0, P->n, part);
                    if (threadIdx.x == 0) { P->rowpart[0] = part[0]; P->rowpart[1] = part[1]; }
                    __syncthreads();
                }
            }
            cta_finish<true>(P, R, ok);
            publish_early(q, p, R);
            problem_done(q);
        } else if (kind == BI_INIT) {
            const bool ok = cta_init(P);
            if (ok) {
                q_push(q, P->row_tiles, [&](int t) { return batch_item(BI_ROW, p, t); });
            } else {
                cta_finish<false>(P, R, false);
                publish_early(q, p, R);
                problem_done(q);
            }
        } else if (kind == BI_ROW || kind == BI_FINAL) {
            const int r0 = tile * P->rows_per_tile;
            const int r1 = min(P->n, r0 + P->rows_per_tile);
            double part[2];
            if (kind == BI_ROW) cta_rows<false, false>(P, r0, r1, part);
            else cta_rows<true, false>(P, r0, r1, part);
            if (threadIdx.x == 0) {
                P->rowpart[2 * tile] = part[0];
                P->rowpart[2 * tile + 1] = part[1];
            }
            if (arrive_last(P, P->row_tiles)) {
                if (kind == BI_ROW) {
                    q_push(q, P->col_items, [&](int t) { return batch_item(BI_COL, p, t); });
                } else {
                    cta_finish<false>(P, R, true);
                    publish_early(q, p, R);
                    problem_done(q);
                }
            }
        } else if (kind == BI_COL) {
            const bool is_acc = P->method == 1;
            const StageK K = cta_stage_constants(is_acc, __ldcg(&P->mu));
            const bool check = is_acc && !__ldcg(&P->first) && P->stability != 0;
            if (P->KTh) {
                const int j0 = tile * P->cols_per_item;
                cta_colsT(P, j0, min(P->m, j0 + P->cols_per_item), K, check);
            } else {
                double ws[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                double lo3[3] = {DBL_MAX, DBL_MAX, DBL_MAX};
                double hi3[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
                cta_cols<false>(P, tile, K, check, ws, lo3, hi3);
                cta_colrec(P, tile, ws, lo3, hi3);
            }
            if (arrive_last(P, P->col_items)) {
                if (P->step_items > 0) {
                    // large problem: P1 totals here, P2 and the update as items
                    if (split_step_begin(P)) {
                        q_push(q, P->step_items, [&](int t) { return batch_item(BI_P2, p, t); });
                    } else {
                        const bool stop = split_step_decide(P, false);
                        step_continue(q, P, R, p, stop, true);
                    }
                } else {
                    const bool stop = cta_step<false>(P, P->col_tiles);
                    step_continue(q, P, R, p, stop, false);
                }
            }
        } else if (kind == BI_P2) {
            split_step_p2(P, tile);
            if (arrive_last(P, P->step_items)) {
                const bool stop = split_step_decide(P, true);
                step_continue(q, P, R, p, stop, true);
            }
        } else if (kind == BI_UPD) {
            split_step_update(P, tile);
            if (arrive_last(P, P->step_items))
                q_push(q, P->row_tiles, [&](int t) { return batch_item(BI_ROW, p, t); });
        }
        __syncthreads();
    }
}

cudaError_t launch_batch_form(const BatchProb *P, const BatchTile *tiles, int ntiles, int dmax,
                              cudaStream_t s)
{
    (void)dmax;
    if (ntiles <= 0) return cudaSuccess;
    k_batch_form<<<ntiles, 256, 0, s>>>(const_cast<BatchProb *>(P), tiles);
    return cudaGetLastError();
}

cudaError_t launch_batch_scale(BatchProb *P, const BatchTile *tiles, int ntiles, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    k_batch_scale<<<ntiles, 256, 0, s>>>(P, tiles);
    return cudaGetLastError();
}

cudaError_t launch_batch_solve(BatchProb *P, BatchQueue *q, BatchResult *res, int grid,
                               cudaStream_t s)
{
    k_batch_solve<<<grid, kBatchThreads, 0, s>>>(P, q, res);
    return cudaGetLastError();
}

int occupancy_batch_solve()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_solve, kBatchThreads, 0);
    return b > 0 ? b : 1;
}

}  // namespace accsink

namespace accsink {

// Sets every queue slot free for its first position, then publishes the
// initial items (one per problem) at positions 0 .. count - 1.
__global__ void k_queue_init(BatchQueue *q, const unsigned long long *items0, int count)
{
    const unsigned long long cap = q->cap;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        if (i < (unsigned long long)count) {
            q->items[i] = items0[i];
            q->seq[i] = i + 1;
        } else {
            q->seq[i] = i;
        }
    }
}

cudaError_t launch_queue_init(BatchQueue *q, const unsigned long long *items0, int count,
                              unsigned long long cap, cudaStream_t s)
{
    const int grid = (int)std::min<unsigned long long>(1024, (cap + 255) / 256);
    k_queue_init<<<grid, 256, 0, s>>>(q, items0, count);
    return cudaGetLastError();
}

}  // namespace accsink

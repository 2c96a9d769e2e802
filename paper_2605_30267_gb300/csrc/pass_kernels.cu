// Streaming O(nm) kernels: the row log-sum-exp pass, the column log-sum-exp
// pass (Sec. 2, u- and v-updates in the log domain of Sec. 5), and a one-off
// pass that gathers the cost statistics (max C for MAX_TO_ONE scaling,
// Sec. 5; max|C| for the operand shifts; a NaN/Inf scan).
//
// All three are bound by HBM bandwidth: the cost is read exactly once per
// launch with 128-bit non-allocating loads, and every other operand (the
// potentials as double-float pairs) is a few KB to a few hundred KB that
// stays in L1/L2. See accsink_internal.cuh for the precision argument.
#include <float.h>
#include <cstdlib>

#include "accsink_internal.cuh"

namespace accsink {

// ------------------------------------------------------------------------
// Cost statistics: per-CTA partial (max C, min C, max |C|, #non-finite).
// ------------------------------------------------------------------------
template <bool VEC>
__global__ void __launch_bounds__(256) k_cost_stats(CostView cv, Work w)
{
    float mx = -FLT_MAX, mn = FLT_MAX, ab = 0.0f;
    int bad = 0;
    const int64_t total_rows = cv.n;
    const int m = cv.m;
    auto visit = [&](float c) {
        if (!isfinite(c)) { ++bad; return; }
        mx = fmaxf(mx, c);
        mn = fminf(mn, c);
        ab = fmaxf(ab, fabsf(c));
    };
    for (int64_t i = blockIdx.x; i < total_rows; i += gridDim.x) {
        const float *row = cv.C + i * cv.ldc;
        if (VEC) {
            const int m4 = m >> 2;
            for (int v = threadIdx.x; v < m4; v += blockDim.x) {
                float4 c = ld_stream4(row + 4 * v);
                visit(c.x); visit(c.y); visit(c.z); visit(c.w);
            }
            for (int j = 4 * m4 + threadIdx.x; j < m; j += blockDim.x) visit(ld_stream1(row + j));
        } else {
            for (int j = threadIdx.x; j < m; j += blockDim.x) visit(ld_stream1(row + j));
        }
    }
    __shared__ float s_mx[8], s_mn[8], s_ab[8];
    __shared__ int s_bad[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        ab = fmaxf(ab, __shfl_xor_sync(0xffffffffu, ab, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { s_mx[wid] = mx; s_mn[wid] = mn; s_ab[wid] = ab; s_bad[wid] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            mx = fmaxf(mx, s_mx[q]); mn = fminf(mn, s_mn[q]);
            ab = fmaxf(ab, s_ab[q]); bad += s_bad[q];
        }
        w.statpart[4 * blockIdx.x + 0] = mx;
        w.statpart[4 * blockIdx.x + 1] = mn;
        w.statpart[4 * blockIdx.x + 2] = ab;
        w.statpart[4 * blockIdx.x + 3] = bad;
    }
}

cudaError_t launch_cost_stats(const CostView &cv, const Work &w, int grid, cudaStream_t s)
{
    if (cv.vec) k_cost_stats<true><<<grid, 256, 0, s>>>(cv, w);
    else k_cost_stats<false><<<grid, 256, 0, s>>>(cv, w);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Online log-sum-exp accumulator for one output (row or column) held by one
// thread: reference R (a running max of s = G - C, FP32 exact), FP32 Kahan
// pair (S, K) of sum 2^((s - R) k), and optionally the same for C * 2^(...).
// ------------------------------------------------------------------------
struct Acc {
    float R, S, K;
};

__device__ __forceinline__ void acc_rescale(Acc &a, float newR, float kh, float kl)
{
    const float f = exp2_scaled(a.R - newR, kh, kl);
    a.S = __fmul_rn(a.S, f);
    a.K = __fmul_rn(a.K, f);
    a.R = newR;
}

__device__ __forceinline__ void kahan_add(Acc &a, float x)
{
    const float y = x - a.K;
    const float t = a.S + y;
    a.K = (t - a.S) - y;
    a.S = t;
}

// One element: exact split G - c = s + e (Fast2Sum, |G| >= |c|), returns
// 2^((s - R + e + gamma) k) with the gamma*k part pre-scaled in gk.
__device__ __forceinline__ float lse_term(float G, float gk, float c, float R, float kh, float kl)
{
    const float s = G - c;
    const float z = s - G;
    const float e = -c - z;
    const float q = fmaf(e, kh, gk);
    const float t = s - R;
    return ex2_approx(fmaf(t, kh, fmaf(t, kl, q)));
}

// Same with s = fl(G - c) already formed.
__device__ __forceinline__ float lse_term_s(float s, float G, float gk, float c, float R,
                                            float kh, float kl)
{
    const float z = s - G;
    const float e = -c - z;
    const float q = fmaf(e, kh, gk);
    const float t = s - R;
    return ex2_approx(fmaf(t, kh, fmaf(t, kl, q)));
}

// ------------------------------------------------------------------------
// Row pass: one CTA owns a contiguous block of rows; all its threads sweep
// each group of RG rows together (so every G/Gk load from L1 is reused RG
// times) and the row totals are merged across the CTA in FP64.
//   u_i = log a_i - LSE_j(x_j - C_ij / eps_c)
// is written together with the column-pass operand F_i = eps_c u_i + shift_f
// as an FP32 pair, and per-CTA partials of sum a_i u_i (dual objective) and,
// with WITH_COST, of sum_ij C_ij P_ij.
// ------------------------------------------------------------------------
constexpr int kRowNT = 256;

template <int RG, int U, bool VEC, bool WITH_COST>
__global__ void __launch_bounds__(kRowNT) k_row_pass(CostView cv, Work w)
{
    DevState *st = w.st;
    if (!w.ignore_done && *(volatile int32_t *)&st->done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->barrier = 0u;   // for the step kernel

    constexpr int NW = kRowNT / 32;
    const float kh = st->k_hi, kl = st->k_lo;
    const int n = cv.n, m = cv.m;
    const int64_t ldc = cv.ldc;
    const int r0 = (int)((int64_t)blockIdx.x * n / gridDim.x);
    const int r1 = (int)((int64_t)(blockIdx.x + 1) * n / gridDim.x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int m4 = m >> 2;
    const int tail0 = 4 * m4;

    __shared__ float sh_R[NW][RG];
    __shared__ double sh_S[NW][RG];
    __shared__ double sh_CS[NW][RG];
    __shared__ double sh_out[2][RG];

    double my_dual = 0.0, my_cost = 0.0;   // used by threads < RG

    const float4 *G4 = reinterpret_cast<const float4 *>(w.G);
    const float4 *Gk4 = reinterpret_cast<const float4 *>(w.Gk);

    for (int i0 = r0; i0 < r1; i0 += RG) {
        const float *crow[RG];
        Acc acc[RG];
        Acc cacc[RG];
#pragma unroll
        for (int r = 0; r < RG; ++r) {
            const int i = (i0 + r < r1) ? (i0 + r) : i0;
            crow[r] = cv.C + (int64_t)i * ldc;
            acc[r] = {0.0f, 0.0f, 0.0f};
            cacc[r] = {0.0f, 0.0f, 0.0f};
        }
        for (int vb = threadIdx.x; vb < m4; vb += kRowNT * U) {
            float4 g[U], gk[U];
            float4 c[RG][U];
            bool val[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int v = vb + u * kRowNT;
                val[u] = v < m4;
                if (val[u]) {
                    g[u] = __ldg(G4 + v);
                    gk[u] = __ldg(Gk4 + v);
#pragma unroll
                    for (int r = 0; r < RG; ++r) {
                        if (VEC) {
                            c[r][u] = ld_stream4(crow[r] + 4 * v);
                        } else {
                            c[r][u].x = ld_stream1(crow[r] + 4 * v + 0);
                            c[r][u].y = ld_stream1(crow[r] + 4 * v + 1);
                            c[r][u].z = ld_stream1(crow[r] + 4 * v + 2);
                            c[r][u].w = ld_stream1(crow[r] + 4 * v + 3);
                        }
                    }
                } else {
                    g[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    gk[u] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
#pragma unroll
                    for (int r = 0; r < RG; ++r) c[r][u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                // chunk max of s = G - C (invalid slots give 0 <= R)
                float cm = acc[r].R;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    cm = fmaxf(cm, fmaxf(fmaxf(g[u].x - c[r][u].x, g[u].y - c[r][u].y),
                                         fmaxf(g[u].z - c[r][u].z, g[u].w - c[r][u].w)));
                }
                if (cm > acc[r].R) {
                    if (WITH_COST) {
                        const float f = exp2_scaled(acc[r].R - cm, kh, kl);
                        cacc[r].S = __fmul_rn(cacc[r].S, f);
                        cacc[r].K = __fmul_rn(cacc[r].K, f);
                    }
                    acc_rescale(acc[r], cm, kh, kl);
                }
                float cs = 0.0f, ccs = 0.0f;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float R = acc[r].R;
                    float p;
                    p = lse_term(g[u].x, gk[u].x, c[r][u].x, R, kh, kl); cs += p;
                    if (WITH_COST) ccs = fmaf(c[r][u].x, p, ccs);
                    p = lse_term(g[u].y, gk[u].y, c[r][u].y, R, kh, kl); cs += p;
                    if (WITH_COST) ccs = fmaf(c[r][u].y, p, ccs);
                    p = lse_term(g[u].z, gk[u].z, c[r][u].z, R, kh, kl); cs += p;
                    if (WITH_COST) ccs = fmaf(c[r][u].z, p, ccs);
                    p = lse_term(g[u].w, gk[u].w, c[r][u].w, R, kh, kl); cs += p;
                    if (WITH_COST) ccs = fmaf(c[r][u].w, p, ccs);
                }
                kahan_add(acc[r], cs);
                if (WITH_COST) kahan_add(cacc[r], ccs);
            }
        }
        // ragged tail (m % 4 columns), one column per thread
        if (tail0 + (int)threadIdx.x < m) {
            const int j = tail0 + threadIdx.x;
            const float Gj = w.G[j], Gkj = w.Gk[j];
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const float c = ld_stream1(crow[r] + j);
                const float s = Gj - c;
                if (s > acc[r].R) {
                    if (WITH_COST) {
                        const float f = exp2_scaled(acc[r].R - s, kh, kl);
                        cacc[r].S = __fmul_rn(cacc[r].S, f);
                        cacc[r].K = __fmul_rn(cacc[r].K, f);
                    }
                    acc_rescale(acc[r], s, kh, kl);
                }
                const float p = lse_term(Gj, Gkj, c, acc[r].R, kh, kl);
                kahan_add(acc[r], p);
                if (WITH_COST) kahan_add(cacc[r], c * p);
            }
        }
        // CTA merge: reference = CTA max of R, then FP64 sums of rescaled partials
#pragma unroll
        for (int r = 0; r < RG; ++r) {
            const float rm = warp_max(acc[r].R);
            if (lane == 0) sh_R[wid][r] = rm;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RG; ++r) {
            float Rrow = sh_R[0][r];
#pragma unroll
            for (int q = 1; q < NW; ++q) Rrow = fmaxf(Rrow, sh_R[q][r]);
            const double sc = (double)exp2_scaled(acc[r].R - Rrow, kh, kl);
            double v = ((double)acc[r].S - (double)acc[r].K) * sc;
            v = warp_sum(v);
            if (lane == 0) sh_S[wid][r] = v;
            if (WITH_COST) {
                double cv2 = ((double)cacc[r].S - (double)cacc[r].K) * sc;
                cv2 = warp_sum(cv2);
                if (lane == 0) sh_CS[wid][r] = cv2;
            }
        }
        __syncthreads();
        if (threadIdx.x < RG) {
            const int r = threadIdx.x;
            const int i = i0 + r;
            if (i < r1) {
                float Rrow = sh_R[0][r];
                double S = 0.0, CS = 0.0;
                for (int q = 0; q < NW; ++q) {
                    Rrow = fmaxf(Rrow, sh_R[q][r]);
                    S += sh_S[q][r];
                    if (WITH_COST) CS += sh_CS[q][r];
                }
                const double lse = ((double)Rrow - st->shift_g) * st->inv_eps_c + log(S);
                const double ui = w.loga[i] - lse;
                w.u[i] = ui;
                const double F = st->eps_c * ui + st->shift_f;
                const float Fh = (float)F;
                const float Fl = (float)(F - (double)Fh);
                w.FF[i] = make_float2(Fh, Fl * kh);
                w.Fh[i] = Fh;
                w.Fk[i] = Fl * kh;
                my_dual += w.a[i] * ui;
                // P_ij = a_i 2^{(s_ij - R) k} / S after the row pass, so
                // sum_j C_ij P_ij = a_i CS / S; for given potentials f the
                // row weight is exp(f_i / eps + LSE_i) instead of a_i.
                if (WITH_COST) {
                    const double wi = w.f_given ? exp(w.f_given[i] / st->eps_user + lse) : w.a[i];
                    my_cost += wi * (CS / S);
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < RG) {
        sh_out[0][threadIdx.x] = my_dual;
        sh_out[1][threadIdx.x] = my_cost;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d = 0.0, c = 0.0;
        for (int r = 0; r < RG; ++r) { d += sh_out[0][r]; c += sh_out[1][r]; }
        w.rowpart[2 * blockIdx.x + 0] = d;
        w.rowpart[2 * blockIdx.x + 1] = c;
    }
}

constexpr int kRowRG = 2;
constexpr int kRowU = 4;

cudaError_t launch_row_pass(const CostView &cv, const Work &w, int grid, const RowSplit &sp,
                            bool with_cost, cudaStream_t s)
{
    // 128-bit-aligned costs stream through the TMA pipeline (row_tma.cu);
    // the plain kernel below serves the unaligned layouts.
    if (cv.vec) {
        if (row_kernel_choice() == 1) return launch_row_pass_tma(cv, w, grid, with_cost, s);
        return launch_row_pass_warp(cv, w, grid, sp, with_cost, s);
    }
    if (cv.vec) {
        if (with_cost) k_row_pass<kRowRG, kRowU, true, true><<<grid, kRowNT, 0, s>>>(cv, w);
        else k_row_pass<kRowRG, kRowU, true, false><<<grid, kRowNT, 0, s>>>(cv, w);
    } else {
        if (with_cost) k_row_pass<kRowRG, kRowU, false, true><<<grid, kRowNT, 0, s>>>(cv, w);
        else k_row_pass<kRowRG, kRowU, false, false><<<grid, kRowNT, 0, s>>>(cv, w);
    }
    return cudaGetLastError();
}

int occupancy_row_pass(int vec)
{
    int b = 0;
    if (vec)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_row_pass<kRowRG, kRowU, true, false>,
                                                      kRowNT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_row_pass<kRowRG, kRowU, false, false>,
                                                      kRowNT, 0);
    return b > 0 ? b : 1;
}

// ------------------------------------------------------------------------
// Column pass: CTA (strip, split) covers 128 columns (4 per lane) and the
// rows of one split; its 8 warps take interleaved rows, so each row segment
// of 512 B is one fully coalesced warp load. Per column it produces a
// partial (R, S) with sum_i over the split of 2^((F_i - C_ij - R) k) = S,
// which the step kernel merges across splits.
// ------------------------------------------------------------------------
constexpr int kColNT = 256;
constexpr int kColU = 8;

template <int U, bool VEC>
__global__ void __launch_bounds__(kColNT) k_col_pass(CostView cv, Work w)
{
    DevState *st = w.st;
    if (*(volatile int32_t *)&st->done) return;
    constexpr int NW = kColNT / 32;
    const float kh = st->k_hi, kl = st->k_lo;
    const int n = cv.n, m = cv.m;
    const int64_t ldc = cv.ldc;
    const int split = blockIdx.y, splits = gridDim.y;
    const int r0 = (int)((int64_t)split * n / splits);
    const int r1 = (int)((int64_t)(split + 1) * n / splits);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col0 = blockIdx.x * kColStrip + 4 * lane;
    // columns of this lane: col0 .. col0+3 (some may be >= m)
    const bool full4 = VEC && (col0 + 3 < m);

    Acc acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = {0.0f, 0.0f, 0.0f};

    for (int ib = r0 + wid; ib < r1; ib += NW * U) {
        float4 c[U];
        float2 ff[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = ib + u * NW;
            if (i < r1) {
                ff[u] = __ldg(w.FF + i);
                const float *p = cv.C + (int64_t)i * ldc + col0;
                if (full4) {
                    c[u] = ld_stream4(p);
                } else {
                    c[u].x = (col0 + 0 < m) ? ld_stream1(p + 0) : 0.0f;
                    c[u].y = (col0 + 1 < m) ? ld_stream1(p + 1) : 0.0f;
                    c[u].z = (col0 + 2 < m) ? ld_stream1(p + 2) : 0.0f;
                    c[u].w = (col0 + 3 < m) ? ld_stream1(p + 3) : 0.0f;
                }
            } else {
                ff[u] = make_float2(0.0f, -INFINITY);
                c[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float cm0 = acc[0].R, cm1 = acc[1].R, cm2 = acc[2].R, cm3 = acc[3].R;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cm0 = fmaxf(cm0, ff[u].x - c[u].x);
            cm1 = fmaxf(cm1, ff[u].x - c[u].y);
            cm2 = fmaxf(cm2, ff[u].x - c[u].z);
            cm3 = fmaxf(cm3, ff[u].x - c[u].w);
        }
        if (cm0 > acc[0].R) acc_rescale(acc[0], cm0, kh, kl);
        if (cm1 > acc[1].R) acc_rescale(acc[1], cm1, kh, kl);
        if (cm2 > acc[2].R) acc_rescale(acc[2], cm2, kh, kl);
        if (cm3 > acc[3].R) acc_rescale(acc[3], cm3, kh, kl);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            s0 += lse_term(ff[u].x, ff[u].y, c[u].x, acc[0].R, kh, kl);
            s1 += lse_term(ff[u].x, ff[u].y, c[u].y, acc[1].R, kh, kl);
            s2 += lse_term(ff[u].x, ff[u].y, c[u].z, acc[2].R, kh, kl);
            s3 += lse_term(ff[u].x, ff[u].y, c[u].w, acc[3].R, kh, kl);
        }
        kahan_add(acc[0], s0);
        kahan_add(acc[1], s1);
        kahan_add(acc[2], s2);
        kahan_add(acc[3], s3);
    }
    // merge the NW warps' partials of each column
    __shared__ float sh_R[NW][kColStrip];
    __shared__ float sh_S[NW][kColStrip];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        sh_R[wid][4 * lane + q] = acc[q].R;
        sh_S[wid][4 * lane + q] = acc[q].S - acc[q].K;
    }
    __syncthreads();
    if (threadIdx.x < kColStrip) {
        const int t = threadIdx.x;
        const int j = blockIdx.x * kColStrip + t;
        if (j < m) {
            float R = sh_R[0][t];
#pragma unroll
            for (int q = 1; q < NW; ++q) R = fmaxf(R, sh_R[q][t]);
            double S = 0.0;
#pragma unroll
            for (int q = 0; q < NW; ++q)
                S += (double)sh_S[q][t] * (double)exp2_scaled(sh_R[q][t] - R, kh, kl);
            w.colpart[(int64_t)split * m + j] = make_float2(R, (float)S);
        }
    }
}

cudaError_t launch_col_pass(const CostView &cv, const Work &w, int splits, cudaStream_t s)
{
    dim3 grid((cv.m + kColStrip - 1) / kColStrip, splits);
    if (cv.vec) k_col_pass<kColU, true><<<grid, kColNT, 0, s>>>(cv, w);
    else k_col_pass<kColU, false><<<grid, kColNT, 0, s>>>(cv, w);
    return cudaGetLastError();
}

int occupancy_col_pass(int vec)
{
    int b = 0;
    if (vec)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_col_pass<kColU, true>, kColNT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_col_pass<kColU, false>, kColNT, 0);
    return b > 0 ? b : 1;
}

void setup_col_pass() {}

}  // namespace accsink

// Log-sum-exp over the rows of a row-major FP32 matrix X, one warp per row
// (the 128-bit-aligned path). It serves both passes of an S evaluation:
//   MODE_ROW: X = C, operand G (columns): u_i and the column-pass operand;
//   MODE_COL: X = C^T (a transposed copy kept by the solver), operand F
//             (rows of C): ell_j = LSE_i((f_i - C_ij) / eps).
//
// Every warp streams whole rows on its own: no shared memory, no CTA
// barriers, so no warp ever waits for another. Lanes read 128-bit slots of
// the row (a warp covers 512 contiguous bytes per slot); the column operand
// (G, gamma k) is read through L1, where it stays resident because the cost
// is read with non-allocating loads. The next chunk of the row is loaded
// while the current one is reduced (register double buffering), so each warp
// keeps 2 x U x 512 bytes of the cost in flight.
//
// Per element the arithmetic is the exact-split scheme of the plain row
// pass. The per-row merge across lanes is done in FP32 double-float (no FP64
// pipe in the hot loop), and lane 0 finishes the row in FP64.
#include "accsink_internal.cuh"

namespace accsink {

namespace {

constexpr int kWarpNT = 256;
constexpr int kU = 4;   // float4 slots per lane per chunk

struct Acc {
    float R, S, K;
};

__device__ __forceinline__ void kahan(Acc &a, float x)
{
    const float y = x - a.K;
    const float t = a.S + y;
    a.K = (t - a.S) - y;
    a.S = t;
}

__device__ __forceinline__ float term_s(float s, float G, float gk, float c, float R, float kh,
                                        float kl)
{
    const float z = s - G;
    const float e = -c - z;
    const float q = fmaf(e, kh, gk);
    const float t = s - R;
    return ex2_approx(fmaf(t, kh, fmaf(t, kl, q)));
}

// Error-free sum of two floats (Knuth 2Sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

}  // namespace

enum { MODE_ROW = 0, MODE_COL = 1 };

template <int MODE, bool WITH_COST>
__global__ void __launch_bounds__(kWarpNT) k_lse_rows(CostView cv, const float *Oh,
                                                      const float *Ok, Work w)
{
    DevState *st = w.st;
    if (!w.ignore_done && *(volatile int32_t *)&st->done) return;
    if (MODE == MODE_ROW && blockIdx.x == 0 && threadIdx.x == 0)
        st->barrier = 0u;   // for the step kernel

    const float kh = st->k_hi, kl = st->k_lo;
    const int n = cv.n, m = cv.m;
    const int64_t ldc = cv.ldc;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * kWarpNT + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kWarpNT) >> 5;
    const int m4 = m >> 2;
    const int tail0 = 4 * m4;
    const float4 *G4 = reinterpret_cast<const float4 *>(Oh);
    const float4 *Gk4 = reinterpret_cast<const float4 *>(Ok);
    constexpr int kStep = 32 * kU;     // float4 slots per chunk per warp

    double my_dual = 0.0, my_cost = 0.0;   // lane 0
    for (int i = gwarp; i < n; i += nwarps) {
        const float4 *row = reinterpret_cast<const float4 *>(cv.C + (int64_t)i * ldc);
        Acc acc = {0.0f, 0.0f, 0.0f};
        Acc cacc = {0.0f, 0.0f, 0.0f};
        float4 cbuf[kU];
        // prefetch the first chunk
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int v = lane + 32 * u;
            cbuf[u] = (v < m4) ? ld_stream4(reinterpret_cast<const float *>(row + v))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int vb = 0; vb < m4; vb += kStep) {
            float4 c[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) c[u] = cbuf[u];
            // issue the next chunk's loads before reducing this one
            const int nb = vb + kStep;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = nb + lane + 32 * u;
                if (v < m4) cbuf[u] = ld_stream4(reinterpret_cast<const float *>(row + v));
            }
            float4 g[kU], gk[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = vb + lane + 32 * u;
                if (v < m4) {
                    g[u] = __ldg(G4 + v);
                    gk[u] = __ldg(Gk4 + v);
                } else {
                    g[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    gk[u] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
                    c[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            float4 sv[kU];
            float cm = acc.R;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                sv[u] = make_float4(g[u].x - c[u].x, g[u].y - c[u].y, g[u].z - c[u].z,
                                    g[u].w - c[u].w);
                cm = fmaxf(cm, fmaxf(fmaxf(sv[u].x, sv[u].y), fmaxf(sv[u].z, sv[u].w)));
            }
            if (cm > acc.R) {
                const float f = exp2_scaled(acc.R - cm, kh, kl);
                acc.S *= f;
                acc.K *= f;
                if (WITH_COST) { cacc.S *= f; cacc.K *= f; }
                acc.R = cm;
            }
            const float R = acc.R;
            float cs[kU], ccs[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const float p0 = term_s(sv[u].x, g[u].x, gk[u].x, c[u].x, R, kh, kl);
                const float p1 = term_s(sv[u].y, g[u].y, gk[u].y, c[u].y, R, kh, kl);
                const float p2 = term_s(sv[u].z, g[u].z, gk[u].z, c[u].z, R, kh, kl);
                const float p3 = term_s(sv[u].w, g[u].w, gk[u].w, c[u].w, R, kh, kl);
                cs[u] = (p0 + p1) + (p2 + p3);
                if (WITH_COST)
                    ccs[u] = fmaf(c[u].x, p0, fmaf(c[u].y, p1, fmaf(c[u].z, p2, c[u].w * p3)));
            }
            float csum = (cs[0] + cs[1]) + (cs[2] + cs[3]);
            kahan(acc, csum);
            if (WITH_COST) kahan(cacc, (ccs[0] + ccs[1]) + (ccs[2] + ccs[3]));
        }
        // ragged tail (m % 4 columns)
        if (tail0 + lane < m) {
            const int j = tail0 + lane;
            const float Gj = Oh[j], Gkj = Ok[j];
            const float c = ld_stream1(cv.C + (int64_t)i * ldc + j);
            const float s = Gj - c;
            if (s > acc.R) {
                const float f = exp2_scaled(acc.R - s, kh, kl);
                acc.S *= f;
                acc.K *= f;
                if (WITH_COST) { cacc.S *= f; cacc.K *= f; }
                acc.R = s;
            }
            const float p = term_s(s, Gj, Gkj, c, acc.R, kh, kl);
            kahan(acc, p);
            if (WITH_COST) kahan(cacc, c * p);
        }
        // merge the lanes: common reference, then a double-float tree sum
        const float Rrow = warp_max(acc.R);
        const float sc = exp2_scaled(acc.R - Rrow, kh, kl);
        float hi, lo;
        two_sum(acc.S * sc, -acc.K * sc, hi, lo);
        float chi = 0.f, clo = 0.f;
        if (WITH_COST) two_sum(cacc.S * sc, -cacc.K * sc, chi, clo);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
            const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
            float s, e;
            two_sum(hi, ohi, s, e);
            lo = lo + olo + e;
            two_sum(s, lo, hi, lo);
            if (WITH_COST) {
                const float ochi = __shfl_xor_sync(0xffffffffu, chi, o);
                const float oclo = __shfl_xor_sync(0xffffffffu, clo, o);
                two_sum(chi, ochi, s, e);
                clo = clo + oclo + e;
                two_sum(s, clo, chi, clo);
            }
        }
        if (MODE == MODE_COL && lane == 0) {
            const double S = (double)hi + (double)lo;
            w.ell[i] = ((double)Rrow - st->shift_f) * st->inv_eps_c + log(S);
        }
        if (MODE == MODE_ROW && lane == 0) {
            const double S = (double)hi + (double)lo;
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
            if (WITH_COST) {
                const double CS = (double)chi + (double)clo;
                const double wi = w.f_given ? exp(w.f_given[i] / st->eps_user + lse) : w.a[i];
                my_cost += wi * (CS / S);
            }
        }
    }
    if (MODE == MODE_COL) return;
    // per-CTA partials, fixed order over the CTA's warps
    __shared__ double sh[2][kWarpNT / 32];
    if (lane == 0) {
        sh[0][threadIdx.x >> 5] = my_dual;
        sh[1][threadIdx.x >> 5] = my_cost;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d = 0.0, c = 0.0;
        for (int q = 0; q < kWarpNT / 32; ++q) { d += sh[0][q]; c += sh[1][q]; }
        w.rowpart[2 * blockIdx.x + 0] = d;
        w.rowpart[2 * blockIdx.x + 1] = c;
    }
}

cudaError_t launch_row_pass_warp(const CostView &cv, const Work &w, int grid, bool with_cost,
                                 cudaStream_t s)
{
    if (with_cost) k_lse_rows<MODE_ROW, true><<<grid, kWarpNT, 0, s>>>(cv, w.G, w.Gk, w);
    else k_lse_rows<MODE_ROW, false><<<grid, kWarpNT, 0, s>>>(cv, w.G, w.Gk, w);
    return cudaGetLastError();
}

// Column pass as a row pass over the transposed cost CT (m x n, row stride
// ldct, 16-byte aligned rows): ell_j for every column j of C.
cudaError_t launch_col_pass_transposed(const float *CT, int64_t ldct, int n, int m,
                                       const Work &w, int grid, cudaStream_t s)
{
    CostView tv;
    tv.C = CT;
    tv.ldc = ldct;
    tv.n = m;
    tv.m = n;
    tv.vec = 1;
    k_lse_rows<MODE_COL, false><<<grid, kWarpNT, 0, s>>>(tv, w.Fh, w.Fk, w);
    return cudaGetLastError();
}

int occupancy_row_pass_warp()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lse_rows<MODE_ROW, false>, kWarpNT, 0);
    return b > 0 ? b : 1;
}

// Tiled transpose CT[j][i] = C[i][j] through a padded 32 x 33 shared tile,
// coalesced on both sides; blocks (32, 8), grid (ceil(m/32), ceil(n/32)).
__global__ void k_transpose(const float *__restrict__ C, int64_t ldc, int n, int m,
                            float *__restrict__ CT, int64_t ldct)
{
    __shared__ float tile[32][33];
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int i = i0 + ty + k, j = j0 + tx;
        if (i < n && j < m) tile[ty + k][tx] = ld_stream1(C + (int64_t)i * ldc + j);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int j = j0 + ty + k, i = i0 + tx;
        if (i < n && j < m) CT[(int64_t)j * ldct + i] = tile[tx][ty + k];
    }
}

cudaError_t launch_transpose(const CostView &cv, float *CT, int64_t ldct, cudaStream_t s)
{
    dim3 grid((cv.m + 31) / 32, (cv.n + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, s>>>(cv.C, cv.ldc, cv.n, cv.m, CT, ldct);
    return cudaGetLastError();
}

}  // namespace accsink

// Costs built on the fly from point clouds (Sec. 5: squared Euclidean for
// colour transfer, cosine 1 - <x, y> for word alignment); no n x m matrix is
// stored.
//
// Precision. The problem is the cost formed in FP64 from the FP32 points, and
// at eps = 1e-3 every exponent must be right to ~1e-7, so each s C_ij (s the
// scale, 1 or 1 / max C) must be right to ~1e-10. FP32 products (or TF32
// tensor-core tiles) are four orders short. Instead the kernels use the exact
// expansion
//     G_j - s C_ij = (G_j - By_j) - Bx_i + sum_k x_ik Q_jk,
// with Bx_i = s ||x_i||^2, By_j = s ||y_j||^2, Q_j = 2 s y_j (squared
// Euclidean) or Bx_i = 0, By_j = s, Q_j = s y_j (cosine). Bx, By, Q and the
// operand (G_j - By_j) are precomputed in FP64 and held as FP32 (hi, lo)
// pairs; each product x_ik Q_jk is formed exactly with an FMA and accumulated
// with Fast2Sum into a double-float sum. The operand shifts make the running
// sum dominate every product (see setup), so Fast2Sum is exact at every step.
// The column pass is the same kernel with the roles of X and Y swapped.
#include <float.h>

#include "accsink_internal.cuh"

namespace accsink {

namespace {

constexpr int kPtNT = 256;
constexpr int kPtU = 2;   // float4 column slots per lane per chunk

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

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

}  // namespace

// rows r of P (AoS, nr x d) against columns c of Q (SoA hi/lo, d x ldq):
//   h + l = A_c - B_r + sum_k P_rk Q_kc   (A = Ah + Al per column, B per row)
// MODE 0 (row pass): A = G - By, B = Bx, finish u_i, the column operand
//   A'_i = F_i - Bx_i and the CTA partials (dual, cost).
// MODE 1 (column pass): A = A', B = By, finish ell_j.
template <int MODE, int DMAX, bool WITH_COST>
__global__ void __launch_bounds__(kPtNT) k_lse_points(PointView pv, Work w)
{
    DevState *st = w.st;
    if (!w.ignore_done && *(volatile int32_t *)&st->done) return;
    if (MODE == 0 && blockIdx.x == 0 && threadIdx.x == 0) st->barrier = 0u;

    const float kh = st->k_hi, kl = st->k_lo;
    const int nr = pv.nr, nc = pv.nc, d = pv.d;
    const int64_t ldq = pv.ldq;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * kPtNT + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kPtNT) >> 5;
    const int nc4 = (nc + 3) >> 2;   // float4 groups (arrays padded to 4)
    constexpr int kStep = 32 * kPtU;

    double my_dual = 0.0, my_cost = 0.0;
    for (int r = gwarp; r < nr; r += nwarps) {
        float p[DMAX];
#pragma unroll
        for (int k = 0; k < DMAX; ++k) p[k] = (k < d) ? pv.P[(int64_t)r * d + k] : 0.0f;
        const float bh = pv.Bh[r], bl = pv.Bl[r];
        Acc acc = {0.0f, 0.0f, 0.0f};
        Acc cacc = {0.0f, 0.0f, 0.0f};
        for (int vb = 0; vb < nc4; vb += kStep) {
            float hh[kPtU][4], ll[kPtU][4], cc[kPtU][4];
            float cm = acc.R;
#pragma unroll
            for (int u = 0; u < kPtU; ++u) {
                const int v = vb + lane + 32 * u;
                if (v < nc4) {
                    const float4 ah = __ldg(reinterpret_cast<const float4 *>(pv.Ah) + v);
                    const float4 al = __ldg(reinterpret_cast<const float4 *>(pv.Al) + v);
                    float h[4] = {ah.x, ah.y, ah.z, ah.w};
                    float l[4] = {al.x, al.y, al.z, al.w};
                    float dt[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        // h - B: Fast2Sum (|A| >= |B| by the operand shift)
                        const float hn = h[e] - bh;
                        const float z = hn - h[e];
                        l[e] += (-bh - z) - bl;
                        h[e] = hn;
                    }
#pragma unroll
                    for (int k = 0; k < DMAX; ++k) {
                        if (k < d) {
                            const float4 qh = __ldg(reinterpret_cast<const float4 *>(pv.Qh + k * ldq) + v);
                            const float4 ql = __ldg(reinterpret_cast<const float4 *>(pv.Ql + k * ldq) + v);
                            const float qhv[4] = {qh.x, qh.y, qh.z, qh.w};
                            const float qlv[4] = {ql.x, ql.y, ql.z, ql.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float pr = p[k] * qhv[e];
                                float pe = fmaf(p[k], qhv[e], -pr);    // exact product error
                                pe = fmaf(p[k], qlv[e], pe);
                                const float hn = h[e] + pr;            // Fast2Sum, |h| >= |pr|
                                const float z = hn - h[e];
                                l[e] += (pr - z) + pe;
                                h[e] = hn;
                                if (WITH_COST) dt[e] = fmaf(p[k], qhv[e], dt[e]);
                            }
                        }
                    }
                    const int c0 = 4 * v;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const bool ok = c0 + e < nc;
                        hh[u][e] = ok ? h[e] : 0.0f;
                        ll[u][e] = ok ? l[e] : -INFINITY;
                        if (WITH_COST) cc[u][e] = ok ? (bh + pv.Ch[c0 + e] - dt[e]) : 0.0f;
                        cm = fmaxf(cm, hh[u][e]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        hh[u][e] = 0.0f;
                        ll[u][e] = -INFINITY;
                        cc[u][e] = 0.0f;
                    }
                }
            }
            if (cm > acc.R) {
                const float f = exp2_scaled(acc.R - cm, kh, kl);
                acc.S *= f;
                acc.K *= f;
                if (WITH_COST) { cacc.S *= f; cacc.K *= f; }
                acc.R = cm;
            }
            const float R = acc.R;
            float cs = 0.0f, ccs = 0.0f;
#pragma unroll
            for (int u = 0; u < kPtU; ++u) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float t = hh[u][e] - R;
                    const float pterm = ex2_approx(fmaf(t, kh, fmaf(t, kl, ll[u][e] * kh)));
                    cs += pterm;
                    if (WITH_COST) ccs = fmaf(cc[u][e], pterm, ccs);
                }
            }
            kahan(acc, cs);
            if (WITH_COST) kahan(cacc, ccs);
        }
        // lane merge (double-float tree), FP64 finish by lane 0
        const float Rrow = warp_max(acc.R);
        const float sc = exp2_scaled(acc.R - Rrow, kh, kl);
        float hi, lo, chi = 0.f, clo = 0.f;
        two_sum(acc.S * sc, -acc.K * sc, hi, lo);
        if (WITH_COST) two_sum(cacc.S * sc, -cacc.K * sc, chi, clo);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
            const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
            float s2, e2;
            two_sum(hi, ohi, s2, e2);
            lo = lo + olo + e2;
            two_sum(s2, lo, hi, lo);
            if (WITH_COST) {
                const float ochi = __shfl_xor_sync(0xffffffffu, chi, o);
                const float oclo = __shfl_xor_sync(0xffffffffu, clo, o);
                two_sum(chi, ochi, s2, e2);
                clo = clo + oclo + e2;
                two_sum(s2, clo, chi, clo);
            }
        }
        if (lane == 0) {
            const double S = (double)hi + (double)lo;
            if (MODE == 1) {
                w.ell[r] = ((double)Rrow - st->shift_f) * st->inv_eps_c + log(S);
            } else {
                const double lse = ((double)Rrow - st->shift_g) * st->inv_eps_c + log(S);
                const double ui = w.loga[r] - lse;
                w.u[r] = ui;
                // column-pass operand A'_r = F_r - Bx_r, F = eps u + shift_f
                const double A2 = st->eps_c * ui + st->shift_f - w.Bx64[r];
                const float A2h = (float)A2;
                w.Fh[r] = A2h;
                w.Fk[r] = (float)(A2 - (double)A2h);
                my_dual += w.a[r] * ui;
                if (WITH_COST) {
                    // row weight: a_r after the row pass, or the mass of row r
                    // under given potentials f (f_r / eps + LSE_r)
                    const double wr = w.f_given ? exp(w.f_given[r] / st->eps_user + lse) : w.a[r];
                    my_cost += wr * (((double)chi + (double)clo) / S);
                }
            }
        }
    }
    if (MODE == 1) return;
    __shared__ double sh[2][kPtNT / 32];
    if (lane == 0) {
        sh[0][threadIdx.x >> 5] = my_dual;
        sh[1][threadIdx.x >> 5] = my_cost;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double dd = 0.0, c = 0.0;
        for (int q = 0; q < kPtNT / 32; ++q) { dd += sh[0][q]; c += sh[1][q]; }
        w.rowpart[2 * blockIdx.x + 0] = dd;
        w.rowpart[2 * blockIdx.x + 1] = c;
    }
}

template <int MODE, bool WC>
static cudaError_t launch_pts(const PointView &pv, const Work &w, int grid, cudaStream_t s)
{
    if (pv.d <= 4) k_lse_points<MODE, 4, WC><<<grid, kPtNT, 0, s>>>(pv, w);
    else if (pv.d <= 16) k_lse_points<MODE, 16, WC><<<grid, kPtNT, 0, s>>>(pv, w);
    else k_lse_points<MODE, 64, WC><<<grid, kPtNT, 0, s>>>(pv, w);
    return cudaGetLastError();
}

cudaError_t launch_points_pass(const PointView &pv, const Work &w, int grid, int mode,
                               bool with_cost, cudaStream_t s)
{
    if (mode == 1) return launch_pts<1, false>(pv, w, grid, s);
    if (with_cost) return launch_pts<0, true>(pv, w, grid, s);
    return launch_pts<0, false>(pv, w, grid, s);
}

int occupancy_points_pass()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lse_points<0, 4, false>, kPtNT, 0);
    return b > 0 ? b : 1;
}

// ------------------------------------------------------------------------
// Set-up of a point-cloud solve.
// ------------------------------------------------------------------------

// Per row i of X: max_j ||x_i - y_j||^2 (or 1 - <x_i, y_j>) in double-float
// (exact differences and products), written as FP64 (MAX_TO_ONE scaling).
template <int DMAX>
__global__ void __launch_bounds__(kPtNT) k_points_rowmax(const float *X, const float *Y, int n,
                                                         int m, int d, int kind, double *rowmax)
{
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * kPtNT + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kPtNT) >> 5;
    for (int i = gwarp; i < n; i += nwarps) {
        float x[DMAX];
#pragma unroll
        for (int k = 0; k < DMAX; ++k) x[k] = (k < d) ? X[(int64_t)i * d + k] : 0.0f;
        float bh = -INFINITY, bl = 0.0f;
        for (int j = lane; j < m; j += 32) {
            float h = 0.0f, l = 0.0f;
#pragma unroll
            for (int k = 0; k < DMAX; ++k) {
                if (k < d) {
                    const float y = Y[(int64_t)j * d + k];
                    float term, te;
                    if (kind == 1) {
                        float dh, de;
                        two_sum(x[k], -y, dh, de);          // exact difference
                        term = dh * dh;                      // (dh + de)^2 to double-float
                        te = fmaf(dh, dh, -term) + 2.0f * dh * de;
                    } else {
                        term = x[k] * y;
                        te = fmaf(x[k], y, -term);
                    }
                    float s2, e2;
                    two_sum(h, term, s2, e2);
                    l += e2 + te;
                    h = s2;
                }
            }
            if (kind != 1) {   // cosine: 1 - <x, y>
                float s2, e2;
                two_sum(1.0f, -h, s2, e2);
                h = s2;
                l = e2 - l;
            }
            two_sum(h, l, h, l);
            if (h > bh || (h == bh && l > bl)) { bh = h; bl = l; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, bh, o);
            const float ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (oh > bh || (oh == bh && ol > bl)) { bh = oh; bl = ol; }
        }
        if (lane == 0) rowmax[i] = (double)bh + (double)bl;
    }
}

cudaError_t launch_points_rowmax(const float *X, const float *Y, int n, int m, int d, int kind,
                                 double *rowmax, int grid, cudaStream_t s)
{
    if (d <= 4) k_points_rowmax<4><<<grid, kPtNT, 0, s>>>(X, Y, n, m, d, kind, rowmax);
    else if (d <= 16) k_points_rowmax<16><<<grid, kPtNT, 0, s>>>(X, Y, n, m, d, kind, rowmax);
    else k_points_rowmax<64><<<grid, kPtNT, 0, s>>>(X, Y, n, m, d, kind, rowmax);
    return cudaGetLastError();
}

// Scale s = 1 / max C (or 1), from the row maxima; one block.
__global__ void k_points_scale(const double *rowmax, int n, int scale_max, double *out2)
{
    __shared__ double sh[256];
    double mx = -DBL_MAX;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, rowmax[i]);
    sh[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = sh[0];                                     // max C
        out2[1] = (scale_max && sh[0] > 0.0) ? 1.0 / sh[0] : 1.0;   // s
    }
}

// Bx, By in FP64 and as pairs; Q (scaled Y) and Q' (scaled X) in SoA pairs;
// per-block maxima for the shift bound and a count of non-finite coordinates. `scal` = {max C, s}.
__global__ void k_points_setup(const float *X, const float *Y, int n, int m, int d, int kind,
                               const double *scal, Work w, double *blockmax)
{
    const double s = scal[1];
    const double qs = (kind == 1) ? 2.0 * s : s;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    double mbx = 0.0, mby = 0.0, mdot = 0.0, nbad = 0.0;
    // rows (X): Bx and Q' = qs X
    for (int64_t i = tid; i < n; i += nthr) {
        double nx = 0.0, ax = 0.0;
        for (int k = 0; k < d; ++k) {
            const double xv = (double)X[i * d + k];
            if (!isfinite(xv)) nbad += 1.0;
            nx += xv * xv;
            ax = fmax(ax, fabs(xv));
            const double q = qs * xv;
            const float qh = (float)q;
            w.PXh[(int64_t)k * w.ldx + i] = qh;
            w.PXl[(int64_t)k * w.ldx + i] = (float)(q - (double)qh);
        }
        const double bx = (kind == 1) ? s * nx : 0.0;
        w.Bx64[i] = bx;
        const float bh = (float)bx;
        w.Bxh[i] = bh;
        w.Bxl[i] = (float)(bx - (double)bh);
        mbx = fmax(mbx, bx);
        mdot = fmax(mdot, ax);
    }
    double mdoty = 0.0;
    for (int64_t j = tid; j < m; j += nthr) {
        double ny = 0.0, ay = 0.0;
        for (int k = 0; k < d; ++k) {
            const double yv = (double)Y[j * d + k];
            if (!isfinite(yv)) nbad += 1.0;
            ny += yv * yv;
            ay = fmax(ay, fabs(yv));
            const double q = qs * yv;
            const float qh = (float)q;
            w.PYh[(int64_t)k * w.ldy + j] = qh;
            w.PYl[(int64_t)k * w.ldy + j] = (float)(q - (double)qh);
        }
        const double by = (kind == 1) ? s * ny : s;
        w.By64[j] = by;
        const float bh = (float)by;
        w.Byh[j] = bh;
        w.Byl[j] = (float)(by - (double)bh);
        mby = fmax(mby, by);
        mdoty = fmax(mdoty, ay);
    }
    // padding of the SoA rows and pair arrays to a multiple of 4 (zeros)
    for (int64_t i = n + tid; i < w.ldx; i += nthr) {
        for (int k = 0; k < d; ++k) { w.PXh[(int64_t)k * w.ldx + i] = 0.f; w.PXl[(int64_t)k * w.ldx + i] = 0.f; }
    }
    for (int64_t j = m + tid; j < w.ldy; j += nthr) {
        for (int k = 0; k < d; ++k) { w.PYh[(int64_t)k * w.ldy + j] = 0.f; w.PYl[(int64_t)k * w.ldy + j] = 0.f; }
    }
    __shared__ double sh[5][256];
    sh[0][threadIdx.x] = mbx;
    sh[1][threadIdx.x] = mby;
    sh[2][threadIdx.x] = mdot;
    sh[3][threadIdx.x] = mdoty;
    sh[4][threadIdx.x] = nbad;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        for (int q = 0; q < (int)blockDim.x; ++q) {
            a0 = fmax(a0, sh[0][q]); a1 = fmax(a1, sh[1][q]);
            a2 = fmax(a2, sh[2][q]); a3 = fmax(a3, sh[3][q]);
            a4 += sh[4][q];
        }
        double *o = blockmax + 5 * blockIdx.x;
        o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3; o[4] = a4;
    }
}

// Writes the cost-statistics record the init kernel reads: max C, a lower
// bound of s C (-bound), and the bound itself in place of max |C|:
//   bound = 2 (max Bx + max By + d qs max|x| max|y|),
// which makes every partial sum of the expansion dominate the next term.
__global__ void k_points_stats(const double *blockmax, int nblk, int d, int kind,
                               const double *scal, double *statpart)
{
    if (threadIdx.x != 0) return;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    for (int b = 0; b < nblk; ++b) {
        const double *o = blockmax + 5 * b;
        a0 = fmax(a0, o[0]); a1 = fmax(a1, o[1]);
        a2 = fmax(a2, o[2]); a3 = fmax(a3, o[3]);
        a4 += o[4];
    }
    const double s = scal[1];
    const double qs = (kind == 1) ? 2.0 * s : s;
    const double bound = 2.0 * (a0 + a1 + (double)d * qs * a2 * a3) + 1e-30;
    statpart[0] = scal[0];       // max C of the input (reported)
    statpart[1] = -bound;
    statpart[2] = bound;
    statpart[3] = a4;            // non-finite coordinates
}

cudaError_t launch_points_setup(const float *X, const float *Y, int n, int m, int d, int kind,
                                int scale_max, const Work &w, double *scal, double *blockmax,
                                int nblk, cudaStream_t s)
{
    k_points_scale<<<1, 256, 0, s>>>(w.rowmax, n, scale_max, scal);
    k_points_setup<<<nblk, 256, 0, s>>>(X, Y, n, m, d, kind, scal, w, blockmax);
    k_points_stats<<<1, 32, 0, s>>>(blockmax, nblk, d, kind, scal, w.statpart);
    return cudaGetLastError();
}

}  // namespace accsink

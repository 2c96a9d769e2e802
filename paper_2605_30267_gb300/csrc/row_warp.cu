// Log-sum-exp over the rows of a row-major FP32 matrix X, one warp per row
// (the 128-bit-aligned path). It serves both passes of an S evaluation:
//   MODE_ROW: X = C, operand G (columns): u_i and the column-pass operand;
//   MODE_COL: X = C^T (a transposed copy kept by the solver), operand F
//             (rows of C): ell_j = LSE_i((f_i - C_ij) / eps).
//
// Every warp streams whole rows on its own: no CTA barrier inside the row
// loop, so no warp ever waits for another. Lanes read 128-bit slots of
// the row (a warp covers 512 contiguous bytes per slot); the column operand
// (G, gamma k) is read through L1, where it stays resident because the cost
// is read with non-allocating loads. The next chunk of the row is loaded
// while the current one is reduced (register double buffering), so each warp
// keeps 2 x U x 512 bytes of the cost in flight.
//
// Per element the arithmetic is the exact-split scheme of the plain row
// pass. The per-row merge across lanes is done in FP32 double-float (no FP64
// pipe in the hot loop). The FP64 finish of a row (log, u_i, F_i) is
// deferred: the merged sums wait in a per-warp shared-memory slot, and every
// 32 rows the warp finishes them together, one row per lane. GB300's FP64
// rate is 1/64 of FP32, so a finish in one lane per row held the warp (and
// its next loads) for longer than the finish of 32 rows at once.
//
// Load balance: rows are dealt to warps whole, except the rows of a last,
// part-empty wave, which are split into column parts (plan_row_split) so
// every resident warp stays busy to the end; the last part of such a row to
// finish merges the parts in part order (merge_parts), so the result does not
// depend on the order in which they finished.
#include <algorithm>
#include <cfloat>
#include <cstdint>

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

// term_s in two halves: q = e k_hi + gamma k (e the rounding error of
// s = G - c) before the running reference is known, then the exponential.
// Same operations and roundings as term_s.
__device__ __forceinline__ float split_q(float s, float G, float gk, float c, float kh)
{
    const float z = s - G;
    const float e = -c - z;
    return fmaf(e, kh, gk);
}

__device__ __forceinline__ float term_q(float s, float q, float R, float kh, float kl)
{
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

// A finished row's warp-merged sums, parked in a shared-memory slot of its
// warp until 32 rows (or the warp's last row) are ready: the FP64 finish
// (log, u_i, F_i) then runs once for all of them, one row per lane, instead
// of once per row in lane 0.
struct Parked {
    float R, hi, lo, chi, clo;
    int row;
};

// Outputs of the FP64 row finish, passed by value to the out-of-line finish
// (only a few pointers, not the whole parameter block).
struct FinishOut {
    double *ell;                        // column pass
    const double *loga, *a, *f_given;   // row pass
    double *u;
    float2 *FF;
    float *Fh, *Fk;
};

__device__ __forceinline__ FinishOut finish_out(const Work &w)
{
    return FinishOut{w.ell, w.loga, w.a, w.f_given, w.u, w.FF, w.Fh, w.Fk};
}

// FP64 finish of the parked rows, one per lane: ell_j (column pass), or u_i
// and the column-pass operand F_i (row pass). Returns the lane's share of
// the transport-cost sum (WITH_COST), else 0.
template <int MODE, bool WITH_COST>
__device__ __noinline__ double finish_parked(const Parked *slots, int count, int lane,
                                             const DevState *st, FinishOut o, float kh)
{
    __syncwarp();
    if (lane >= count) return 0.0;
    const Parked p = slots[lane];
    const int i = p.row;
    const double S = (double)p.hi + (double)p.lo;
    if (MODE == MODE_COL) {
        o.ell[i] = ((double)p.R - st->shift_f) * st->inv_eps_c + log(S);
        return 0.0;
    }
    const double lse = ((double)p.R - st->shift_g) * st->inv_eps_c + log(S);
    const double ui = o.loga[i] - lse;
    o.u[i] = ui;
    const double F = st->eps_c * ui + st->shift_f;
    const float Fh = (float)F;
    const float Fl = (float)(F - (double)Fh);
    o.FF[i] = make_float2(Fh, Fl * kh);
    o.Fh[i] = Fh;
    o.Fk[i] = Fl * kh;
    if (!WITH_COST) return 0.0;
    const double CS = (double)p.chi + (double)p.clo;
    const double wi = o.f_given ? exp(o.f_given[i] / st->eps_user + lse) : o.a[i];
    return wi * (CS / S);
}

// Double-float (hi, lo) sum over the warp by a fixed xor tree (every lane
// ends with the total).
__device__ __forceinline__ void warp_sum_df(float &hi, float &lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, ohi, s, e);
        lo = lo + olo + e;
        two_sum(s, lo, hi, lo);
    }
}

// Merges the column parts of one split row from their records (reference R,
// double-float sum (hi, lo) relative to R; (chi, clo) for the cost): lane q
// takes part q, scales it to the common reference (the product split exactly
// by an FMA), and the warp adds the parts in a fixed order, so the result
// does not depend on which part finished last.
template <bool WITH_COST>
__device__ __noinline__ void merge_parts(const float4 *prec, const float2 *pcrec, int parts,
                                         int lane, float kh, float kl, float &R, float &hi,
                                         float &lo, float &chi, float &clo)
{
    const bool have = lane < parts;
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 c = make_float2(0.f, 0.f);
    if (have) {
        r = __ldcg(prec + lane);
        if (WITH_COST) c = __ldcg(pcrec + lane);
    }
    R = warp_max(have ? r.x : -INFINITY);
    const float sc = have ? exp2_scaled(r.x - R, kh, kl) : 0.0f;
    float h = __fmul_rn(r.y, sc);
    float l = fmaf(r.y, sc, -h) + r.z * sc;
    two_sum(h, l, hi, lo);
    warp_sum_df(hi, lo);
    if (WITH_COST) {
        h = __fmul_rn(c.x, sc);
        l = fmaf(c.x, sc, -h) + c.y * sc;
        two_sum(h, l, chi, clo);
        warp_sum_df(chi, clo);
    }
}

// Work units: rows [0, nfull) whole, then every row of [nfull, n) in `parts`
// column parts: unit nfull + q * parts + p is part p of row nfull + q and
// covers the float4 slots [p * part4, min(m4, (p + 1) * part4)); the last
// part of a row also takes its m % 4 ragged columns. The split rows are the
// ones a last, part-empty wave of whole rows would leave to a few warps.
template <int MODE, bool WITH_COST>
__global__ void __launch_bounds__(kWarpNT, WITH_COST ? 2 : 3) k_lse_rows(CostView cv, const float *Oh,
                                                      const float *Ok, Work w, int nfull,
                                                      int parts, int part4)
{
    DevState *st = w.st;
    if (!w.ignore_done && *(volatile int32_t *)&st->done) return;
    if (MODE == MODE_ROW && blockIdx.x == 0 && threadIdx.x == 0)
        st->barrier = 0u;   // for the step kernel

    const float kh = st->k_hi, kl = st->k_lo;
    const int m = cv.m;
    const int64_t ldc = cv.ldc;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * kWarpNT + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kWarpNT) >> 5;
    const int m4 = m >> 2;
    const int tail0 = 4 * m4;
    const float4 *G4 = reinterpret_cast<const float4 *>(Oh);
    const float4 *Gk4 = reinterpret_cast<const float4 *>(Ok);
    constexpr int kStep = 32 * kU;     // float4 slots per chunk per warp

    __shared__ Parked park[kWarpNT / 32][32];
    Parked *slots = park[threadIdx.x >> 5];
    double my_cost = 0.0;
    int parked = 0;
    for (int unit = gwarp; unit < nfull + (cv.n - nfull) * parts; unit += nwarps) {
        // (the row and part are recomputed after the chunk loop rather than
        // kept live across it)
        int v0 = 0, v1 = m4;
        const float4 *row;
        {
            int i = unit;
            if (unit >= nfull) {
                const int q = (unit - nfull) / parts;
                i = nfull + q;
                v0 = (unit - nfull - q * parts) * part4;
                v1 = min(m4, v0 + part4);
            }
            row = reinterpret_cast<const float4 *>(cv.C + (int64_t)i * ldc);
        }
        Acc acc = {0.0f, 0.0f, 0.0f};
        Acc cacc = {0.0f, 0.0f, 0.0f};
        float4 cbuf[kU];
        // prefetch the first chunk
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int v = v0 + lane + 32 * u;
            cbuf[u] = (v < v1) ? ld_stream4(reinterpret_cast<const float *>(row + v))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int vb = v0; vb < v1; vb += kStep) {
            float4 c[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) c[u] = cbuf[u];
            // issue the next chunk's loads before reducing this one
            const int nb = vb + kStep;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = nb + lane + 32 * u;
                if (v < v1) cbuf[u] = ld_stream4(reinterpret_cast<const float *>(row + v));
            }
            // per element: s = G - c (rounded) and q = e k_hi + gamma k with e
            // the rounding error of s, so that only (s, q) stay live until
            // the exponentials (c too for the cost sum)
            float4 sv[kU], qv[kU];
            float cm = acc.R;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = vb + lane + 32 * u;
                float4 g, gk;
                if (v < v1) {
                    g = __ldg(G4 + v);
                    gk = __ldg(Gk4 + v);
                } else {
                    g = make_float4(0.f, 0.f, 0.f, 0.f);
                    gk = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
                    c[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                sv[u] = make_float4(g.x - c[u].x, g.y - c[u].y, g.z - c[u].z, g.w - c[u].w);
                qv[u] = make_float4(split_q(sv[u].x, g.x, gk.x, c[u].x, kh),
                                    split_q(sv[u].y, g.y, gk.y, c[u].y, kh),
                                    split_q(sv[u].z, g.z, gk.z, c[u].z, kh),
                                    split_q(sv[u].w, g.w, gk.w, c[u].w, kh));
                cm = fmaxf(cm, fmaxf(fmaxf(sv[u].x, sv[u].y), fmaxf(sv[u].z, sv[u].w)));
            }
            if (cm > acc.R) {
                const float f = exp2_scaled(acc.R - cm, kh, kl);
                acc.S = __fmul_rn(acc.S, f);
                acc.K = __fmul_rn(acc.K, f);
                if (WITH_COST) { cacc.S = __fmul_rn(cacc.S, f); cacc.K = __fmul_rn(cacc.K, f); }
                acc.R = cm;
            }
            const float R = acc.R;
            float cs[kU], ccs[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const float p0 = term_q(sv[u].x, qv[u].x, R, kh, kl);
                const float p1 = term_q(sv[u].y, qv[u].y, R, kh, kl);
                const float p2 = term_q(sv[u].z, qv[u].z, R, kh, kl);
                const float p3 = term_q(sv[u].w, qv[u].w, R, kh, kl);
                cs[u] = (p0 + p1) + (p2 + p3);
                if (WITH_COST)
                    ccs[u] = fmaf(c[u].x, p0, fmaf(c[u].y, p1, fmaf(c[u].z, p2, c[u].w * p3)));
            }
            float csum = (cs[0] + cs[1]) + (cs[2] + cs[3]);
            kahan(acc, csum);
            if (WITH_COST) kahan(cacc, (ccs[0] + ccs[1]) + (ccs[2] + ccs[3]));
        }
        int i = unit, part = 0;
        if (unit >= nfull) {
            const int q = (unit - nfull) / parts;
            i = nfull + q;
            part = unit - nfull - q * parts;
        }
        // ragged tail (m % 4 columns), in the row's last part
        if ((unit < nfull || part == parts - 1) && tail0 + lane < m) {
            const int j = tail0 + lane;
            const float Gj = Oh[j], Gkj = Ok[j];
            const float c = ld_stream1(cv.C + (int64_t)i * ldc + j);
            const float s = Gj - c;
            if (s > acc.R) {
                const float f = exp2_scaled(acc.R - s, kh, kl);
                acc.S = __fmul_rn(acc.S, f);
                acc.K = __fmul_rn(acc.K, f);
                if (WITH_COST) { cacc.S = __fmul_rn(cacc.S, f); cacc.K = __fmul_rn(cacc.K, f); }
                acc.R = s;
            }
            const float p = term_s(s, Gj, Gkj, c, acc.R, kh, kl);
            kahan(acc, p);
            if (WITH_COST) kahan(cacc, c * p);
        }
        // merge the lanes: common reference, then a double-float tree sum
        float Rrow = warp_max(acc.R);
        const float sc = exp2_scaled(acc.R - Rrow, kh, kl);
        float hi, lo;
        two_sum(__fmul_rn(acc.S, sc), -__fmul_rn(acc.K, sc), hi, lo);
        float chi = 0.f, clo = 0.f;
        if (WITH_COST) two_sum(__fmul_rn(cacc.S, sc), -__fmul_rn(cacc.K, sc), chi, clo);
        warp_sum_df(hi, lo);
        if (WITH_COST) warp_sum_df(chi, clo);
        if (unit >= nfull) {
            // publish this part; the last of the row's parts merges them
            const int64_t rbase = (int64_t)(i - nfull) * parts;
            int last = 0;
            if (lane == 0) {
                w.prec[rbase + part] = make_float4(Rrow, hi, lo, 0.0f);
                if (WITH_COST) w.pcrec[rbase + part] = make_float2(chi, clo);
                __threadfence();
                last = atomicAdd(&w.pcnt[i - nfull], 1u) == (unsigned)(parts - 1);
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (!last) continue;
            __threadfence();
            merge_parts<WITH_COST>(w.prec + rbase, w.pcrec + rbase, parts, lane, kh, kl, Rrow,
                                   hi, lo, chi, clo);
            if (lane == 0) w.pcnt[i - nfull] = 0u;   // ready for the next pass
        }
        if (lane == 0) slots[parked] = Parked{Rrow, hi, lo, chi, clo, i};
        if (++parked == 32) {
            my_cost += finish_parked<MODE, WITH_COST>(slots, parked, lane, st, finish_out(w), kh);
            __syncwarp();
            parked = 0;
        }
    }
    my_cost += finish_parked<MODE, WITH_COST>(slots, parked, lane, st, finish_out(w), kh);
    if (!WITH_COST) return;
    // the final pass: per-warp cost sums in a fixed lane order, then per-CTA
    // partials in a fixed order over the CTA's warps (the dual's <a, u> is
    // summed by the step kernel from u)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_cost += __shfl_xor_sync(0xffffffffu, my_cost, o);
    __shared__ double sh[kWarpNT / 32];
    if (lane == 0) sh[threadIdx.x >> 5] = my_cost;
    __syncthreads();
    if (threadIdx.x == 0) {
        double c = 0.0;
        for (int q = 0; q < kWarpNT / 32; ++q) c += sh[q];
        w.rowpart[2 * blockIdx.x + 0] = 0.0;
        w.rowpart[2 * blockIdx.x + 1] = c;
    }
}

// Plans the units of a warp-per-row pass over `rows` rows of `cols` columns
// with `max_warps` warps resident. Whole rows fill the full waves; when the
// rows left for a last wave would leave at least half of the warps idle, each
// of them is split into P = min(32, max_warps / rest, chunks / 4) parts
// (parts of at least four chunks; P <= 32 for the merge's one lane per part),
// and every warp is launched. Otherwise k = ceil(rows / max_warps) rows per
// warp with just enough warps for that.
RowSplit plan_row_split(int rows, int cols, int64_t max_warps)
{
    constexpr int64_t kChunk4 = 32 * kU;     // float4 slots per chunk
    constexpr int64_t kMinPartChunks = 4;
    constexpr int64_t kMaxParts = 32;
    RowSplit r;
    const int m4 = cols / 4;
    const int64_t nch = (m4 + kChunk4 - 1) / kChunk4;
    max_warps = std::max<int64_t>(1, max_warps);
    r.nfull = rows;
    r.parts = 1;
    r.part4 = m4;
    const int64_t full = (int64_t)rows / max_warps * max_warps;
    const int64_t rest = rows - full;
    if (rest > 0) {
        const int64_t P = std::min(kMaxParts, std::min(max_warps / rest, nch / kMinPartChunks));
        if (P >= 2) {
            const int64_t per = (nch + P - 1) / P;   // chunks per part
            r.nfull = (int)full;
            r.part4 = (int)(per * kChunk4);
            r.parts = (int)((nch + per - 1) / per);  // every part non-empty
        }
    }
    int64_t warps;
    if (r.parts > 1) {
        warps = std::min<int64_t>(max_warps, full + rest * r.parts);
    } else {
        const int64_t k = std::max<int64_t>(1, (rows + max_warps - 1) / max_warps);
        warps = (rows + k - 1) / k;
    }
    r.grid = (int)std::max<int64_t>(1, (warps + kWarpNT / 32 - 1) / (kWarpNT / 32));
    return r;
}

int64_t row_split_records(const RowSplit &r, int rows)
{
    return r.parts > 1 ? (int64_t)(rows - r.nfull) * r.parts : 0;
}

cudaError_t launch_row_pass_warp(const CostView &cv, const Work &w, int grid,
                                 const RowSplit &sp, bool with_cost, cudaStream_t s)
{
    // the final pass (with the cost sum) is never split: its per-CTA cost
    // partials then do not depend on which warp finished a row
    if (with_cost) {
        k_lse_rows<MODE_ROW, true><<<grid, kWarpNT, 0, s>>>(cv, w.G, w.Gk, w, cv.n, 1, cv.m / 4);
    } else if (sp.parts > 1) {
        k_lse_rows<MODE_ROW, false><<<grid, kWarpNT, 0, s>>>(cv, w.G, w.Gk, w, sp.nfull, sp.parts,
                                                              sp.part4);
    } else {
        k_lse_rows<MODE_ROW, false><<<grid, kWarpNT, 0, s>>>(cv, w.G, w.Gk, w, cv.n, 1, cv.m / 4);
    }
    return cudaGetLastError();
}

// Column pass as a row pass over the transposed cost CT (m x n, row stride
// ldct, 16-byte aligned rows): ell_j for every column j of C.
cudaError_t launch_col_pass_transposed(const float *CT, int64_t ldct, int n, int m,
                                       const Work &w, int grid, const RowSplit &sp,
                                       cudaStream_t s)
{
    CostView tv;
    tv.C = CT;
    tv.ldc = ldct;
    tv.n = m;
    tv.m = n;
    tv.vec = 1;
    if (sp.parts > 1)
        k_lse_rows<MODE_COL, false><<<grid, kWarpNT, 0, s>>>(tv, w.Fh, w.Fk, w, sp.nfull, sp.parts,
                                                              sp.part4);
    else
        k_lse_rows<MODE_COL, false><<<grid, kWarpNT, 0, s>>>(tv, w.Fh, w.Fk, w, m, 1, n / 4);
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

// C^T and the cost statistics (max C, min C, max |C|, count of non-finite
// entries over the finite ones, as k_cost_stats) in one read of C, for a
// 16-byte-aligned C with ldc % 4 == 0. Each CTA walks 64 x 64 tiles (row-major
// tile order, grid-stride): 128-bit loads of the tile into shared memory
// (4 per thread), then 128-bit stores of its transpose, each gathered from a
// shared-memory column; the CTA's statistics go to statpart[4 blockIdx.x ..].
// Entries of a stored float4 past n (the padding of a C^T row) are zero; no
// column past m is read.
__global__ void __launch_bounds__(256) k_transpose_stats(const float *__restrict__ C, int64_t ldc,
                                                         int n, int m,
                                                         float *__restrict__ CT, int64_t ldct,
                                                         double *statpart, int r0, int r1)
{
    constexpr int T = 64;
    __shared__ float tile[T][T + 1];
    const int tid = threadIdx.x;
    const int tr = tid >> 4, tc = tid & 15;       // 16 threads per 64-float row segment
    const int tiles_j = (m + T - 1) / T;
    const int64_t ntiles = (int64_t)((r1 - r0 + T - 1) / T) * tiles_j;
    float mx = -FLT_MAX, mn = FLT_MAX, ab = 0.0f;
    int bad = 0;
    // tile t's four float4 of this thread (zeros outside C), and the
    // statistics of the ones inside
    auto load = [&](int64_t t, float4 (&v)[4]) {
        const int i0 = r0 + (int)(t / tiles_j) * T, j0 = (int)(t % tiles_j) * T;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + tr + 16 * r, j = j0 + 4 * tc;
            const float *src = C + (int64_t)i * ldc + j;
            if (i < r1 && j + 3 < m) {
                v[r] = ld_stream4(src);
            } else if (i < r1 && j < m) {
                // a row's last m % 4 columns: no read past column m - 1 (the
                // last row of C may end there)
                v[r] = make_float4(ld_stream1(src), j + 1 < m ? ld_stream1(src + 1) : 0.f,
                                   j + 2 < m ? ld_stream1(src + 2) : 0.f, 0.f);
            } else {
                v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    auto visit = [&](int64_t t, const float4 (&v)[4]) {
        const int i0 = r0 + (int)(t / tiles_j) * T, j0 = (int)(t % tiles_j) * T;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + tr + 16 * r, j = j0 + 4 * tc;
            if (i < r1 && j < m) {
                const float e[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (j + q >= m) continue;        // the row's padding (ldc > m)
                    if (!isfinite(e[q])) { ++bad; continue; }
                    mx = fmaxf(mx, e[q]);
                    mn = fminf(mn, e[q]);
                    ab = fmaxf(ab, fabsf(e[q]));
                }
            }
        }
    };
    float4 v[4];
    int64_t t = blockIdx.x;
    if (t < ntiles) load(t, v);
    for (; t < ntiles; t += gridDim.x) {
        const int i0 = r0 + (int)(t / tiles_j) * T, j0 = (int)(t % tiles_j) * T;
        visit(t, v);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float *row = tile[tr + 16 * r];
            row[4 * tc + 0] = v[r].x;
            row[4 * tc + 1] = v[r].y;
            row[4 * tc + 2] = v[r].z;
            row[4 * tc + 3] = v[r].w;
        }
        __syncthreads();
        // the next tile's loads go out before this tile's stores
        if (t + gridDim.x < ntiles) load(t + gridDim.x, v);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int jl = tr + 16 * r, il = 4 * tc;
            const int j = j0 + jl, i = i0 + il;
            if (j < m && i < n) {
                float4 o;
                o.x = tile[il + 0][jl];
                o.y = (i + 1 < n) ? tile[il + 1][jl] : 0.0f;
                o.z = (i + 2 < n) ? tile[il + 2][jl] : 0.0f;
                o.w = (i + 3 < n) ? tile[il + 3][jl] : 0.0f;
                *reinterpret_cast<float4 *>(CT + (int64_t)j * ldct + i) = o;
            }
        }
        __syncthreads();
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
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) { s_mx[wid] = mx; s_mn[wid] = mn; s_ab[wid] = ab; s_bad[wid] = bad; }
    __syncthreads();
    if (tid == 0) {
        for (int q = 1; q < 8; ++q) {
            mx = fmaxf(mx, s_mx[q]); mn = fminf(mn, s_mn[q]);
            ab = fmaxf(ab, s_ab[q]); bad += s_bad[q];
        }
        statpart[4 * blockIdx.x + 0] = mx;
        statpart[4 * blockIdx.x + 1] = mn;
        statpart[4 * blockIdx.x + 2] = ab;
        statpart[4 * blockIdx.x + 3] = bad;
    }
}

cudaError_t launch_transpose_stats(const CostView &cv, float *CT, int64_t ldct, const Work &w,
                                   int grid, cudaStream_t s, int r0, int r1, int part0)
{
    if (!cv.vec) return cudaErrorInvalidValue;
    if (r1 < 0) r1 = cv.n;
    if (r0 % 64 != 0 || r1 < r0 || r1 > cv.n || (r1 % 64 != 0 && r1 != cv.n))
        return cudaErrorInvalidValue;
    k_transpose_stats<<<std::max(1, grid), 256, 0, s>>>(cv.C, cv.ldc, cv.n, cv.m, CT, ldct,
                                                        w.statpart + 4 * (int64_t)part0, r0, r1);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const CostView &cv, float *CT, int64_t ldct, cudaStream_t s)
{
    dim3 grid((cv.m + 31) / 32, (cv.n + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, s>>>(cv.C, cv.ldc, cv.n, cv.m, CT, ldct);
    return cudaGetLastError();
}

}  // namespace accsink

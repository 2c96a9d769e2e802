// Costs built on the fly from point clouds (Sec. 5: squared Euclidean for
// colour transfer, cosine 1 - <x, y> for word alignment); no n x m matrix is
// stored.
//
// Precision. The problem is the cost formed in FP64 from the FP32 points, and
// at eps = 1e-3 every exponent must be right to ~1e-7, so each s C_ij (s the
// scale, 1 or 1 / max C) must be right to ~1e-10. FP32 products (or 3xTF32
// tensor-core tiles, ~2^-24 relative) are orders short. Instead the kernels
// use the exact expansion
//     G_j - s C_ij = (G_j - By_j) - Bx_i + sum_k x_ik Q_jk,
// with Bx_i = s ||x_i||^2, By_j = s ||y_j||^2, Q_j = 2 s y_j (squared
// Euclidean) or Bx_i = 0, By_j = s, Q_j = s y_j (cosine), everything
// multiplied by k = log2(e) / eps so that the sum is the exponent in log2
// units. Q and the column operand k (G_j - By_j) are precomputed in FP64 and
// held as FP32 (hi, lo) pairs; each product x_ik Q_jk is formed exactly with
// an FMA and added with Fast2Sum into a double-float sum. The operand shifts
// make the running sum dominate every product (see the set-up), so Fast2Sum
// is exact at every step. The row term Bx_i is constant along a row and is
// applied once, in FP64, when the row is finished. The column pass is the
// same kernel with the roles of X and Y swapped.
#include <float.h>

#include <algorithm>

#include <cub/device/device_radix_sort.cuh>

#include "accsink_internal.cuh"

namespace accsink {

namespace {

constexpr int kPtNT = 256;

}  // namespace

// One slot (4 consecutive columns) of one row: h + l = A_c + sum_k p_k Q_kc
// in log2 units, each product formed exactly (FMA) and added by Fast2Sum
// (exact: the operand shift makes |h| >= |p_k Q_kc| at every step, see the
// set-up).
// Small DMAX: the slot's Q columns were loaded into qh/ql once for all RW
// rows (PRE). Larger DMAX: they are read per k from Qh/Ql (L1-resident).
// f32: plain FP32 FMAs on the high parts only (precision FP32).
template <int DMAX, bool PRE>
__device__ __forceinline__ void slot_dot(const float *p, int d, const float4 &ah,
                                         const float4 &al, const float4 *qh, const float4 *ql,
                                         const float *Qh, const float *Ql, int64_t ldq, int v,
                                         float h[4], float l[4], const bool f32)
{
    h[0] = ah.x; h[1] = ah.y; h[2] = ah.z; h[3] = ah.w;
    if (f32) {
        l[0] = l[1] = l[2] = l[3] = 0.0f;
#pragma unroll
        for (int k = 0; k < DMAX; ++k) {
            if (k < d) {
                const float4 a4 =
                    PRE ? qh[k] : __ldg(reinterpret_cast<const float4 *>(Qh + k * ldq) + v);
                h[0] = fmaf(p[k], a4.x, h[0]);
                h[1] = fmaf(p[k], a4.y, h[1]);
                h[2] = fmaf(p[k], a4.z, h[2]);
                h[3] = fmaf(p[k], a4.w, h[3]);
            }
        }
        return;
    }
    l[0] = al.x; l[1] = al.y; l[2] = al.z; l[3] = al.w;
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            float4 a4, b4;
            if (PRE) {
                a4 = qh[k];
                b4 = ql[k];
            } else {
                a4 = __ldg(reinterpret_cast<const float4 *>(Qh + k * ldq) + v);
                b4 = __ldg(reinterpret_cast<const float4 *>(Ql + k * ldq) + v);
            }
            const float qv[4] = {a4.x, a4.y, a4.z, a4.w};
            const float qlv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float pr = __fmul_rn(p[k], qv[e]);   // never fused: pe is its error
                float pe = fmaf(p[k], qv[e], -pr);     // exact product error
                pe = fmaf(p[k], qlv[e], pe);
                const float hn = h[e] + pr;             // Fast2Sum
                const float z = hn - h[e];
                l[e] += (pr - z) + pe;
                h[e] = hn;
            }
        }
    }
}

// Cost entries C_ij (scaled by s) of one slot, formed directly from the
// points in FP32 for the transport cost: sum_k (x_k - y_k)^2 for squared
// Euclidean (no cancellation between norms), 1 - <x, y> for cosine.
template <int DMAX>
__device__ __forceinline__ void slot_cost(const float *p, int d, int kind, float s,
                                          const float *Pc, int c0, int nc, float cst[4])
{
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int c = min(c0 + e, nc - 1);
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < DMAX; ++k) {
            if (k < d) {
                const float y = __ldg(Pc + (int64_t)c * d + k);
                if (kind == 1) {
                    const float df = p[k] - y;
                    acc = fmaf(df, df, acc);
                } else {
                    acc = fmaf(p[k], y, acc);
                }
            }
        }
        cst[e] = s * (kind == 1 ? acc : 1.0f - acc);
    }
}

// Rows r of P against all columns of Q (see PointView), RW rows per warp so
// each column slot is loaded once per RW rows. EXACT: the dimension is DMAX
// itself (d = 2, 3, 4), so every per-k guard is resolved at compile time
// (13% fewer cycles per pass at d = 3 than the DMAX = 4 bound).
//   MODE 0 (row pass): A = k (G - By), rows of X, B64 = Bx; finishes u_i,
//     the column operand A'_i = k (F_i - Bx_i) and the CTA partials.
//   MODE 1 (column pass): A = A', rows of Y, B64 = By; finishes ell_j.
// With h_rc = k (A-term + x.Q) the row's log-sum-exp in natural units is
//   (R + log2 S) ln 2 - (B_r + shift) / eps_c.
// PRUNE (d <= 4, points sorted along a space-filling curve): a slot whose
// FP32 estimate of every exponent, for every row of the warp, lies more than
// pv.skip below the lane's running maximum (a lower bound of the row's) is
// skipped. With block records (pv.qbox, sorted solves) blocks of 64 columns
// (kBoxSlots slots) are tested instead, without loading them: an upper bound
// of the block's exponents for a row p is max A + sum_k max(p_k Qmin_k,
// p_k Qmax_k) over the block's coordinate box (for squared-Euclidean costs
// the tighter bound through the box's distance to the row, see
// k_points_abox), and a block whose bound lies more than pv.skip below the
// warp's running maximum for every row of the group is passed over; each
// lane tests one of 32 blocks at a time and the warp then works on the near
// ones two at a time (half a warp per block, a slot per lane). Blocks of 64
// columns were faster than blocks of 32 or 128 (colour solve 0.489 s against
// 0.537 and 0.504 s): smaller boxes prune more but cost more tests.
// Each row's running maximum starts just below its largest term in
// the slot that holds the column nearest to the group's first row (pv.hint,
// found once per solve from the points alone): the FP32 estimate of that term
// less the estimate's error bound, which is below an actual term of the row
// and so still a lower bound of its maximum; far slots are then skipped from
// the start of the row rather than only once the loop has reached the row's
// best columns. The hints depend only on the points, so repeated and resumed
// solves take the same steps bit for bit. Each skipped term is below
// 2^-(skip + 1) of its row's largest, and skip = 29 + ceil(log2 nc), so all
// of a row's skipped terms together stay below 2^-30 (~1e-9) of its sum:
// two orders of magnitude below the FP32 passes' own accuracy (~1e-7 in
// each log-sum-exp). The estimate A_hi + sum_k p_k Q_hi,k (and the block
// bound, with at most nine FP32 roundings for d <= 4) differs from the exact
// exponent by at most 2^-20 of the terms' magnitude |A| + sum_k |p_k| |Q_k|
// (the roundings and the dropped low parts, each below 2^-24 of it), so the
// threshold is lowered by 2^-20 of a bound on that magnitude.

// The constant c of the squared-Euclidean block bound (see k_points_abox);
// any c > 0 gives a valid bound, c = 4 k s (Q = 2 k s y) the tightest. The
// block-record kernel and the passes compute it with the same expression.
__device__ __forceinline__ float box_cq(const DevState *st, const PointView &pv)
{
    return 4.0f * (float)(st->k2 * pv.scal[1]);
}

// Running maxima at the start of a row group: every lane evaluates the FP32
// estimate of the hinted slot hv (the same loads for all lanes) and takes, per
// row, its largest term less the estimate's error bound, which stays below
// that actual term (the margin of the skip test). The slot's terms themselves
// are added in the pass's loop. Out of line: it runs once per row group and
// keeps its registers out of the loop's.
template <int DMAX, int RW>
__device__ __noinline__ void hinted_start(const PointView &pv, const float (&p)[RW][DMAX], int d,
                                          int hv, float (&R0)[RW])
{
    const float4 ah = __ldg(reinterpret_cast<const float4 *>(pv.Ah) + hv);
    float4 qh[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
        if (k < d) qh[k] = __ldg(reinterpret_cast<const float4 *>(pv.Qh + k * pv.ldq) + hv);
    const float amax = fmaxf(fmaxf(fabsf(ah.x), fabsf(ah.y)), fmaxf(fabsf(ah.z), fabsf(ah.w)));
#pragma unroll
    for (int q = 0; q < RW; ++q) {
        float mag = amax;
        float e4[4] = {ah.x, ah.y, ah.z, ah.w};
#pragma unroll
        for (int k = 0; k < DMAX; ++k) {
            if (k < d) {
                const float qm = fmaxf(fmaxf(fabsf(qh[k].x), fabsf(qh[k].y)),
                                       fmaxf(fabsf(qh[k].z), fabsf(qh[k].w)));
                mag = fmaf(fabsf(p[q][k]), qm, mag);
                e4[0] = fmaf(p[q][k], qh[k].x, e4[0]);
                e4[1] = fmaf(p[q][k], qh[k].y, e4[1]);
                e4[2] = fmaf(p[q][k], qh[k].z, e4[2]);
                e4[3] = fmaf(p[q][k], qh[k].w, e4[3]);
            }
        }
        R0[q] = fmaxf(fmaxf(e4[0], e4[1]), fmaxf(e4[2], e4[3])) - 1.0f - mag * 0x1p-20f;
    }
}

template <int MODE, int DMAX, int RW, bool WC, bool EXACT = false, bool PRUNE = false,
          bool F32 = false>
__global__ void __launch_bounds__(kPtNT) k_lse_points(PointView pv, Work w)
{
    DevState *st = w.st;
    if (!w.ignore_done && *(volatile int32_t *)&st->done) return;
    if (MODE == 0 && blockIdx.x == 0 && threadIdx.x == 0) st->barrier = 0u;

    const int nr = pv.nr, nc = pv.nc, d = EXACT ? DMAX : pv.d;
    const int64_t ldq = pv.ldq;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * kPtNT + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kPtNT) >> 5;
    const int nc4 = (nc + 3) >> 2;             // float4 slots (operands padded to 4)
    const int nfull = (nc >> 2) & ~31;         // slots in whole, unmasked 32-lane chunks
    const float cs_scale = WC ? (float)pv.scal[1] : 0.0f;
    constexpr bool PRE = DMAX <= 4;
    constexpr bool f32 = F32;   // x.Q in plain FP32 (precision FP32)
    const float4 *Ah4 = reinterpret_cast<const float4 *>(pv.Ah);
    const float4 *Al4 = reinterpret_cast<const float4 *>(pv.Al);

    double my_dual = 0.0, my_cost = 0.0;
    // row groups dealt round-robin, or taken from the counter (the next
    // group's number is fetched while this one is worked on); each group's
    // rows are reduced the same way whichever warp takes them, and the
    // with-cost pass, whose per-warp sums must not depend on the order,
    // stays round-robin
    const bool dyn = PRUNE && !WC && pv.next_group != nullptr;
    int r0 = gwarp * RW;
    if (dyn) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(pv.next_group, 1u);
        r0 = (int)__shfl_sync(0xffffffffu, g0, 0) * RW;
    }
    while (r0 < nr) {
        unsigned gnext = 0;
        if (dyn && lane == 0) gnext = atomicAdd(pv.next_group, 1u);
        float p[RW][DMAX];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            const int rr = min(r0 + q, nr - 1);
#pragma unroll
            for (int k = 0; k < DMAX; ++k) p[q][k] = (k < d) ? pv.P[(int64_t)rr * d + k] : 0.0f;
        }
        Lse2 acc[RW], cacc[RW];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            acc[q] = {-INFINITY, 0.0f, 0.0f};
            cacc[q] = {0.0f, 0.0f, 0.0f};
        }
        if (PRUNE && pv.hint) {
            const int hv = pv.hint[r0 / RW];
            if (hv >= 0 && hv < nfull) {
                float R0[RW];
                hinted_start<DMAX, RW>(pv, p, d, hv, R0);
#pragma unroll
                for (int q = 0; q < RW; ++q) acc[q].R = R0[q];
            }
        }
        // whole chunks: every element valid; chunk(v) works on slot v
        auto chunk = [&](int v) {
            const float4 ah = __ldg(Ah4 + v);
            float4 qh[PRE ? DMAX : 1], ql[PRE ? DMAX : 1];
            if (PRE) {
#pragma unroll
                for (int k = 0; k < DMAX; ++k)
                    if (k < d) qh[k] = __ldg(reinterpret_cast<const float4 *>(pv.Qh + k * ldq) + v);
            }
            if (PRUNE && !pv.qbox) {
                // the slot test (when no block records: the block test
                // already passed over the far blocks, and repeating it per
                // slot cost 6% of the colour solve)
                float amax = fmaxf(fmaxf(fabsf(ah.x), fabsf(ah.y)), fmaxf(fabsf(ah.z), fabsf(ah.w)));
                float qmax[DMAX];
#pragma unroll
                for (int k = 0; k < DMAX; ++k)
                    qmax[k] = (k < d) ? fmaxf(fmaxf(fabsf(qh[k].x), fabsf(qh[k].y)),
                                              fmaxf(fabsf(qh[k].z), fabsf(qh[k].w)))
                                      : 0.0f;
                bool far = true;
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                    float mag = amax;
#pragma unroll
                    for (int k = 0; k < DMAX; ++k)
                        if (k < d) mag = fmaf(fabsf(p[q][k]), qmax[k], mag);
                    const float lim = acc[q].R - pv.skip - 1.0f - mag * 0x1p-20f;
                    float e4[4] = {ah.x, ah.y, ah.z, ah.w};
#pragma unroll
                    for (int k = 0; k < DMAX; ++k) {
                        if (k < d) {
                            e4[0] = fmaf(p[q][k], qh[k].x, e4[0]);
                            e4[1] = fmaf(p[q][k], qh[k].y, e4[1]);
                            e4[2] = fmaf(p[q][k], qh[k].z, e4[2]);
                            e4[3] = fmaf(p[q][k], qh[k].w, e4[3]);
                        }
                    }
                    far = far && fmaxf(fmaxf(e4[0], e4[1]), fmaxf(e4[2], e4[3])) < lim;
                }
                if (__all_sync(0xffffffffu, far)) return;
            }
            float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!f32) {
                al = __ldg(Al4 + v);
                if (PRE) {
#pragma unroll
                    for (int k = 0; k < DMAX; ++k)
                        if (k < d) ql[k] = __ldg(reinterpret_cast<const float4 *>(pv.Ql + k * ldq) + v);
                }
            }
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                float h[4], l[4], cst[4];
                slot_dot<DMAX, PRE>(p[q], d, ah, al, qh, ql, pv.Qh, pv.Ql, ldq, v, h, l, f32);
                if (WC) slot_cost<DMAX>(p[q], d, pv.kind, cs_scale, pv.Pc, 4 * v, nc, cst);
                slot_accumulate<WC>(acc[q], cacc[q], h, l, cst);
            }
        };
        if (PRUNE && pv.qbox) {
            constexpr int S = kBoxSlots, G = 32 / S;   // slots per block, blocks per warp pass
            const int nb = nfull / S;
            // squared Euclidean: the bound through the box's distance to the rows
            const float cq = pv.kind == 1 ? box_cq(st, pv) : 1.0f;
            const bool geo = pv.kind == 1 && cq > 0.0f && cq < FLT_MAX;
            for (int b0 = 0; b0 < nb; b0 += 32) {
                bool near = false;
                const int b = b0 + lane;
                // the warp's running maxima: lower bounds of the rows' largest terms
                float Rw[RW];
#pragma unroll
                for (int q = 0; q < RW; ++q) Rw[q] = warp_max(acc[q].R);
                if (b < nb) {
                    const float2 ab = pv.abox[b];
                    const float4 qlo = pv.qbox[2 * b], qhi = pv.qbox[2 * b + 1];
                    const float qmn[4] = {qlo.x, qlo.y, qlo.z, qlo.w};
                    const float qmx[4] = {qhi.x, qhi.y, qhi.z, qhi.w};
#pragma unroll
                    for (int q = 0; q < RW; ++q) {
                        float ub, mag;
                        if (geo) {
                            // max g - |Q - z|^2 / c over the box + |z|^2 / c, z = (c / 2) p;
                            // the margin covers ~20 roundings of terms below mag
                            float zz = 0.f, dd = 0.f, qq = 0.f;
#pragma unroll
                            for (int k = 0; k < DMAX; ++k) {
                                if (k < d) {
                                    const float z = 0.5f * cq * p[q][k];
                                    const float dq = fmaxf(0.0f, fmaxf(qmn[k] - z, z - qmx[k]));
                                    const float qa = fmaxf(fabsf(qmn[k]), fabsf(qmx[k]));
                                    zz = fmaf(z, z, zz);
                                    dd = fmaf(dq, dq, dd);
                                    qq = fmaf(qa, qa, qq);
                                }
                            }
                            ub = ab.x + (zz - dd) / cq;
                            mag = ab.y + 2.0f * (zz + qq) / cq;
                            mag *= 0x1p-18f;
                        } else {
                            ub = ab.x;
                            mag = ab.y;
#pragma unroll
                            for (int k = 0; k < DMAX; ++k) {
                                if (k < d) {
                                    ub += fmaxf(p[q][k] * qmn[k], p[q][k] * qmx[k]);
                                    mag = fmaf(fabsf(p[q][k]), fmaxf(fabsf(qmn[k]), fabsf(qmx[k])), mag);
                                }
                            }
                            mag *= 0x1p-20f;
                        }
                        near = near || !(ub < Rw[q] - pv.skip - 1.0f - mag);
                    }
                }
                // the near blocks, G at a time: lane group lane / S takes the
                // (lane / S)-th remaining one, a slot of it per lane
                unsigned mask = __ballot_sync(0xffffffffu, near);
                while (mask) {
                    unsigned mine = mask;
                    for (int i = 0; i < lane / S; ++i) mine &= mine - 1;
#pragma unroll
                    for (int i = 0; i < G; ++i) mask &= mask - 1;
                    if (mine) chunk(S * (b0 + __ffs(mine) - 1) + (lane % S));
                }
            }
        } else {
            for (int v = lane; v < nfull; v += 32) chunk(v);
        }
        // ragged tail: at most one slot per lane, masked per element
        for (int v = nfull + lane; v < nc4; v += 32) {
            const float4 ah = __ldg(Ah4 + v), al = __ldg(Al4 + v);
            float4 qh[PRE ? DMAX : 1], ql[PRE ? DMAX : 1];
            if (PRE) {
#pragma unroll
                for (int k = 0; k < DMAX; ++k) {
                    if (k < d) {
                        qh[k] = __ldg(reinterpret_cast<const float4 *>(pv.Qh + k * ldq) + v);
                        ql[k] = __ldg(reinterpret_cast<const float4 *>(pv.Ql + k * ldq) + v);
                    }
                }
            }
            const int c0 = 4 * v;
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                float h[4], l[4], cst[4];
                slot_dot<DMAX, PRE>(p[q], d, ah, al, qh, ql, pv.Qh, pv.Ql, ldq, v, h, l, f32);
                if (WC) slot_cost<DMAX>(p[q], d, pv.kind, cs_scale, pv.Pc, c0, nc, cst);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (c0 + e >= nc) { h[e] = -INFINITY; l[e] = 0.0f; }
                }
                slot_accumulate<WC>(acc[q], cacc[q], h, l, cst);
            }
        }
        // per row: lane merge (double-float tree), FP64 finish by lane 0
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            const int r = r0 + q;
            const float Rrow = warp_max(acc[q].R);
            const float sc = ex2_approx(acc[q].R - Rrow);
            float hi, lo, chi = 0.f, clo = 0.f;
            two_sum_f(__fmul_rn(acc[q].S, sc), -__fmul_rn(acc[q].K, sc), hi, lo);
            if (WC) two_sum_f(__fmul_rn(cacc[q].S, sc), -__fmul_rn(cacc[q].K, sc), chi, clo);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
                const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
                float s2, e2;
                two_sum_f(hi, ohi, s2, e2);
                lo = lo + olo + e2;
                two_sum_f(s2, lo, hi, lo);
                if (WC) {
                    const float ochi = __shfl_xor_sync(0xffffffffu, chi, o);
                    const float oclo = __shfl_xor_sync(0xffffffffu, clo, o);
                    two_sum_f(chi, ochi, s2, e2);
                    clo = clo + oclo + e2;
                    two_sum_f(s2, clo, chi, clo);
                }
            }
            if (lane == 0 && r < nr) {
                const double S = (double)hi + (double)lo;
                const double l2 = (double)Rrow * kLn2 + log(S);
                if (MODE == 1) {
                    w.ell[r] = l2 - (pv.B64[r] + st->shift_f) * st->inv_eps_c;
                } else {
                    const double bx = pv.B64[r];
                    const double lse = l2 - (bx + st->shift_g) * st->inv_eps_c;
                    const double ui = w.loga[r] - lse;
                    w.u[r] = ui;
                    // column-pass operand A'_r = k (F_r - Bx_r), F = eps u + shift_f
                    const double A2 = st->k2 * (st->eps_c * ui + st->shift_f - bx);
                    const float A2h = (float)A2;
                    w.Fh[r] = A2h;
                    w.Fk[r] = (float)(A2 - (double)A2h);
                    my_dual += w.a[r] * ui;
                    if (WC) {
                        // row mass: a_r after the row pass, or f_r / eps + LSE_r
                        // under given potentials f
                        const double wr =
                            w.f_given ? exp(w.f_given[r] / st->eps_user + lse) : w.a[r];
                        my_cost += wr * (((double)chi + (double)clo) / S);
                    }
                }
            }
        }
        if (dyn) r0 = (int)__shfl_sync(0xffffffffu, gnext, 0) * RW;
        else r0 += nwarps * RW;
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

// Rows per warp for a dimension bound: enough registers for RW rows of
// points plus one slot of column operands.
template <int DMAX>
constexpr int rows_per_warp() { return DMAX <= 8 ? 4 : (DMAX <= 16 ? 2 : 1); }

// abox[b] = (max, max |.|) over block b (kBoxSlots slots, a lane per slot) of
// the high parts of A, or for squared-Euclidean costs of g_j = A_j +
// |Q_j|^2 / c and |A_j| + |Q_j|^2 / c: with z = (c / 2) p the exponent of a
// row p is A_j + p.Q_j = g_j - |Q_j - z|^2 / c + |z|^2 / c for any c > 0, so
// max g less the box's distance term bounds the block (k G_j less the
// squared distance, when c = 4 k s). The A of a pass is written by the step
// kernel (row pass) or by the row pass (column pass), so this runs before
// every pass.
__global__ void __launch_bounds__(kPtNT) k_points_abox(PointView pv, const DevState *st, int nb)
{
    if (pv.next_group && blockIdx.x == 0 && threadIdx.x == 0) *pv.next_group = 0u;
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * kPtNT + threadIdx.x) >> 5, nw = (gridDim.x * kPtNT) >> 5;
    const float cq = pv.kind == 1 ? box_cq(st, pv) : 1.0f;
    const bool geo = pv.kind == 1 && cq > 0.0f && cq < FLT_MAX;
    constexpr int S = kBoxSlots;
    for (int b0 = wg * (32 / S); b0 < nb; b0 += nw * (32 / S)) {
        const int b = b0 + lane / S;
        const int v = S * b + lane % S;
        const bool have = b < nb;
        const float4 a = have ? __ldg(reinterpret_cast<const float4 *>(pv.Ah) + v)
                              : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        float g[4] = {a.x, a.y, a.z, a.w};
        float m4[4] = {fabsf(a.x), fabsf(a.y), fabsf(a.z), fabsf(a.w)};
        if (geo) {
            float qq[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < pv.d && k < 4 && have; ++k) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(pv.Qh + k * pv.ldq) + v);
                qq[0] = fmaf(q.x, q.x, qq[0]); qq[1] = fmaf(q.y, q.y, qq[1]);
                qq[2] = fmaf(q.z, q.z, qq[2]); qq[3] = fmaf(q.w, q.w, qq[3]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float t = qq[e] / cq;
                g[e] += t;
                m4[e] += t;
            }
        }
        float mx = fmaxf(fmaxf(g[0], g[1]), fmaxf(g[2], g[3]));
        float mg = have ? fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3])) : 0.0f;
#pragma unroll
        for (int o = S / 2; o > 0; o >>= 1) {
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            mg = fmaxf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
        }
        if (have && lane % S == 0) pv.abox[b] = make_float2(mx, mg);
    }
}

// qbox[2 b] / qbox[2 b + 1] = per-coordinate minimum / maximum of block b's
// Q (coordinates k >= d are 0), a lane per slot.
__global__ void __launch_bounds__(kPtNT) k_points_qbox(const float *Qh, int64_t ldq, int nb,
                                                       int d, float4 *qbox)
{
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * kPtNT + threadIdx.x) >> 5, nw = (gridDim.x * kPtNT) >> 5;
    constexpr int S = kBoxSlots;
    for (int b0 = wg * (32 / S); b0 < nb; b0 += nw * (32 / S)) {
        const int b = b0 + lane / S;
        const bool have = b < nb;
        float mn[4] = {0.f, 0.f, 0.f, 0.f}, mx[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < d && k < 4; ++k) {
            float lo = INFINITY, hi = -INFINITY;
            if (have) {
                const float4 q =
                    __ldg(reinterpret_cast<const float4 *>(Qh + k * ldq) + S * b + lane % S);
                lo = fminf(fminf(q.x, q.y), fminf(q.z, q.w));
                hi = fmaxf(fmaxf(q.x, q.y), fmaxf(q.z, q.w));
            }
#pragma unroll
            for (int o = S / 2; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            mn[k] = lo;
            mx[k] = hi;
        }
        if (have && lane % S == 0) {
            qbox[2 * b] = make_float4(mn[0], mn[1], mn[2], mn[3]);
            qbox[2 * b + 1] = make_float4(mx[0], mx[1], mx[2], mx[3]);
        }
    }
}

cudaError_t launch_points_qbox(const float *Qh, int64_t ldq, int nc, int d, float4 *qbox,
                               cudaStream_t s)
{
    const int nb = points_blocks(nc);
    if (nb <= 0) return cudaSuccess;
    const int per_cta = (kPtNT / 32) * (32 / kBoxSlots);
    k_points_qbox<<<(nb + per_cta - 1) / per_cta, kPtNT, 0, s>>>(Qh, ldq, nb, d, qbox);
    return cudaGetLastError();
}

template <int MODE, bool WC>
static cudaError_t launch_pts(const PointView &pv, const Work &w, int grid, cudaStream_t s)
{
    if (pv.prune && pv.d <= 4 && pv.qbox) {
        // block records and the row-group counter, before every pruned pass
        const int nb = points_blocks(pv.nc);
        const int per_cta = (kPtNT / 32) * (32 / kBoxSlots);
        k_points_abox<<<std::max(1, (nb + per_cta - 1) / per_cta), kPtNT, 0, s>>>(pv, w.st, nb);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (pv.prune && pv.d <= 4 && pv.fp32) {
        // sorted point clouds, FP32 arguments (precision FP32)
        if (pv.d == 2) k_lse_points<MODE, 2, rows_per_warp<2>(), WC, true, true, true><<<grid, kPtNT, 0, s>>>(pv, w);
        else if (pv.d == 3) k_lse_points<MODE, 3, rows_per_warp<3>(), WC, true, true, true><<<grid, kPtNT, 0, s>>>(pv, w);
        else if (pv.d == 4) k_lse_points<MODE, 4, rows_per_warp<4>(), WC, true, true, true><<<grid, kPtNT, 0, s>>>(pv, w);
        else k_lse_points<MODE, 4, rows_per_warp<4>(), WC, false, true, true><<<grid, kPtNT, 0, s>>>(pv, w);
        return cudaGetLastError();
    }
    if (pv.prune && pv.d <= 4) {
        // sorted point clouds (see the set-up): the pruned kernels
        if (pv.d == 2) k_lse_points<MODE, 2, rows_per_warp<2>(), WC, true, true><<<grid, kPtNT, 0, s>>>(pv, w);
        else if (pv.d == 3) k_lse_points<MODE, 3, rows_per_warp<3>(), WC, true, true><<<grid, kPtNT, 0, s>>>(pv, w);
        else if (pv.d == 4) k_lse_points<MODE, 4, rows_per_warp<4>(), WC, true, true><<<grid, kPtNT, 0, s>>>(pv, w);
        else k_lse_points<MODE, 4, rows_per_warp<4>(), WC, false, true><<<grid, kPtNT, 0, s>>>(pv, w);
        return cudaGetLastError();
    }
    if (pv.d == 2) k_lse_points<MODE, 2, rows_per_warp<2>(), WC, true><<<grid, kPtNT, 0, s>>>(pv, w);
    else if (pv.d == 3) k_lse_points<MODE, 3, rows_per_warp<3>(), WC, true><<<grid, kPtNT, 0, s>>>(pv, w);
    else if (pv.d == 4) k_lse_points<MODE, 4, rows_per_warp<4>(), WC, true><<<grid, kPtNT, 0, s>>>(pv, w);
    else if (pv.d < 4) k_lse_points<MODE, 4, rows_per_warp<4>(), WC><<<grid, kPtNT, 0, s>>>(pv, w);
    else if (pv.d <= 8) k_lse_points<MODE, 8, rows_per_warp<8>(), WC><<<grid, kPtNT, 0, s>>>(pv, w);
    else if (pv.d <= 16) k_lse_points<MODE, 16, rows_per_warp<16>(), WC><<<grid, kPtNT, 0, s>>>(pv, w);
    else k_lse_points<MODE, 64, rows_per_warp<64>(), WC><<<grid, kPtNT, 0, s>>>(pv, w);
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lse_points<0, 4, 4, false>, kPtNT, 0);
    return b > 0 ? b : 1;
}

int occupancy_points_pruned(int d)
{
    int b = 0;
    if (d == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lse_points<0, 2, 4, false, true, true>, kPtNT, 0);
    else if (d == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lse_points<0, 3, 4, false, true, true>, kPtNT, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lse_points<0, 4, 4, false, true, true>, kPtNT, 0);
    return b > 0 ? b : 1;
}

int points_rows_per_warp(int d)
{
    return d <= 8 ? rows_per_warp<4>() : (d <= 16 ? rows_per_warp<16>() : rows_per_warp<64>());
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
                        two_sum_f(x[k], -y, dh, de);          // exact difference
                        term = __fmul_rn(dh, dh);            // (dh + de)^2 to double-float
                        te = fmaf(dh, dh, -term) + 2.0f * dh * de;
                    } else {
                        term = __fmul_rn(x[k], y);
                        te = fmaf(x[k], y, -term);
                    }
                    float s2, e2;
                    two_sum_f(h, term, s2, e2);
                    l += e2 + te;
                    h = s2;
                }
            }
            if (kind != 1) {   // cosine: 1 - <x, y>
                float s2, e2;
                two_sum_f(1.0f, -h, s2, e2);
                h = s2;
                l = e2 - l;
            }
            two_sum_f(h, l, h, l);
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

// Bx, By in FP64 and as pairs; Q (scaled Y) and Q' (scaled X), both times
// k = log2(e) / eps, in SoA pairs;
// per-block maxima for the shift bound and a count of non-finite coordinates. `scal` = {max C, s}.
__global__ void k_points_setup(const float *X, const float *Y, int n, int m, int d, int kind,
                               const double *scal, double eps, Work w, double *blockmax)
{
    const double s = scal[1];
    const double qs = (kind == 1) ? 2.0 * s : s;
    const double kq = (kLog2e / eps) * qs;   // Q in log2 units
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
            const double q = kq * xv;
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
            const double q = kq * yv;
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
                                int scale_max, double eps, const Work &w, double *scal,
                                double *blockmax, int nblk, cudaStream_t s)
{
    k_points_scale<<<1, 256, 0, s>>>(w.rowmax, n, scale_max, scal);
    k_points_setup<<<nblk, 256, 0, s>>>(X, Y, n, m, d, kind, scal, eps, w, blockmax);
    k_points_stats<<<1, 32, 0, s>>>(blockmax, nblk, d, kind, scal, w.statpart);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Spatial sort of a point cloud (set-up of a solve). The pruned passes skip
// a block of columns only when all of its columns are far from all of a
// warp's rows, which happens for most blocks once nearby points are adjacent: the
// clouds are put in Hilbert-curve order of their first min(d, 3) coordinates
// over the bounding box (10 bits per coordinate). A Hilbert curve has no
// long jumps between consecutive cells, so fewer slots straddle near and far
// points than with Morton order (about 4 points more of skipped slots on the
// colour workload). The order only changes which terms share a slot and the
// summation order; the solve is the same problem.
// ------------------------------------------------------------------------

namespace {

__device__ __forceinline__ uint32_t ord_f(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u >> 31) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float unord_f(uint32_t e)
{
    return __uint_as_float((e >> 31) ? (e & 0x7fffffffu) : ~e);
}

// box[0..2] = ordered min, box[3..5] = ordered max per coordinate
__global__ void k_bbox(const float *P, int n, int d, uint32_t *box)
{
    const int dd = d < 3 ? d : 3;
    uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int k = 0; k < dd; ++k) {
            const uint32_t e = ord_f(P[(int64_t)i * d + k]);
            mn[k] = min(mn[k], e);
            mx[k] = max(mx[k], e);
        }
    }
    for (int k = 0; k < dd; ++k) {
        const uint32_t a = __reduce_min_sync(0xffffffffu, mn[k]);
        const uint32_t b = __reduce_max_sync(0xffffffffu, mx[k]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(box + k, a);
            atomicMax(box + 3 + k, b);
        }
    }
}

// Index along the Hilbert curve of the cell q[0..nd-1] (10 bits each,
// nd <= 3), by Skilling's transform of the axes to the curve's transposed
// index (J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707,
// 2004): undo the rotations and reflections level by level, Gray-encode,
// then interleave the transposed bits, highest level first.
__device__ __forceinline__ uint32_t hilbert_index(uint32_t q[3], int nd)
{
    constexpr uint32_t M = 1u << 9;
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < nd; ++i) {
            if (q[i] & Q) {
                q[0] ^= P;
            } else {
                const uint32_t t = (q[0] ^ q[i]) & P;
                q[0] ^= t;
                q[i] ^= t;
            }
        }
    }
    for (int i = 1; i < nd; ++i) q[i] ^= q[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (q[nd - 1] & Q) t ^= Q - 1;
    for (int i = 0; i < nd; ++i) q[i] ^= t;
    uint32_t h = 0;
    for (int b = 9; b >= 0; --b)
        for (int i = 0; i < nd; ++i) h = (h << 1) | ((q[i] >> b) & 1u);
    return h;
}

__global__ void k_curve_keys(const float *P, int n, int d, const uint32_t *box, uint32_t *code,
                         int *idx)
{
    const int dd = d < 3 ? d : 3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t q[3] = {0u, 0u, 0u};
        for (int k = 0; k < dd; ++k) {
            const float lo = unord_f(box[k]), hi = unord_f(box[3 + k]);
            const float t = hi > lo ? (P[(int64_t)i * d + k] - lo) / (hi - lo) : 0.0f;
            q[k] = (uint32_t)min(1023, max(0, __float2int_rz(t * 1024.0f)));
        }
        code[i] = hilbert_index(q, dd);
        idx[i] = i;
    }
}

__global__ void k_gather_points(const float *P, const double *a, int n, int d, const int *perm,
                                float *P_out, double *a_out)
{
    const int64_t total = (int64_t)n * d;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / d, k = t - i * d;
        P_out[t] = P[(int64_t)perm[i] * d + k];
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        a_out[i] = a[perm[i]];
}

__global__ void k_scatter_scaled(const double *src, double scale, const int *perm, int n,
                                 double *dst)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[perm[i]] = scale * src[i];
}

}  // namespace

size_t points_sort_temp_bytes(int count)
{
    size_t t = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, t, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                    (const int *)nullptr, (int *)nullptr, count, 0, 30);
    return t;
}

// Slot hints of the pruned passes (d <= 4, sorted clouds): for each group of
// four rows of P (nr x d), the float4 slot of Q (nc x d) holding the column of
// smallest cost to the group's first row (squared distance, or 1 - <p, q>),
// by brute force with one warp per group and ties to the lower column; -1 when
// that slot lies in the ragged tail (the passes never skip tail slots).
template <int DMAX>
__global__ void __launch_bounds__(kPtNT) k_points_hint(const float *P, int nr, const float *Q,
                                                       int nc, int d, int kind, int32_t *hint)
{
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * kPtNT + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kPtNT) >> 5;
    const int groups = (nr + 3) / 4;
    const int nfull = (nc >> 2) & ~31;
    for (int g = gwarp; g < groups; g += nwarps) {
        float p[DMAX];
#pragma unroll
        for (int k = 0; k < DMAX; ++k) p[k] = (k < d) ? P[(int64_t)(4 * g) * d + k] : 0.0f;
        float best = INFINITY;
        int bj = 0x7fffffff;
        for (int j = lane; j < nc; j += 32) {
            float c = 0.0f;
#pragma unroll
            for (int k = 0; k < DMAX; ++k) {
                if (k < d) {
                    const float q = Q[(int64_t)j * d + k];
                    if (kind == 1) { const float t = p[k] - q; c = fmaf(t, t, c); }
                    else c = fmaf(-p[k], q, c);
                }
            }
            if (c < best) { best = c; bj = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; }
        }
        if (lane == 0) hint[g] = (bj != 0x7fffffff && bj / 4 < nfull) ? bj / 4 : -1;
    }
}

cudaError_t launch_points_hint(const float *P, int nr, const float *Q, int nc, int d, int kind,
                               int32_t *hint, int grid, cudaStream_t s)
{
    if (d == 2) k_points_hint<2><<<grid, kPtNT, 0, s>>>(P, nr, Q, nc, d, kind, hint);
    else if (d == 3) k_points_hint<3><<<grid, kPtNT, 0, s>>>(P, nr, Q, nc, d, kind, hint);
    else k_points_hint<4><<<grid, kPtNT, 0, s>>>(P, nr, Q, nc, d, kind, hint);
    return cudaGetLastError();
}

cudaError_t launch_points_sort(const float *P, const double *a, int n, int d, const PointSort &ps,
                               cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(ps.box, 0xff, 3 * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ps.box + 3, 0, 3 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(1024, (n + 255) / 256));
    k_bbox<<<grid, 256, 0, s>>>(P, n, d, ps.box);
    k_curve_keys<<<grid, 256, 0, s>>>(P, n, d, ps.box, ps.code, ps.idx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t t = ps.temp_bytes;
    e = cub::DeviceRadixSort::SortPairs(ps.temp, t, ps.code, ps.code2, ps.idx, ps.perm, n, 0, 30,
                                        s);
    if (e != cudaSuccess) return e;
    k_gather_points<<<grid, 256, 0, s>>>(P, a, n, d, ps.perm, ps.P, ps.a);
    return cudaGetLastError();
}

cudaError_t launch_scatter_scaled(const double *src, double scale, const int *perm, int n,
                                  double *dst, cudaStream_t s)
{
    k_scatter_scaled<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, s>>>(src, scale, perm,
                                                                                 n, dst);
    return cudaGetLastError();
}

}  // namespace accsink

// Cosine costs of the batched solver on the 5th-generation tensor cores.
//
// For word-vector-sized d the cost C_ij = 1 - <x_i, y_j> is a dense
// contraction, so it runs as tcgen05 MMAs (operands staged by TMA, FP32
// accumulators in TMEM) instead of the exact CUDA-core expansion of
// k_batch_form. The cost must stay accurate far beyond FP32 (the solver
// reads it as a double-float pair), and the tensor cores can deliver that
// exactly: a product of two FP16 integers is exact, and an FP32 accumulator
// holding integer-valued sums below 2^24 never rounds, whatever order the
// hardware adds in. Each vector is therefore split into integer slices (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of
// matrix multiplication", Numer. Algorithms 59, 2012):
//
//   x_k = 2^e sum_{l < L} q_{l,k} 2^{-beta (l+1)} + r_k,   |r_k| <= 2^{e - beta L - 1},
//
// with 2^{e-1} <= max_k |x_k| < 2^e, rounding to nearest at each level, so
// q_0 lies in [-2^beta, 2^beta] and q_l (l >= 1) in [-2^{beta-1}, 2^{beta-1}].
// Slice pairs (i, j) with the same class c = i + j share the scale
// 2^{-beta (c + 2)}, so one TMEM accumulator per class sums them:
//
//   <x, y> ~= 2^{ex + ey - 2 beta} sum_{c < L} 2^{-beta c} sum_{i + j = c} sum_k q_{i,k} q'_{j,k}.
//
// A class sum is an integer of magnitude at most d 2^14 for c = 0 and
// d (2 * 2^beta 2^{beta-1} + (c - 1) 2^{2 beta - 2}) = d (c + 3) 2^12 for
// c >= 1, so at most d 2^15 for c <= 5 (beta = 7): below 2^24 for d <= 480,
// and every partial sum the tensor cores form (of any subset of the terms)
// is an integer below 2^24 too, so they return each class exactly.
// The classes left out (i + j >= L) and the residuals r bound the error of
// the dot product by d 2^{-39} |x| |y| (2^{-30.8} for d = 300) in the worst
// case; with slices of random sign the terms largely cancel (about
// sqrt(d) 2^{-42}). The epilogue adds the six exact classes in double-float,
// forms 1 - <x, y> and k C as (hi, lo) pairs like the CUDA-core path, and
// folds in the cost statistics.
//
// A persistent CTA per SM forms 128 x 64 tiles (128 rows of X on the TMEM
// lanes, 64 rows of Y on the accumulator columns) in turn. Warp 0 issues TMA
// loads of all six slices of both operands, 32 contraction elements at a
// time, into a three-stage ring that runs across tiles; warp 1 owns the TMEM
// allocation and issues the 21 slice-pair MMAs per stage (two K = 16 steps
// each); warps 2-9 read the accumulators back (two warps per TMEM lane
// quadrant, 32 columns each), release them to the next tile's MMAs as soon
// as they are read, and then write the costs. Every wait is bounded: a wait
// that runs out marks the problem (nonfinite bit 2), and the CTA stops,
// drains its copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <float.h>
#include <stdint.h>

#include "accsink_internal.cuh"
#include "batch_internal.cuh"

namespace accsink {

namespace {

constexpr int kTcM = kBatchTcRows;        // X rows per tile (TMEM lanes)
constexpr int kTcN = kBatchTcCols;        // Y rows per tile (accumulator columns)
constexpr int kTcK = kBatchTcK;           // contraction elements per stage: 64-byte rows
constexpr int kTcL = kBatchTcLevels;      // slices per vector
constexpr int kTcBeta = 7;                // bits per slice
constexpr int kTcStages = 3;
constexpr int kTcEpiWarps = 8;            // two per TMEM lane quadrant
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;   // TMA warp, MMA warp, epilogue warps
constexpr uint32_t kTcSliceA = kTcM * kTcK * 2;           // one slice of the X tile, bytes
constexpr uint32_t kTcSliceB = kTcN * kTcK * 2;           // one slice of the Y tile
constexpr uint32_t kTcABytes = kTcL * kTcSliceA;
constexpr uint32_t kTcBBytes = kTcL * kTcSliceB;
constexpr uint32_t kTcStageBytes = kTcABytes + kTcBBytes;
constexpr uint32_t kTcSmemBytes = kTcStages * kTcStageBytes + 1024;   // + alignment slack
constexpr uint32_t kTcTmemCols = 512;     // six 64-column accumulators, rounded to a power of two
constexpr uint64_t kTcWaitNs = 2000000000ull;

static_assert(kTcL * kTcN <= (int)kTcTmemCols, "accumulators exceed the TMEM allocation");
static_assert(kTcStageBytes % 1024 == 0, "stages must keep the 1024-byte alignment");
static_assert(kTcK * 2 == 64, "the 64-byte swizzle needs 64-byte operand rows");

// ------------------------------------------------------------ PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity to complete; false after the limit.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_test(bar, parity))
        if (globaltimer_ns() - t0 > kTcWaitNs) return false;
    return true;
}

// TMA: a 3-D box (contraction, rows, slices) of the slice tensor into shared
// memory, completion counted in bytes on the stage's barrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] B[smem]^T, both K-major FP16, FP32 accumulate.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives on the barrier once every MMA this thread issued so far completed.
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Orders the uses of loaded registers after tcgen05.wait::ld.
__device__ __forceinline__ void tie16(float (&v)[16])
{
    asm volatile(""
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]),
                   "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]),
                   "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]));
}

// Shared-memory matrix descriptor of one K-major operand slice stored with
// the 64-byte swizzle (64-byte rows, 8-row groups 512 bytes apart): start
// address >> 4, leading offset (unused for swizzled K-major operands),
// stride offset 512 >> 4, descriptor version 1, swizzle mode 4 (64 B).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// FP16 A and B (format 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kTcIdesc =
    (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

// 2^k for -126 <= k <= 127.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// ------------------------------------------------------------- slicing --

// One warp per vector (a row of X or Y of a tensor-core problem): its
// exponent e and its six slices, zero-padded to dpad contraction elements.
// tcs is the exclusive prefix of n + m over the problems listed in tcp.
__global__ void __launch_bounds__(256) k_batch_slice(BatchProb *Pall, const int32_t *tcp,
                                                     const int64_t *tcs, int ntc, int dpad,
                                                     int64_t R, __half *SL, int32_t *expo)
{
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= R) return;
    int lo = 0, hi = ntc - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tcs[mid] <= row) lo = mid;
        else hi = mid - 1;
    }
    BatchProb *P = Pall + tcp[lo];
    const int li = (int)(row - tcs[lo]);
    const int d = P->d;
    const float *src = li < P->n ? P->X + (int64_t)li * d : P->Y + (int64_t)(li - P->n) * d;
    float amax = 0.0f;
    bool bad = false;
    for (int k = lane; k < d; k += 32) {
        const float v = src[k];
        amax = fmaxf(amax, fabsf(v));
        bad = bad || !isfinite(v);
    }
    amax = warp_max(amax);
    bad = __any_sync(0xffffffffu, bad);
    if (bad && lane == 0) atomicOr(&P->nonfinite, 1u);
    // vectors below 2^-60 are treated as zero: their cosine terms are below
    // 2^-60 |y| and the exponent stays in range for the epilogue's scaling
    const bool zero = bad || !(amax >= 0x1p-60f);
    int e = 0;
    if (!zero) frexpf(amax, &e);
    if (lane == 0) expo[row] = e;
    for (int k0 = 8 * lane; k0 < dpad; k0 += 256) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u;
            t[u] = (!zero && k < d) ? ldexpf(src[k], -e) : 0.0f;
        }
#pragma unroll
        for (int l = 0; l < kTcL; ++l) {
            uint32_t hv[4];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                const float w0 = t[u] * (float)(1 << kTcBeta), w1 = t[u + 1] * (float)(1 << kTcBeta);
                const float q0 = rintf(w0), q1 = rintf(w1);
                t[u] = w0 - q0;          // exact: q0 is the integer nearest w0
                t[u + 1] = w1 - q1;
                const __half2 h2 = __floats2half2_rn(q0, q1);   // |q| <= 128: exact in FP16
                hv[u / 2] = *reinterpret_cast<const uint32_t *>(&h2);
            }
            *reinterpret_cast<uint4 *>(SL + ((int64_t)l * R + row) * dpad + k0) =
                make_uint4(hv[0], hv[1], hv[2], hv[3]);
        }
    }
}

// -------------------------------------------------------------- the tile --

// Lexicographic max / min of normalised double-float pairs (numeric order).
__device__ __forceinline__ void df_max(float &mh, float &ml, float h, float l)
{
    if (h > mh || (h == mh && l > ml)) { mh = h; ml = l; }
}

__device__ __forceinline__ void df_min(float &mh, float &ml, float h, float l)
{
    if (h < mh || (h == mh && l < ml)) { mh = h; ml = l; }
}

// Arrives once on the barrier (count 1 per arriving warp).
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The 21 slice-pair MMAs of one stage, two K = 16 steps each; the first
// MMA of each class overwrites its accumulator when `first` is set.
__device__ __forceinline__ void stage_mmas(uint32_t tmem, uint64_t dA, uint64_t dB, uint32_t first)
{
#pragma unroll
    for (int c = 0; c < kTcL; ++c) {
#pragma unroll
        for (int i = 0; i <= c; ++i) {
#pragma unroll
            for (int ks = 0; ks < kTcK / 16; ++ks) {
                // descriptor start fields advance by the byte offset >> 4
                const uint64_t a = dA + (uint64_t)((i * kTcSliceA + ks * 32) >> 4);
                const uint64_t b = dB + (uint64_t)(((c - i) * kTcSliceB + ks * 32) >> 4);
                tc_mma(tmem + c * kTcN, a, b, kTcIdesc, (i == 0 && ks == 0) ? !first : 1u);
            }
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_batch_form_tc(BatchProb *Pall, const BatchTile *tiles, int ntiles, const int32_t *expo,
                    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB)
{
    extern __shared__ uint8_t tc_smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kTcStages], empty_bar[kTcStages];
    __shared__ __align__(8) uint64_t accf_bar, acce_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_s;
    const uint32_t smem0 = (smem_u32(tc_smem_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&accf_bar), 1);
        mbar_init(smem_u32(&acce_bar), kTcEpiWarps);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: a ring of stages shared by all of this CTA's tiles
            uint32_t it = 0;
            for (int t = blockIdx.x; t < ntiles && !abort_s; t += gridDim.x) {
                const BatchTile tl = tiles[t];
                const BatchProb *P = Pall + tl.prob;
                const int nk = (P->d + kTcK - 1) / kTcK;
                const int xrow = P->tc_xoff + tl.row0, yrow = P->tc_yoff + tl.col0;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kTcStages;
                    if (it >= kTcStages &&
                        !mbar_wait(smem_u32(&empty_bar[s]), ((it / kTcStages) - 1) & 1)) {
                        atomicOr(&Pall[tl.prob].nonfinite, 2u);
                        abort_s = 1;
                        break;
                    }
                    const uint32_t sa = smem0 + s * kTcStageBytes;
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    mbar_expect_tx(fb, kTcStageBytes);
                    tma_load_3d(sa, &tmA, kc * kTcK, xrow, 0, fb);
                    tma_load_3d(sa + kTcABytes, &tmB, kc * kTcK, yrow, 0, fb);
                }
            }
            // drain: the last load of each stage has landed before the CTA exits
            for (uint32_t j = it > (uint32_t)kTcStages ? it - kTcStages : 0u; j < it; ++j)
                if (!mbar_wait(smem_u32(&full_bar[j % kTcStages]), (j / kTcStages) & 1)) abort_s = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issue: class c = i + j accumulates in columns [c N, c N + N)
            uint32_t it = 0;
            int lt = 0;
            for (int t = blockIdx.x; t < ntiles && !abort_s; t += gridDim.x, ++lt) {
                const BatchTile tl = tiles[t];
                const int nk = (Pall[tl.prob].d + kTcK - 1) / kTcK;
                // the epilogue has read the previous tile's accumulators
                if (lt > 0 && !mbar_wait(smem_u32(&acce_bar), (lt - 1) & 1)) {
                    atomicOr(&Pall[tl.prob].nonfinite, 2u);
                    abort_s = 1;
                    break;
                }
                tc_fence_after();
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kTcStages;
                    if (!mbar_wait(smem_u32(&full_bar[s]), (it / kTcStages) & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem0 + s * kTcStageBytes;
                    stage_mmas(tmem, sdesc_sw64(sa), sdesc_sw64(sa + kTcABytes), kc == 0);
                    tc_commit(smem_u32(&empty_bar[s]));
                }
                tc_commit(smem_u32(&accf_bar));
                if (!ok) {
                    atomicOr(&Pall[tl.prob].nonfinite, 2u);
                    abort_s = 1;
                    ++lt;            // this tile's commit is the last one to wait for
                    break;
                }
            }
            // every MMA issued has completed before the CTA frees its TMEM
            if (lt > 0 && !mbar_wait(smem_u32(&accf_bar), (lt - 1) & 1)) abort_s = 1;
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns
        // [32 h, 32 h + 32) with h = (w - 2) / 4
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const BatchTile tl = tiles[t];
            BatchProb *P = Pall + tl.prob;
            const int n = P->n, m = P->m;
            const int r = tl.row0 + 32 * quad + lane;
            const bool rv = r < n;
            int ok = 0;
            if (lane == 0) ok = (!abort_s && mbar_wait(smem_u32(&accf_bar), lt & 1)) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicOr(&P->nonfinite, 2u);
                    abort_s = 1;
                }
                break;
            }
            tc_fence_after();
            const int ex = rv ? expo[P->tc_xoff + r] : 0;
            const float sx = pow2f(ex - kTcBeta);
            const double kd = P->scale ? 1.0 : kLog2e / P->eps;
            const float kh = (float)kd, kl = (float)(kd - (double)kh);
            float mxh = -INFINITY, mxl = 0.0f, mnh = INFINITY, mnl = 0.0f;
            int bad = 0;
            const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16) + 32 * half;
            // read this warp's 32 columns, two classes at a time, adding the
            // exact classes into double-float sums (h, l), largest scale first
            float h[32], l[32];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int c0 = 0; c0 < kTcL; c0 += 2) {
                    float a0[16], a1[16];
                    tmem_ld16(trow + c0 * kTcN + 16 * j, a0);
                    tmem_ld16(trow + (c0 + 1) * kTcN + 16 * j, a1);
                    tmem_wait_ld();
                    tie16(a0);
                    tie16(a1);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        float s2, e2;
                        if (c0 == 0) {
                            h[16 * j + e] = a0[e];
                            l[16 * j + e] = 0.0f;
                        } else {
                            two_sum_f(h[16 * j + e], a0[e] * pow2f(-kTcBeta * c0), s2, e2);
                            h[16 * j + e] = s2;
                            l[16 * j + e] += e2;
                        }
                        two_sum_f(h[16 * j + e], a1[e] * pow2f(-kTcBeta * (c0 + 1)), s2, e2);
                        h[16 * j + e] = s2;
                        l[16 * j + e] += e2;
                    }
                }
            }
            // the accumulators are read: the MMA warp may start the next tile
            // while this warp writes the costs
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce_bar));
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int cb = tl.col0 + 32 * half + 16 * j;
                float oh[16], ol[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int col = cb + e;
                    const int ey = col < m ? expo[P->tc_yoff + col] : 0;
                    // <x, y> = 2^(ex + ey - 2 beta) (h + l): two exact power-of-two scalings
                    const float sy = pow2f(ey - kTcBeta);
                    const float dh = h[16 * j + e] * sx * sy;
                    const float dl = l[16 * j + e] * sx * sy;
                    // C = 1 - <x, y>
                    float ch, cl, tt;
                    two_sum_f(1.0f, -dh, ch, tt);
                    two_sum_f(ch, tt - dl, ch, cl);
                    if (rv && col < m) {
                        if (!isfinite(ch)) bad = 1;
                        df_max(mxh, mxl, ch, cl);
                        df_min(mnh, mnl, ch, cl);
                    }
                    // k C as (hi, lo): Dekker product with FMA
                    const float pp = __fmul_rn(kh, ch);
                    const float pe = fmaf(kh, cl, fmaf(kl, ch, fmaf(kh, ch, -pp)));
                    float vh, vl;
                    two_sum_f(pp, pe, vh, vl);
                    const bool keep = col < m;
                    oh[e] = keep ? vh : 0.0f;
                    ol[e] = keep ? vl : 0.0f;
                }
                if (rv) {
                    const int64_t base = (int64_t)r * P->ldm;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        const int c4 = cb + 4 * g;
                        if (c4 < P->ldm) {
                            *reinterpret_cast<float4 *>(P->Kh + base + c4) =
                                make_float4(oh[4 * g], oh[4 * g + 1], oh[4 * g + 2], oh[4 * g + 3]);
                            *reinterpret_cast<float4 *>(P->Kl + base + c4) =
                                make_float4(ol[4 * g], ol[4 * g + 1], ol[4 * g + 2], ol[4 * g + 3]);
                        }
                    }
                    if (P->KTh) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int col = cb + e;
                            if (col < m) {
                                P->KTh[(int64_t)col * P->ldn + r] = oh[e];
                                P->KTl[(int64_t)col * P->ldn + r] = ol[e];
                            }
                        }
                    }
                }
            }
            // cost statistics of the tile (FP64 encodings, one atomic per warp)
            double mx = mxh == -INFINITY ? -DBL_MAX : (double)mxh + (double)mxl;
            double mn = mnh == INFINITY ? DBL_MAX : (double)mnh + (double)mnl;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                bad |= __shfl_xor_sync(0xffffffffu, bad, o);
            }
            if (lane == 0) {
                if (mx != -DBL_MAX) {
                    atomicMax(&P->cmax_enc, enc_d(mx));
                    atomicMin(&P->cmin_enc, enc_d(mn));
                    atomicMax(&P->cabs_enc, enc_d(fmax(fabs(mx), fabs(mn))));
                }
                if (bad) atomicOr(&P->nonfinite, 1u);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // after a wait that ran out, every problem with a tile on this CTA is
    // marked (some of its costs may never have been written)
    if (abort_s && threadIdx.x == 0)
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
            atomicOr(&Pall[tiles[t].prob].nonfinite, 2u);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------- tensor maps --

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// The slice tensor [L][R][dpad] FP16, read in boxes of (32, rows, L) with the
// 64-byte swizzle; rows past R read as zeros.
bool encode_slices(CUtensorMap *map, const __half *SL, int64_t R, int dpad, int rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)dpad, (cuuint64_t)R, (cuuint64_t)kTcL};
    const cuuint64_t strides[2] = {(cuuint64_t)dpad * 2, (cuuint64_t)R * dpad * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kTcK, (cuuint32_t)rows, (cuuint32_t)kTcL};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half *>(SL), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool batch_tc_available() { return encode_fn() != nullptr; }

size_t batch_tc_slice_bytes(int64_t R, int dpad) { return (size_t)kTcL * R * dpad * 2; }

cudaError_t prepare_batch_form_tc(int *sms)
{
    // per batch: the attribute and the SM count belong to the current device
    cudaError_t e = cudaFuncSetAttribute(k_batch_form_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    return e;
}

cudaError_t launch_batch_form_tc(BatchProb *P, const BatchTcLaunch &t, cudaStream_t s)
{
    if (t.ntiles <= 0 || t.R <= 0) return cudaSuccess;
    if (t.dpad % kTcK != 0 || t.dpad > kBatchTcMaxD) return cudaErrorInvalidValue;
    __half *SL = static_cast<__half *>(t.SL);
    k_batch_slice<<<(unsigned)((t.R + 7) / 8), 256, 0, s>>>(P, t.tcp, t.tcs, t.ntc, t.dpad, t.R,
                                                            SL, t.expo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap mA, mB;
    if (!encode_slices(&mA, SL, t.R, t.dpad, kTcM) || !encode_slices(&mB, SL, t.R, t.dpad, kTcN))
        return cudaErrorNotSupported;
    // one persistent CTA per SM (its shared memory allows no second)
    k_batch_form_tc<<<std::min(t.ntiles, std::max(1, t.sms)), kTcThreads, kTcSmemBytes, s>>>(
        P, t.tiles, t.ntiles, t.expo, mA, mB);
    return cudaGetLastError();
}

}  // namespace accsink

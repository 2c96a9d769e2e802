// Row log-sum-exp pass, TMA-pipelined (the 128-bit-aligned path).
//
// One producer warp streams the cost through a ring of shared-memory stages
// with bulk asynchronous copies (cp.async.bulk, completion counted on an
// mbarrier per stage); eight consumer warps each own two rows of the current
// group of 16 rows and sweep the staged tiles. The column operand (G, gamma k)
// of every tile is staged once and shared by all 16 rows. Consumers never
// meet at a CTA barrier inside a group, so the copy engine keeps up to
// kStages tiles in flight while they compute.
//
// The arithmetic per element is the one of the plain row pass (exact
// Fast2Sum split, per-row running reference, double-float scale); every
// row's FP32 partials are merged within its warp in FP64.
//
// Every wait on an mbarrier is bounded by kWaitLimitNs of global time; on
// expiry the kernel records ACCSINK_ERR_TIMEOUT and stops the solve, and the
// producer still waits (bounded) for the copies it issued before exiting.
#include <cstdlib>

#include "accsink_internal.cuh"

namespace accsink {

namespace {

constexpr uint64_t kWaitLimitNs = 1000000000ull;

// Pipeline geometry: RW rows per consumer warp, NCW consumer warps (a group
// is RW * NCW rows), tiles of TW columns (TW / 128 float4 per lane), S stages.
template <int RW, int NCW, int TW, int S>
struct RowGeo {
    static constexpr int kRW = RW, kNCW = NCW, kTW = TW, kStages = S;
    static constexpr int kGR = RW * NCW;
    static constexpr int kNT = 32 * (NCW + 1);
    static constexpr int kSlots = TW / 128;
    struct Stage {
        float C[kGR][TW];
        float G[TW];
        float Gk[TW];
    };
    static constexpr size_t kSmemBytes = sizeof(Stage) * S + 2 * S * sizeof(uint64_t) + 128;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
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

// Bounded wait for the phase of `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, DevState *st)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
            atomicExch(&st->status, 6 /* ACCSINK_ERR_TIMEOUT */);
            atomicExch(&st->done, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

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

// 2^((s - R + e + gamma) k) for s = fl(G - c) already formed; e is the exact
// rounding error of s (Fast2Sum, |G| >= |c|).
__device__ __forceinline__ float term_s(float s, float G, float gk, float c, float R, float kh,
                                        float kl)
{
    const float z = s - G;
    const float e = -c - z;
    const float q = fmaf(e, kh, gk);
    const float t = s - R;
    return ex2_approx(fmaf(t, kh, fmaf(t, kl, q)));
}

}  // namespace

template <class GEO, bool WITH_COST>
__global__ void __launch_bounds__(GEO::kNT, 1) k_row_pass_tma(CostView cv, Work w)
{
    constexpr int kRW = GEO::kRW, kNCW = GEO::kNCW, kTW = GEO::kTW, kStages = GEO::kStages;
    constexpr int kGR = GEO::kGR, kSlots = GEO::kSlots;
    using Stage = typename GEO::Stage;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    DevState *st = w.st;
    if (!w.ignore_done && *(volatile int32_t *)&st->done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->barrier = 0u;   // for the step kernel

    Stage *stages = reinterpret_cast<Stage *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *full = reinterpret_cast<uint64_t *>(stages + kStages);
    uint64_t *empty = full + kStages;

    const int n = cv.n, m = cv.m;
    const int64_t ldc = cv.ldc;
    const int r0 = (int)((int64_t)blockIdx.x * n / gridDim.x);
    const int r1 = (int)((int64_t)(blockIdx.x + 1) * n / gridDim.x);
    const int ngroups = (r1 - r0 + kGR - 1) / kGR;
    const int ntiles_row = (m + kTW - 1) / kTW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Each CTA starts its sweep of a row at a different tile: with a row
    // pitch of a power of two, CTAs moving in lockstep would otherwise hit
    // the same address bits below the pitch at the same time.
    const int rot = (int)(blockIdx.x % (unsigned)ntiles_row);
    auto tile_col = [&](int ti) {
        int tt = ti + rot;
        if (tt >= ntiles_row) tt -= ntiles_row;
        return tt * kTW;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), kNCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kNCW) {
        // ------------------------------------------------------ producer
        if (lane == 0) {
            int t = 0;
            bool ok = true;
            for (int gi = 0; gi < ngroups && ok; ++gi) {
                const int g0 = r0 + gi * kGR;
                const int nrows = min(kGR, r1 - g0);
                for (int ti = 0; ti < ntiles_row; ++ti, ++t) {
                    const int s = t % kStages;
                    const uint32_t ph = (uint32_t)(t / kStages) & 1u;
                    if (!mbar_wait(smem_addr(&empty[s]), ph ^ 1u, st)) { ok = false; break; }
                    const int c0 = tile_col(ti);
                    const int wdt = min(kTW, m - c0);
                    const int w4 = wdt & ~3;
                    const int gw = (wdt + 3) & ~3;
                    const uint32_t bytes = (uint32_t)(nrows * w4 * 4 + 2 * gw * 4);
                    const uint32_t fb = smem_addr(&full[s]);
                    mbar_expect_tx(fb, bytes);
                    if (w4 > 0) {
                        for (int r = 0; r < nrows; ++r)
                            bulk_g2s(smem_addr(&stages[s].C[r][0]),
                                     cv.C + (int64_t)(g0 + r) * ldc + c0, (uint32_t)(w4 * 4), fb);
                    }
                    bulk_g2s(smem_addr(&stages[s].G[0]), w.G + c0, (uint32_t)(gw * 4), fb);
                    bulk_g2s(smem_addr(&stages[s].Gk[0]), w.Gk + c0, (uint32_t)(gw * 4), fb);
                }
            }
            // wait (bounded) for the copies still in flight before leaving
            const int total = t;
            for (int q = max(0, total - kStages); q < total; ++q)
                mbar_wait(smem_addr(&full[q % kStages]), (uint32_t)(q / kStages) & 1u, st);
        }
        return;
    }

    // ---------------------------------------------------------- consumers
    const float kh = st->k_hi, kl = st->k_lo;
    const double shift_g = st->shift_g, inv_eps = st->inv_eps_c;
    const double eps_c = st->eps_c, shift_f = st->shift_f;
    double my_dual = 0.0, my_cost = 0.0;   // lane 0 of each consumer warp
    int t = 0;
    bool ok = true;
    for (int gi = 0; gi < ngroups && ok; ++gi) {
        const int g0 = r0 + gi * kGR;
        const int nrows = min(kGR, r1 - g0);
        const int lr0 = warp * kRW;                 // first local row of this warp
        Acc acc[kRW], cacc[kRW];
#pragma unroll
        for (int r = 0; r < kRW; ++r) {
            acc[r] = {0.0f, 0.0f, 0.0f};
            cacc[r] = {0.0f, 0.0f, 0.0f};
        }
        for (int ti = 0; ti < ntiles_row; ++ti, ++t) {
            const int s = t % kStages;
            const uint32_t ph = (uint32_t)(t / kStages) & 1u;
            if (!mbar_wait(smem_addr(&full[s]), ph, st)) { ok = false; break; }
            const int c0 = tile_col(ti);
            const int wdt = min(kTW, m - c0);
            const int w4 = wdt & ~3;
            const Stage &S = stages[s];
            // this lane's float4 slots: lane + 32 k, k < kSlots (conflict-free)
            float4 g[kSlots], gk[kSlots];
            bool full4[kSlots], part[kSlots];
            bool any_part = false;
#pragma unroll
            for (int k = 0; k < kSlots; ++k) {
                const int v4 = 4 * (lane + 32 * k);
                full4[k] = v4 < w4;
                part[k] = (v4 == w4) && (v4 < wdt);
                any_part |= part[k];
                if (full4[k] || part[k]) {
                    g[k] = *reinterpret_cast<const float4 *>(&S.G[v4]);
                    gk[k] = *reinterpret_cast<const float4 *>(&S.Gk[v4]);
                } else {
                    g[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    gk[k] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
                }
                if (part[k]) {   // mask the columns past the ragged end
                    if (v4 + 1 >= wdt) { g[k].y = 0.f; gk[k].y = -INFINITY; }
                    if (v4 + 2 >= wdt) { g[k].z = 0.f; gk[k].z = -INFINITY; }
                    if (v4 + 3 >= wdt) { g[k].w = 0.f; gk[k].w = -INFINITY; }
                }
            }
#pragma unroll
            for (int r = 0; r < kRW; ++r) {
                const int lr = lr0 + r;
                if (lr >= nrows) break;
                float4 c[kSlots];
#pragma unroll
                for (int k = 0; k < kSlots; ++k) {
                    const int v4 = 4 * (lane + 32 * k);
                    if (full4[k]) {
                        c[k] = *reinterpret_cast<const float4 *>(&S.C[lr][v4]);
                    } else if (part[k]) {
                        // ragged tail (< 4 columns) straight from global memory
                        const float *src = cv.C + (int64_t)(g0 + lr) * ldc + c0 + v4;
                        c[k].x = ld_stream1(src);
                        c[k].y = (v4 + 1 < wdt) ? ld_stream1(src + 1) : 0.0f;
                        c[k].z = (v4 + 2 < wdt) ? ld_stream1(src + 2) : 0.0f;
                        c[k].w = (v4 + 3 < wdt) ? ld_stream1(src + 3) : 0.0f;
                    } else {
                        c[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                (void)any_part;
                // s = G - C once; the chunk max of s is the new reference
                float4 sv[kSlots];
                float cm = acc[r].R;
#pragma unroll
                for (int k = 0; k < kSlots; ++k) {
                    sv[k] = make_float4(g[k].x - c[k].x, g[k].y - c[k].y, g[k].z - c[k].z,
                                        g[k].w - c[k].w);
                    cm = fmaxf(cm, fmaxf(fmaxf(sv[k].x, sv[k].y), fmaxf(sv[k].z, sv[k].w)));
                }
                if (cm > acc[r].R) {
                    const float f = exp2_scaled(acc[r].R - cm, kh, kl);
                    acc[r].S = __fmul_rn(acc[r].S, f);
                    acc[r].K = __fmul_rn(acc[r].K, f);
                    if (WITH_COST) { cacc[r].S = __fmul_rn(cacc[r].S, f); cacc[r].K = __fmul_rn(cacc[r].K, f); }
                    acc[r].R = cm;
                }
                const float R = acc[r].R;
                float cs[kSlots], ccs[kSlots];
#pragma unroll
                for (int k = 0; k < kSlots; ++k) {
                    float p0 = term_s(sv[k].x, g[k].x, gk[k].x, c[k].x, R, kh, kl);
                    float p1 = term_s(sv[k].y, g[k].y, gk[k].y, c[k].y, R, kh, kl);
                    float p2 = term_s(sv[k].z, g[k].z, gk[k].z, c[k].z, R, kh, kl);
                    float p3 = term_s(sv[k].w, g[k].w, gk[k].w, c[k].w, R, kh, kl);
                    cs[k] = (p0 + p1) + (p2 + p3);
                    if (WITH_COST)
                        ccs[k] = fmaf(c[k].x, p0, fmaf(c[k].y, p1, fmaf(c[k].z, p2, c[k].w * p3)));
                }
                float csum = cs[0], ccsum = WITH_COST ? ccs[0] : 0.0f;
#pragma unroll
                for (int k = 1; k < kSlots; ++k) {
                    csum += cs[k];
                    if (WITH_COST) ccsum += ccs[k];
                }
                kahan(acc[r], csum);
                if (WITH_COST) kahan(cacc[r], ccsum);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
        }
        if (!ok) break;
        // finish this warp's rows: warp max of R, FP64 sum of rescaled partials
#pragma unroll
        for (int r = 0; r < kRW; ++r) {
            const int lr = lr0 + r;
            if (lr >= nrows) break;
            const float Rrow = warp_max(acc[r].R);
            const double sc = (double)exp2_scaled(acc[r].R - Rrow, kh, kl);
            const double S = warp_sum(((double)acc[r].S - (double)acc[r].K) * sc);
            double CS = 0.0;
            if (WITH_COST) CS = warp_sum(((double)cacc[r].S - (double)cacc[r].K) * sc);
            if (lane == 0) {
                const int i = g0 + lr;
                const double lse = ((double)Rrow - shift_g) * inv_eps + log(S);
                const double ui = w.loga[i] - lse;
                w.u[i] = ui;
                const double F = eps_c * ui + shift_f;
                const float Fh = (float)F;
                const float Fl = (float)(F - (double)Fh);
                w.FF[i] = make_float2(Fh, Fl * kh);
                w.Fh[i] = Fh;        // the operand of the column pass over C^T
                w.Fk[i] = Fl * kh;
                my_dual += w.a[i] * ui;
                if (WITH_COST) {
                    const double wi = w.f_given ? exp(w.f_given[i] / st->eps_user + lse) : w.a[i];
                    my_cost += wi * (CS / S);
                }
            }
        }
    }
    // per-CTA partials, summed over consumer warps in a fixed order
    __shared__ double sh_part[2][kNCW];
    if (lane == 0) {
        sh_part[0][warp] = my_dual;
        sh_part[1][warp] = my_cost;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(32 * kNCW) : "memory");
    if (threadIdx.x == 0) {
        double d = 0.0, c = 0.0;
        for (int q = 0; q < kNCW; ++q) { d += sh_part[0][q]; c += sh_part[1][q]; }
        w.rowpart[2 * blockIdx.x + 0] = d;
        w.rowpart[2 * blockIdx.x + 1] = c;
    }
}

using GeoA = RowGeo<2, 8, 512, 5>;    // 16-row groups of 2 rows per consumer warp, 9 warps

static int g_row_kernel = 0;

int row_kernel_choice() { return g_row_kernel; }

cudaError_t launch_row_pass_tma(const CostView &cv, const Work &w, int grid, bool with_cost,
                                cudaStream_t s)
{
    if (with_cost)
        k_row_pass_tma<GeoA, true><<<grid, GeoA::kNT, GeoA::kSmemBytes, s>>>(cv, w);
    else
        k_row_pass_tma<GeoA, false><<<grid, GeoA::kNT, GeoA::kSmemBytes, s>>>(cv, w);
    return cudaGetLastError();
}

// Must run once per process before the first launch (outside any capture):
// opts the kernels in to their dynamic shared memory. ACCSINK_ROW_KERNEL=tma
// selects this pipeline for the 128-bit-aligned row pass instead of the
// warp-per-row kernel (measured slower; kept as the bulk-copy alternative).
cudaError_t setup_row_pass_tma()
{
    const char *k = getenv("ACCSINK_ROW_KERNEL");
    if (k && k[0] == 't') g_row_kernel = 1;
    if (k && k[0] == 'w') g_row_kernel = 0;
    cudaError_t e = cudaFuncSetAttribute(k_row_pass_tma<GeoA, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GeoA::kSmemBytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_row_pass_tma<GeoA, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GeoA::kSmemBytes);
}

int row_pass_tma_smem_bytes() { return (int)GeoA::kSmemBytes; }

}  // namespace accsink

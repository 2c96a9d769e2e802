// Allocation-free variant of the column log-sum-exp pass.
//
// Some callers cannot allocate device memory at the moment they need the
// pass: a serving process whose memory pool has already claimed the whole
// GPU, a plugin running under another framework's allocator, or a real-time
// loop that cannot afford the implicit device synchronisation of cudaMalloc.
// For them, accsink_col_lse_noalloc() runs the same kernels as
// accsink_col_lse() without a context: every intermediate (the column-pass
// operand, the per-split partials, the reduction partials and the small
// solver state) lives in one file-scope device array of fixed size. The
// CUDA module that holds it is loaded on a device, and the array reserved
// there, when the first call on that device looks up its address (under
// lazy module loading, CUDA's default) or when the library's context is
// created (eager loading); it is kept until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "accsink.h"
#include "accsink_internal.cuh"

namespace accsink {

// 16 MiB of scratch per device. It bounds n * 8 + (row splits) * m * 8 bytes
// plus a few KB; the row splits shrink (down to one) to fit larger m.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

__global__ void k_noalloc_state(DevState v, DevState *dst) { *dst = v; }

}  // namespace accsink

using namespace accsink;

namespace {

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];   // device address of the array, per device
bool g_scratch_ready[kMaxDevices];
std::mutex g_scratch_mu;

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" int accsink_col_lse_noalloc(const accsink_problem *prob, double eps,
                                       const double *f, double *ell_out, void *stream)
{
    if (!prob || !f || !ell_out || !prob->C) return ACCSINK_ERR_INVALID_ARG;
    if (prob->cost_kind != ACCSINK_COST_DENSE) return ACCSINK_ERR_UNSUPPORTED;
    if (prob->n < 1 || prob->m < 1) return ACCSINK_ERR_INVALID_ARG;
    const int64_t ldc = prob->ldc ? prob->ldc : prob->m;
    if (ldc < prob->m) return ACCSINK_ERR_INVALID_ARG;
    if (!(eps > 0.0) || !(eps < INFINITY)) return ACCSINK_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ACCSINK_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ACCSINK_ERR_INVALID_ARG;

    CostView cv;
    cv.C = prob->C;
    cv.ldc = ldc;
    cv.n = prob->n;
    cv.m = prob->m;
    cv.vec = ((ldc % 4) == 0 && (((uintptr_t)prob->C) & 15u) == 0) ? 1 : 0;

    // Launch geometry, as the context-based pass chooses it.
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ACCSINK_ERR_CUDA;
    const int n = cv.n, m = cv.m;
    const int stat_grid = std::max(1, std::min(n, 4 * sms));
    const int vec_grid = std::max(1, std::min(sms, (std::max(n, m) + 63) / 64));
    const int strips = (m + kColStrip - 1) / kColStrip;
    int splits = (sms * occupancy_col_pass(cv.vec)) / strips;
    splits = std::max(1, std::min(splits, std::max(1, n / 8)));

    // Carve the scratch; reject sizes that do not fit even with one split,
    // before any kernel touches the caller's data.
    const size_t fixed = up256(sizeof(DevState)) + up256((size_t)stat_grid * 4 * 8) +
                         up256((size_t)vec_grid * kPartStride * 8) + up256((size_t)n * 8);
    const size_t per_split = (size_t)m * 8;
    if (fixed + up256(per_split) > kNoAllocScratchBytes) return ACCSINK_ERR_BUDGET;
    // The chosen splits hold about (SMs x CTAs per SM x 128) columns of
    // partials in all, ~1.2 MB on 152 SMs, so this guard only acts on
    // devices with far more resident CTAs.
    while (splits > 1 && fixed + up256(per_split * (size_t)splits) > kNoAllocScratchBytes)
        --splits;

    // First call on this device: look up the array's device address (the
    // host-side symbol is only a stand-in, not a device pointer).
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ready[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return ACCSINK_ERR_CUDA;
            g_scratch_addr[dev] = ptr;
            g_scratch_ready[dev] = true;
        }
        base = g_scratch_addr[dev];
    }
    char *p = (char *)base;
    Work w{};
    w.st = (DevState *)p;               p += up256(sizeof(DevState));
    w.statpart = (double *)p;           p += up256((size_t)stat_grid * 4 * 8);
    w.steppart = (double *)p;           p += up256((size_t)vec_grid * kPartStride * 8);
    w.FF = (float2 *)p;                 p += up256((size_t)n * 8);
    w.colpart = (float2 *)p;
    w.nstat = stat_grid;
    w.ignore_done = 1;

    // The array keeps whatever the previous call left; the state (including
    // the grid-barrier counter, which must start at zero) is rewritten here.
    // On a completed call every other region is overwritten before it is
    // read. If the preparation kernel's bounded grid barrier runs out, the
    // state records the timeout, the column pass does not run and the
    // finish writes NaN to every ell_j instead of reading stale partials.
    DevState hs;
    memset(&hs, 0, sizeof(hs));
    hs.eps_user = eps;
    hs.col_splits = splits;
    hs.mode = STEP_MAP;
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_state<<<1, 1, 0, s>>>(hs, w.st);
    if (cudaGetLastError() != cudaSuccess) return ACCSINK_ERR_CUDA;
    if (launch_cost_stats(cv, w, stat_grid, s) != cudaSuccess) return ACCSINK_ERR_CUDA;
    if (launch_prep_f(cv, w, vec_grid, f, eps, prob->cost_scale == ACCSINK_SCALE_MAX_TO_ONE, s) !=
        cudaSuccess)
        return ACCSINK_ERR_CUDA;
    if (launch_col_pass(cv, w, splits, s) != cudaSuccess) return ACCSINK_ERR_CUDA;
    if (launch_col_finish_lse(w, m, ell_out, s) != cudaSuccess) return ACCSINK_ERR_CUDA;
    return ACCSINK_OK;
}

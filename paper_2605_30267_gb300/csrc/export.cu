// Export of a solution: the transport plan P_ij = exp((f_i + g_j - C_ij) / eps)
// (eq. P-from-dual) and the barycentric projection of target features through
// it (Sec. 5, colour transfer). These are one-off utilities after a solve, not
// the iteration's hot path: every entry is formed in FP64 from the inputs as
// the problem defines it (FP32 C, or the FP32 points' cost in FP64), and the
// exponential is the FP64 one.
#include <float.h>

#include <algorithm>

#include "accsink.h"
#include "accsink_internal.cuh"

namespace accsink {

namespace {

struct ExportView {
    const float *C, *X, *Y;
    int64_t ldc;
    int32_t n, m, d, kind;
};

__device__ __forceinline__ double cost_entry(const ExportView &v, int i, int j)
{
    if (v.kind == 0) return (double)v.C[(int64_t)i * v.ldc + j];
    double s = 0.0;
    if (v.kind == 1) {
        for (int k = 0; k < v.d; ++k) {
            const double t = (double)v.X[(int64_t)i * v.d + k] - (double)v.Y[(int64_t)j * v.d + k];
            s += t * t;
        }
        return s;
    }
    for (int k = 0; k < v.d; ++k)
        s += (double)v.X[(int64_t)i * v.d + k] * (double)v.Y[(int64_t)j * v.d + k];
    return 1.0 - s;
}

__device__ __forceinline__ unsigned long long enc(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double dec(unsigned long long e)
{
    const unsigned long long b = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    return __longlong_as_double((long long)b);
}

// max_ij C_ij (for MAX_TO_ONE), as an ordered encoding.
__global__ void k_export_cmax(ExportView v, unsigned long long *out)
{
    double mx = -DBL_MAX;
    const int64_t total = (int64_t)v.n * v.m;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        mx = fmax(mx, cost_entry(v, (int)(t / v.m), (int)(t % v.m)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, enc(mx));
}

// Writes P (n rows of ld_p entries) in FP32 (F64 false) or FP64.
template <bool F64>
__global__ void k_export_plan(ExportView v, double eps, const double *f, const double *g,
                              const unsigned long long *cmax_enc, int scale, void *P,
                              int64_t ld_p)
{
    const double s = (scale && cmax_enc) ? 1.0 / dec(*cmax_enc) : 1.0;
    const double inv_eps = 1.0 / eps;
    for (int i = blockIdx.x; i < v.n; i += gridDim.x) {
        const double fi = f[i];
        for (int j = threadIdx.x; j < v.m; j += blockDim.x) {
            const double p = exp((fi + g[j] - s * cost_entry(v, i, j)) * inv_eps);
            if (F64) static_cast<double *>(P)[(int64_t)i * ld_p + j] = p;
            else static_cast<float *>(P)[(int64_t)i * ld_p + j] = (float)p;
        }
    }
}

// out_i = sum_j P_ij Z_j / sum_j P_ij, one warp per row, FP64 sums.
constexpr int kMaxDz = 16;

__global__ void k_export_bary(ExportView v, double eps, const double *f, const double *g,
                              const unsigned long long *cmax_enc, int scale, const float *Z,
                              int dz, int k0, int kc, double *out)
{
    const double s = (scale && cmax_enc) ? 1.0 / dec(*cmax_enc) : 1.0;
    const double inv_eps = 1.0 / eps;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < v.n; i += nw) {
        double acc[kMaxDz], mass = 0.0;
#pragma unroll
        for (int k = 0; k < kMaxDz; ++k) acc[k] = 0.0;
        for (int j = lane; j < v.m; j += 32) {
            const double p = exp((f[i] + g[j] - s * cost_entry(v, i, j)) * inv_eps);
            mass += p;
#pragma unroll
            for (int k = 0; k < kMaxDz; ++k)
                if (k < kc) acc[k] += p * (double)Z[(int64_t)j * dz + k0 + k];
        }
        for (int o = 16; o > 0; o >>= 1) mass += __shfl_xor_sync(0xffffffffu, mass, o);
#pragma unroll
        for (int k = 0; k < kMaxDz; ++k) {
            double a = acc[k];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0 && k < kc) out[(int64_t)i * dz + k0 + k] = a / mass;
        }
    }
}

}  // namespace

}  // namespace accsink

namespace {

using namespace accsink;

int export_view(const accsink_problem *p, ExportView &v)
{
    if (!p || p->n < 1 || p->m < 1) return ACCSINK_ERR_INVALID_ARG;
    v.n = p->n;
    v.m = p->m;
    v.ldc = p->ldc ? p->ldc : p->m;
    v.C = p->C;
    v.X = p->X;
    v.Y = p->Y;
    v.d = p->d;
    if (p->cost_kind == ACCSINK_COST_DENSE) {
        if (!p->C || v.ldc < p->m) return ACCSINK_ERR_INVALID_ARG;
        v.kind = 0;
    } else if (p->cost_kind == ACCSINK_COST_SQEUCLID || p->cost_kind == ACCSINK_COST_COSINE) {
        if (!p->X || !p->Y || p->d < 1 || p->d > 4096) return ACCSINK_ERR_INVALID_ARG;
        v.kind = p->cost_kind == ACCSINK_COST_SQEUCLID ? 1 : 2;
    } else {
        return ACCSINK_ERR_INVALID_ARG;
    }
    if (p->cost_scale != ACCSINK_SCALE_NONE && p->cost_scale != ACCSINK_SCALE_MAX_TO_ONE)
        return ACCSINK_ERR_INVALID_ARG;
    return ACCSINK_OK;
}

// max C into a device scratch word when the problem is scaled; returns the
// device pointer (or null) through *enc_out. The caller frees it.
int export_cmax(const accsink_problem *p, const ExportView &v, cudaStream_t s,
                unsigned long long **enc_out)
{
    *enc_out = nullptr;
    if (p->cost_scale != ACCSINK_SCALE_MAX_TO_ONE) return ACCSINK_OK;
    unsigned long long *e = nullptr;
    if (cudaMallocAsync(&e, sizeof(unsigned long long), s) != cudaSuccess) {
        cudaGetLastError();
        return ACCSINK_ERR_OOM;
    }
    if (cudaMemsetAsync(e, 0, sizeof(unsigned long long), s) != cudaSuccess) return ACCSINK_ERR_CUDA;
    k_export_cmax<<<1024, 256, 0, s>>>(v, e);
    if (cudaGetLastError() != cudaSuccess) return ACCSINK_ERR_CUDA;
    *enc_out = e;
    return ACCSINK_OK;
}

}  // namespace

extern "C" {

int accsink_plan(accsink_ctx *ctx, const accsink_problem *prob, double eps, const double *f,
                 const double *g, void *P_out, int64_t ld_p, int32_t dtype, void *stream)
{
    (void)ctx;
    ExportView v;
    int rc = export_view(prob, v);
    if (rc != ACCSINK_OK) return rc;
    if (!f || !g || !P_out || ld_p < prob->m || (dtype != 0 && dtype != 1) ||
        !(eps > 0.0))
        return ACCSINK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *e = nullptr;
    rc = export_cmax(prob, v, s, &e);
    if (rc != ACCSINK_OK) return rc;
    const int scale = prob->cost_scale == ACCSINK_SCALE_MAX_TO_ONE;
    const int grid = std::min(prob->n, 4096);
    if (dtype == 1) k_export_plan<true><<<grid, 256, 0, s>>>(v, eps, f, g, e, scale, P_out, ld_p);
    else k_export_plan<false><<<grid, 256, 0, s>>>(v, eps, f, g, e, scale, P_out, ld_p);
    const cudaError_t le = cudaGetLastError();
    if (e) cudaFreeAsync(e, s);
    return le == cudaSuccess ? ACCSINK_OK : ACCSINK_ERR_CUDA;
}

int accsink_barycentric(accsink_ctx *ctx, const accsink_problem *prob, double eps,
                        const double *f, const double *g, const float *Z, int32_t dz,
                        double *out, void *stream)
{
    (void)ctx;
    ExportView v;
    int rc = export_view(prob, v);
    if (rc != ACCSINK_OK) return rc;
    if (!f || !g || !Z || !out || dz < 1 || !(eps > 0.0)) return ACCSINK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *e = nullptr;
    rc = export_cmax(prob, v, s, &e);
    if (rc != ACCSINK_OK) return rc;
    const int scale = prob->cost_scale == ACCSINK_SCALE_MAX_TO_ONE;
    const int warps = 8;
    const int grid = std::max(1, std::min((prob->n + warps - 1) / warps, 8192));
    cudaError_t le = cudaSuccess;
    for (int k0 = 0; k0 < dz && le == cudaSuccess; k0 += kMaxDz) {
        k_export_bary<<<grid, 32 * warps, 0, s>>>(v, eps, f, g, e, scale, Z, dz, k0,
                                                  std::min(kMaxDz, dz - k0), out);
        le = cudaGetLastError();
    }
    if (e) cudaFreeAsync(e, s);
    return le == cudaSuccess ? ACCSINK_OK : ACCSINK_ERR_CUDA;
}

}  // extern "C"

// fmm_selftest.cu -- fmm_selftest_fp64: the double-precision square root and
// division helpers of fmm_fp64.cuh (used by the fp64 march and the adjoint)
// evaluated element-wise on caller arrays, so that a test can compare them
// with CUDA's correctly rounded sqrt and '/' over a sweep of operands;
// fmm_selftest_root: the double-float root of Algorithm 11 used by the fp64
// march, so that a test can check its causal set and root against exact
// arithmetic; fmm_probe_fma_rate: the FMA throughput of the device.
#include "fmm.h"
#include "fmm_df.cuh"
#include "fmm_fp64.cuh"

#include <cuda_runtime.h>

namespace {

__global__ void k_selftest_fp64(const double *__restrict__ a, const double *__restrict__ b,
                                double *__restrict__ sq, double *__restrict__ q, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        sq[i] = fmmgb::sqrt_fp64(a[i]);
        q[i] = fmmgb::div_fp64(a[i], b[i]);
    }
}

}  // namespace

extern "C" fmm_status fmm_selftest_fp64(const double *a, const double *b, double *sqrt_out,
                                        double *div_out, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!a || !b || !sqrt_out || !div_out)))
        return FMM_ERR_INVALID;
    if (n == 0)
        return FMM_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    k_selftest_fp64<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, sqrt_out, div_out, n);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// The double-grid root of Algorithm 11 (fmm_df.cuh's df_shifted_root) on
// caller arrays: sorted upwind values m <= v1 <= v2 (nd of them used), speed
// term q; returns the root and the size of the causal set it chose.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_selftest_root(const double *__restrict__ m, const double *__restrict__ v1,
                                const double *__restrict__ v2, const int *__restrict__ nd,
                                const double *__restrict__ q, double *__restrict__ t_out,
                                int *__restrict__ k_out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double t = 0.0;
        // as the march computes it when it records the upwind sets
        const int k = fmmgb::df_shifted_root<true>(m[i], v1[i], v2[i], nd[i], q[i], t);
        t_out[i] = k ? t : __longlong_as_double(0x7ff0000000000000ll);
        k_out[i] = k;
    }
}

}  // namespace

extern "C" fmm_status fmm_selftest_root(const double *m, const double *v1, const double *v2,
                                        const int32_t *nd, const double *q, double *t_out,
                                        int32_t *k_out, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!m || !v1 || !v2 || !nd || !q || !t_out || !k_out)))
        return FMM_ERR_INVALID;
    if (n == 0)
        return FMM_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    k_selftest_root<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(m, v1, v2, (const int *)nd, q, t_out,
                                                                 (int *)k_out, n);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Arithmetic throughput probe: the fused multiply-add rate of the device in
// float or double, the compute ceiling of the march kernels next to HBM
// bandwidth.  Every thread runs kChains independent multiply-add chains (so
// the pipe, not the latency of one chain, is the limit) for `iters` steps;
// the grid fills every SM several times over.
// ---------------------------------------------------------------------------
namespace {

constexpr int kChains = 8;
__device__ double g_probe_sink;

template <typename real>
__global__ void __launch_bounds__(256) k_probe_fma(long long iters, real x, real y)
{
    real a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        a[c] = (real)(threadIdx.x + c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            a[c] = fma(a[c], x, y);
    }
    real s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += a[c];
    if (s == (real)-1.2345)   // never true for these operands; keeps the chains live
        g_probe_sink = (double)s;
}

}  // namespace

extern "C" fmm_status fmm_probe_fma_rate(int32_t dtype, int64_t iters, double *flops_per_s)
{
    if (!flops_per_s || iters < 1 || (dtype != FMM_F32 && dtype != FMM_F64))
        return FMM_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FMM_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FMM_ERR_CUDA;
    }
    // a warm-up launch, then the timed one (x < 1 keeps the chains finite)
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, 0);
        if (dtype == FMM_F64)
            k_probe_fma<double><<<blocks, threads>>>(iters, 0.999999, 1e-3);
        else
            k_probe_fma<float><<<blocks, threads>>>(iters, 0.999999f, 1e-3f);
        cudaEventRecord(e1, 0);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || !(ms > 0.f))
        return FMM_ERR_CUDA;
    const double fmas = (double)blocks * threads * kChains * (double)iters;
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    return FMM_OK;
}

// kt_diag.cu -- diagnostic entry points (checks of device building blocks).
#include <cuda_runtime.h>

#include <cmath>

#include "kt_exp.cuh"
#include "kt_internal.h"

namespace kt {
namespace {

struct ExpTable {
    double v[kExpTable];
};

__global__ void exp_kernel(const double *x, double *out, long long n, int which, const ExpTable tab)
{
    __shared__ double t[kExpTable];
    if (threadIdx.x < kExpTable) t[threadIdx.x] = tab.v[threadIdx.x];
    __syncthreads();
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = which ? tang_exp(x[i], t) : exp(x[i]);
}

}  // namespace
}  // namespace kt

extern "C" KT_API int kt_debug_exp(const double *x, double *out, int64_t n, int which, void *cuda_stream)
{
    if (!x || !out || n < 0) return KT_EINVAL;
    if (n == 0) return KT_OK;
    kt::ExpTable tab;
    for (int j = 0; j < kt::kExpTable; ++j) tab.v[j] = kt::exp2_table(j);
    const int threads = 256;
    kt::exp_kernel<<<static_cast<unsigned>((n + threads - 1) / threads), threads, 0,
                     static_cast<cudaStream_t>(cuda_stream)>>>(x, out, n, which, tab);
    return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ECUDA;
}

// ----------------------------------------------------------------- FMA throughput
//
// A peak probe for the roofline denominators: every thread runs kChains independent
// fused multiply-add chains x <- x*a + b for `iters` rounds (2 flops each), so the
// FP64 or FP32 pipe is the only busy unit.  The result is stored only when it equals a
// value passed at run time that it never reaches, which keeps the loop alive without
// any memory traffic.

namespace kt {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename F>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(F *sink, long long iters, F a, F b, F never)
{
    F x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = static_cast<F>(threadIdx.x + c) * static_cast<F>(1e-3);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    F s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == never) *sink = s;
}

}  // namespace
}  // namespace kt

extern "C" KT_API int kt_fma_peak(int fp32, int64_t iters, int blocks, double *sink, void *cuda_stream,
                                  double *flops)
{
    if (!sink || iters < 1 || blocks < 0) return KT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return KT_ECUDA;
    if (blocks == 0) blocks = 8 * sms;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (fp32)
        kt::fma_peak_kernel<float><<<blocks, kt::kPeakThreads, 0, s>>>(
            reinterpret_cast<float *>(sink), iters, 0.999999f, 1e-7f, -1.2345e30f);
    else
        kt::fma_peak_kernel<double><<<blocks, kt::kPeakThreads, 0, s>>>(sink, iters, 0.999999999, 1e-9,
                                                                         -1.2345e300);
    if (flops)
        *flops = 2.0 * kt::kChains * static_cast<double>(iters) * blocks * kt::kPeakThreads;
    return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ECUDA;
}

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

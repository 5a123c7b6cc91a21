// kt_warp_f32.cu -- FP32-LU instantiations of the warp-per-cell kernels (kt_warp.cuh).
#include "kt_warp.cuh"

namespace kt {

int launch_warp_f32(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_warp_form<true>(a, c, static_cast<cudaStream_t>(stream));
}

}  // namespace kt

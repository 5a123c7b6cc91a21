// kt_warp.cu -- launch dispatch of the warp-per-cell kernels (kt_warp.cuh) and their
// FP64-matrix instantiations; the FP32-LU ones are compiled in kt_warp_f32.cu.
#include "kt_warp.cuh"

namespace kt {

int launch_warp_f64(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_warp_form<false>(a, c, static_cast<cudaStream_t>(stream));
}

int launch_warp(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return c.form == KT_FORM_FP32LU ? launch_warp_f32(a, c, stream) : launch_warp_f64(a, c, stream);
}

}  // namespace kt

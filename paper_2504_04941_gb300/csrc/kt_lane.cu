// kt_lane.cu -- launch dispatch of the lane-per-cell kernels: size-specialised
// instantiations for the networks with 3 and 11 unknowns (compile-time trip counts,
// fully unrolled linear algebra), the runtime-size kernels for every other N <= 16.
// This unit also compiles the runtime-size FP64-matrix kernels.
#include "kt_lane.cuh"

namespace kt {

int launch_lane_any_f64(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_lane_form<0, false>(a, c, static_cast<cudaStream_t>(stream));
}

int launch_lane(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    const bool f32 = c.form == KT_FORM_FP32LU;
    if (a.nv.N == 3) return launch_lane_n3(a, c, stream);
    if (a.nv.N == 11) return f32 ? launch_lane_n11_f32(a, c, stream) : launch_lane_n11_f64(a, c, stream);
    return f32 ? launch_lane_any_f32(a, c, stream) : launch_lane_any_f64(a, c, stream);
}

}  // namespace kt

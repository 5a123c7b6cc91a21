// kt_lane_any_f32.cu -- runtime-size (N <= 16) FP32-LU lane-per-cell kernels.
#include "kt_lane.cuh"

namespace kt {

int launch_lane_any_f32(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_lane_form<0, true>(a, c, static_cast<cudaStream_t>(stream));
}

}  // namespace kt

// kt_lane_n11_f32.cu -- lane-per-cell kernels specialised for 11 unknowns per cell,
// FP32-LU form.
#include "kt_lane.cuh"

namespace kt {

int launch_lane_n11_f32(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_lane_form<11, true>(a, c, static_cast<cudaStream_t>(stream));
}

}  // namespace kt

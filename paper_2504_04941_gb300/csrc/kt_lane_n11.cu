// kt_lane_n11.cu -- lane-per-cell kernels specialised for 11 unknowns per cell, FP64
// iteration matrix (the FP32-LU ones are in kt_lane_n11_f32.cu).
#include "kt_lane.cuh"

namespace kt {

int launch_lane_n11_f64(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_lane_form<11, false>(a, c, static_cast<cudaStream_t>(stream));
}

}  // namespace kt

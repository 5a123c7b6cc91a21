// kt_lane_n11.cu -- lane-per-cell kernels specialised for 11 unknowns per cell.
#include "kt_lane.cuh"

namespace kt {

int launch_lane_n11(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_lane_n<11>(a, c, static_cast<cudaStream_t>(stream));
}

}  // namespace kt

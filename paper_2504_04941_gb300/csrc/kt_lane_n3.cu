// kt_lane_n3.cu -- lane-per-cell kernels specialised for 3 unknowns per cell.
#include "kt_lane.cuh"

namespace kt {

int launch_lane_n3(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    return launch_lane_n<3>(a, c, static_cast<cudaStream_t>(stream));
}

}  // namespace kt

// kt_lane.cu -- launch dispatch of the lane-per-cell kernels: size-specialised
// instantiations for the networks with 3 and 11 unknowns (compile-time trip counts,
// fully unrolled linear algebra), the runtime-size kernels for every other N <= 16.
#include "kt_lane.cuh"

namespace kt {

int launch_lane(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    if (a.nv.N == 3) return launch_lane_n3(a, c, stream);
    if (a.nv.N == 11) return launch_lane_n11(a, c, stream);
    return launch_lane_n<0>(a, c, static_cast<cudaStream_t>(stream));
}

}  // namespace kt

// kt_lane_n3.cu -- lane-per-cell kernels specialised for 3 unknowns per cell (both forms).
#include "kt_lane.cuh"

namespace kt {

int launch_lane_n3(const LaunchArgs &a, const LaunchCfg &c, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return c.form == KT_FORM_FP32LU ? launch_lane_form<3, true>(a, c, s) : launch_lane_form<3, false>(a, c, s);
}

}  // namespace kt

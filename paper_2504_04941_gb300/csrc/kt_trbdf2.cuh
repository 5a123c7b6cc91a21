// kt_trbdf2.cuh -- coefficients of the TR-BDF2 one-step scheme (Bank et al. 1985).
//
// A step of size h is a trapezoidal stage to t + gamma h and a BDF2 stage to t + h,
// gamma = 2 - sqrt(2).  Both stages are y = r + d h f(y) with d = gamma / 2, so one
// iteration matrix I - d h J serves the whole step:
//   stage 1: r = y_n + d h f(y_n)                                  -> y_g
//   stage 2: r = w1 y_g - w0 y_n, w1 = 1 / (gamma (2 - gamma)),
//            w0 = (1 - gamma)^2 / (gamma (2 - gamma))              -> y_{n+1}
// The local error C h^3 y''' (C = (-3 gamma^2 + 4 gamma - 2) / (12 (2 - gamma))) is
// estimated from f at t, t + gamma h and t + h (the quadratic through them):
//   est = 2 C h (a0 f_n + a1 f_g + a2 f_{n+1}),
//   a0 = 1/gamma, a1 = -1/(gamma (1 - gamma)), a2 = 1/(1 - gamma),
// with f_g = (y_g - y_n)/(d h) - f_n and f_{n+1} = (y_{n+1} - r)/(d h) taken from the
// stage equations.  The constants are formed with explicitly rounded operations (no
// contraction into fused multiply-adds) in the order of their definitions above.
#pragma once

#include <cuda_runtime.h>

namespace kt {

struct TrCoef {
    double g, d, w1, w0, C, a0, a1, a2;
};

__device__ __forceinline__ TrCoef tr_coef()
{
    TrCoef k;
    k.g = __dadd_rn(2.0, -__dsqrt_rn(2.0));
    k.d = __dmul_rn(0.5, k.g);
    const double twomg = __dadd_rn(2.0, -k.g), onemg = __dadd_rn(1.0, -k.g);
    const double g2g = __dmul_rn(k.g, twomg);
    k.w1 = __ddiv_rn(1.0, g2g);
    k.w0 = __ddiv_rn(__dmul_rn(onemg, onemg), g2g);
    const double num = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(-3.0, k.g), k.g), __dmul_rn(4.0, k.g)), -2.0);
    k.C = __ddiv_rn(num, __dmul_rn(12.0, twomg));
    k.a0 = __ddiv_rn(1.0, k.g);
    k.a1 = -__ddiv_rn(1.0, __dmul_rn(k.g, onemg));
    k.a2 = __ddiv_rn(1.0, onemg);
    return k;
}

}  // namespace kt

// kt_exp.cuh -- table-driven double-precision exponential (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic",
// ACM TOMS 15(2), 1989), written for this library.
//
// x = (32 m + j) ln2/32 + r with |r| <= ln2/64, so exp(x) = 2^m * 2^(j/32) * e^r.
// ln2/32 is split into a head with 32 significant bits (n * head is exact for
// |n| < 2^21) and a tail; e^r - 1 is the Taylor polynomial of degree 6 (truncation
// below 2e-18 relative for |r| <= 0.0109).  2^(j/32) comes from a 32-entry table,
// built on the host in long double and rounded once.  Valid for -708 <= x <= 709
// (callers flush smaller arguments to zero); ~11 FP64 operations against ~17 for the
// general-purpose exp on this part.
#pragma once

#include <cstdint>

namespace kt {

constexpr int kExpTable = 32;

// exp(x) for -708 <= x <= 709, tab[j] = 2^(j/32) rounded to double.
__device__ __forceinline__ double tang_exp(double x, const double *tab)
{
    const double inv_l = 46.16624130844683;             // 32 / ln 2
    const double l_head = 0x1.62e42ff000000p-6;         // ln2/32 to 32 significant bits
    const double l_tail = -1.312785960212839e-12;       // ln2/32 - l_head
    const double nd = rint(x * inv_l);
    const int n = static_cast<int>(nd);
    const int j = n & 31;
    const int m = (n - j) >> 5;
    const double r = fma(-nd, l_tail, fma(-nd, l_head, x));
    // e^r - 1 = r + r^2 (1/2 + r (1/6 + r (1/24 + r (1/120 + r /720))))
    double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    q = fma(r, q, 1.0 / 24.0);
    q = fma(r, q, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    const double p = fma(r * r, q, r);
    const double s = tab[j];
    const double v = fma(s, p, s);
    // scale by 2^m through the exponent field (v is in [1, 2.2) and m in [-1023, 1023])
    const long long bits = __double_as_longlong(v) + (static_cast<long long>(m) << 52);
    return __longlong_as_double(bits);
}

}  // namespace kt

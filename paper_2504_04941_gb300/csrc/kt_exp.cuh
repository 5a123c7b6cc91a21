// kt_exp.cuh -- table-driven double-precision exponential (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic",
// ACM TOMS 15(2), 1989), written for this library.
//
// x = (256 m + j) ln2/256 + r with |r| <= ln2/512, so exp(x) = 2^m * 2^(j/256) * e^r.
// n = 256 m + j is x * 256/ln2 rounded to the nearest integer by adding 1.5 * 2^52
// (the sum's last bit is the integer: the low word of its bit pattern is n), so no
// FP64 rounding or conversion instruction is needed.  ln2/256 is split into a head
// with 32 significant bits (n * head is exact for |n| < 2^21) and a tail; e^r - 1 is
// the Taylor polynomial of degree 4 (truncation below 4e-17 relative for
// |r| <= 0.00136).  2^(j/256) comes from a 256-entry table, built on the host in long
// double and rounded once.  Valid for -708 <= x <= 709 (callers flush smaller
// arguments to zero); 9 FP64 operations against ~17 for the general-purpose exp on
// this part.
#pragma once

#include <cstdint>

#include "kt_internal.h"

namespace kt {

// exp(x) for -708 <= x <= 709, tab[j] = 2^(j/256) rounded to double.
__device__ __forceinline__ double tang_exp(double x, const double *tab)
{
    const double inv_l = 369.3299304675746;             // 256 / ln 2
    const double shift = 6755399441055744.0;            // 1.5 * 2^52
    const double l_head = 0x1.62e42fee00000p-9;         // ln2/256 to 32 significant bits
    const double l_tail = 0x1.a39ef35793c76p-41;        // ln2/256 - l_head
    const double t = fma(x, inv_l, shift);
    const int n = __double2loint(t);
    const double nd = t - shift;
    const int j = n & (kExpTable - 1);
    const int m = (n - j) >> 8;
    const double r = fma(-nd, l_tail, fma(-nd, l_head, x));
    // e^r - 1 = r + r^2 (1/2 + r (1/6 + r / 24))
    double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    const double p = fma(r * r, q, r);
    const double s = tab[j];
    const double v = fma(s, p, s);
    // scale by 2^m through the exponent field (v is in [1, 2.01) and m in [-1023, 1023])
    const long long bits = __double_as_longlong(v) + (static_cast<long long>(m) << 52);
    return __longlong_as_double(bits);
}

}  // namespace kt

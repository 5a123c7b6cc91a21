// kt_lane.cuh -- lane-per-cell fused integrator for small networks (N <= 16 unknowns).
//
// One CUDA thread owns one cell for its whole integration (Sec. 2.2 of the paper:
// cells are independent).  The paper gives each cell a thread block and splits the
// reactions and LU rows over threads (Sec. 2.3); for 3..16 unknowns that leaves most
// of a warp idle on every FP64 instruction, and GB300's FP64 pipe is the scarce
// resource, so here the 32 lanes of a warp integrate 32 different cells with the
// same instruction stream.
//
// The sub-step control is flattened into a per-lane state machine: every trip of the
// main loop performs exactly ONE Newton iteration for every live lane (rates ->
// residual -> Jacobian -> Crout LU -> solve -> update), whatever phase of its
// step-doubling attempt the lane is in.  Lanes of one warp therefore run the heavy
// FP64 work in lockstep even though their cells need very different numbers of
// sub-steps; only the cheap control logic diverges.  With `persistent`, a lane whose
// cell is done pulls the next cell from a device work queue (one atomicAdd per warp
// per refill, warp-aggregated), so no lane idles until the queue is empty.
//
// Per-cell arrays (iteration matrix, factors, pivots, state vectors) live in shared
// memory, lane-interleaved (element e of lane l at [e*32 + l]): a warp reading "the
// same element of its 32 cells" touches 32 consecutive words, conflict-free even
// when the pivot row differs per lane.  The network tables are staged once per block
// by one bulk (TMA) copy and read with warp-uniform addresses (broadcast).
//
// Forms:
//   F32 = false  full Newton, FP64 Jacobian and LU (the plain form; same steps and
//                order as the FP64 oracle).
//   F32 = true   simplified Newton: the Jacobian is assembled in FP32 at the start of
//                each step attempt (and refreshed when the contraction stalls), the
//                iteration matrix I - h J is factorised in FP32 (once for h, once for
//                h/2), while the residual, the update, the convergence test, the
//                error norm and the conservation projection stay in FP64.
//   LEAN = true  (F32, TR-BDF2, size known at compile time) the iteration matrix is
//                assembled directly in FP32 without a Jacobian copy, y_n and f_n live
//                in registers and a failed FP32 solve halves h (no FP64 rescue): half
//                the shared memory per warp of the F32 layout, so twice the warps per
//                SM hide each other's FP64 and shared-memory latencies.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kt_exp.cuh"
#include "kt_internal.h"
#include "kt_mlp.cuh"
#include "kt_tma.cuh"
#include "kt_trbdf2.cuh"

namespace kt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps = 8;

#define LI(p, e) ((p)[(e) << 5])
// per-lane arrays with a stride of 2^SH words (FP32 arrays interleave two per lane)
#define LIS(p, e, SH) ((p)[(e) << (SH)])

enum LaneState : int { kNeed = 0, kRun = 1, kDone = 2 };

// A per-lane FP64 vector: in registers (REG; every index must be a compile-time
// constant once the loops are unrolled) or lane-interleaved in shared memory.
template <bool REG, int NR>
struct LaneVec {
    double r[NR];
    double *p;
    __device__ __forceinline__ double &operator[](int i)
    {
        if constexpr (REG) return r[i];
        else return p[i << 5];
    }
};

struct NetSmem {
    const double *A, *b, *th, *dH, *h, *cv, *cnt, *ex;
    const float *bf, *thf, *dHf;   // FP32 copies for the FP32 Jacobian (no FP64-pipe conversions)
    const unsigned long long *idx;
};

__device__ __forceinline__ NetSmem net_smem(const unsigned char *sm, const NetView &nv)
{
    NetSmem t;
    t.A = reinterpret_cast<const double *>(sm + nv.off_A);
    t.b = reinterpret_cast<const double *>(sm + nv.off_b);
    t.th = reinterpret_cast<const double *>(sm + nv.off_th);
    t.dH = reinterpret_cast<const double *>(sm + nv.off_dH);
    t.h = reinterpret_cast<const double *>(sm + nv.off_h);
    t.cv = reinterpret_cast<const double *>(sm + nv.off_cv);
    t.cnt = reinterpret_cast<const double *>(sm + nv.off_cnt);
    t.idx = reinterpret_cast<const unsigned long long *>(sm + nv.off_idx);
    t.ex = reinterpret_cast<const double *>(sm + nv.off_exp);
    t.bf = reinterpret_cast<const float *>(sm + nv.off_f32);
    t.thf = t.bf + nv.nr;
    t.dHf = t.thf + nv.nr;
    return t;
}

// x < -700 decided on the bit pattern (integer compare; same result as the FP64 compare
// for every non-NaN x): negative and |x| > 700.0 (0x4085E00000000000).
__device__ __forceinline__ bool below_m700(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 && (b & 0x7fffffffffffffffLL) > 0x4085E00000000000LL;
}

// Modified Arrhenius coefficient k = A (T/T_ref)^b exp(-theta/T) and dk/dT
// (Sec. 2.2.1 item 1); exponents below -700 give exactly zero.  The exponential is
// the table-driven one of kt_exp.cuh (within 2 ulp of exp()).
__device__ __forceinline__ void arrhenius(const NetSmem &t, int r, double lt, double invT,
                                          double &k, double &dk)
{
    const double b = t.b[r], th = t.th[r];
    const double arg = b * lt - th * invT;
    if (below_m700(arg)) {
        k = 0.0;
        dk = 0.0;
    } else {
        k = t.A[r] * tang_exp(arg, t.ex);
        dk = k * (b + th * invT) * invT;
    }
}

// k alone; dk/dT = k (b + theta/T) / T is formed only where the Jacobian needs it.
__device__ __forceinline__ double arrhenius_k(const NetSmem &t, int r, double lt, double invT)
{
    const double arg = t.b[r] * lt - t.th[r] * invT;
    return below_m700(arg) ? 0.0 : t.A[r] * tang_exp(arg, t.ex);
}

// log(T / T_ref), skipping the division when T_ref is 1 (the same value bit for bit).
__device__ __forceinline__ double log_t(double T, double t_ref)
{
    return log(t_ref == 1.0 ? T : T / t_ref);
}

// reactions whose rates are formed before their scatter (independent FP64 chains in
// flight); a build-time tuning knob, the results do not depend on it
#ifndef KT_LANE_CHUNK
#define KT_LANE_CHUNK 4
#endif
constexpr int kChunk = KT_LANE_CHUNK;

// Jacobian scatter of one A + B -> C + D reaction with four different species: the
// rows {i0, i1, o0, o1, T} and columns {i0, i1, T} it touches are all different
// entries, so every entry is loaded first and stored after (one shared-memory round
// trip per reaction instead of a chain of read-modify-writes the compiler must keep in
// order).  Each entry receives the same single update as in the general code:
// reactant rows + s d_c, product rows - s d_c, the T row + s (q d_c); s = +1 for
// M = I - h J (d_c = h dw/dy_c), s = -1 for J itself.
template <typename T, int SH, bool ENERGY>
__device__ __forceinline__ void scatter22(T *A, int N, int ns, int i0, int i1, int o0, int o1, T d0, T d1,
                                          T d2, T q, T s)
{
    constexpr int NR = ENERGY ? 5 : 4, NC = ENERGY ? 3 : 2;
    const int rows[5] = {i0, i1, o0, o1, ns};
    const int cols[3] = {i0, i1, ns};
    const T dc[3] = {d0, d1, d2};
    T v[NR][NC];
#pragma unroll
    for (int a = 0; a < NR; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) v[a][c] = LIS(A, rows[a] * N + cols[c], SH);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const T sd = s * dc[c];
        v[0][c] += sd;
        v[1][c] += sd;
        v[2][c] -= sd;
        v[3][c] -= sd;
        if (ENERGY) v[4][c] = fma(s * q, dc[c], v[4][c]);
    }
#pragma unroll
    for (int a = 0; a < NR; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) LIS(A, rows[a] * N + cols[c], SH) = v[a][c];
}

// One pass over the reactions at state yt (Eq. method-ode-thermochem and the
// mass-action / thermal-coupling partials of Eq. method-jacobian):
//   W  <- f(yt)                                   (always, FP64)
//   MODE 1: M64 <- I - hph * J(yt)                (FP64)
//   MODE 2: J32 <- J(yt) when doJ                 (FP32; residual still FP64)
//   MODE 3: J32 <- I - hph * J(yt) when doJ       (FP32, lane stride 32: the lean layout)
// The temperature row uses each reaction's heat dH_r = sum h_out - sum h_in:
// dT/dt = -sum_r dH_r w_r / C_V, an exact rewrite of -sum_s h_s (dn_s/dt) / C_V.
// Reactions go in chunks of kChunk: the rate coefficients and rates of a chunk are
// independent FP64 chains formed first, then scattered in reaction order (the same
// sums in the same order as one reaction at a time).  S2 = true when every reaction
// is A + B -> C + D (straight-line code; multiplying by the absent third reactant's
// 1.0 is exact, so the results are the same as the general code's).
template <int NT, bool ENERGY, int MODE, bool S2>
__device__ __forceinline__ void reaction_pass(const NetView &nv, const NetSmem &t,
                                              const double *__restrict__ yt, const double *__restrict__ K,
                                              double lt, double invT, double invCV, double hph,
                                              double *__restrict__ W, double *__restrict__ M64,
                                              float *__restrict__ J32, bool doJ)
{
    const int N = NT > 0 ? NT : nv.N, ns = nv.ns, nr = nv.nr;
#pragma unroll
    for (int i = 0; i < N; ++i) LI(W, i) = 0.0;
    if (MODE == 1) {
        for (int e = 0; e < N * N; ++e) LI(M64, e) = 0.0;
    }
    if (MODE == 2 && doJ) {
        for (int e = 0; e < N * N; ++e) LIS(J32, e, 6) = 0.0f;
    }
    if (MODE == 3 && doJ) {
        for (int e = 0; e < N * N; ++e) LIS(J32, e, 5) = 0.0f;
    }
    // FP32 Jacobian (MODE 2/3): every partial in FP32, dk/dT = k (b + theta/T)/T included;
    // it only shapes the simplified-Newton iteration matrix
    const float hf = static_cast<float>(hph), invTf = static_cast<float>(invT);
    const float invCVf = static_cast<float>(invCV);
    double fT = 0.0;
    for (int r0 = 0; r0 < nr; r0 += kChunk) {
        unsigned long long ixq[kChunk];
        double kq[kChunk], y0q[kChunk], y1q[kChunk], y2q[kChunk], wq[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int r = r0 + q < nr ? r0 + q : nr - 1;
            const unsigned long long ix = t.idx[r];
            ixq[q] = ix;
            const int nin = S2 ? 2 : static_cast<int>(ix & 0x7f);
            const int i0 = static_cast<int>((ix >> 16) & 0xff), i1 = static_cast<int>((ix >> 24) & 0xff),
                      i2 = static_cast<int>((ix >> 32) & 0xff);
            const double k = ENERGY ? arrhenius_k(t, r, lt, invT) : LI(K, r);
            const double y0 = LI(yt, i0);
            const double y1 = nin > 1 ? LI(yt, i1) : 1.0;
            const double y2 = (!S2 && nin > 2) ? LI(yt, i2) : 1.0;
            kq[q] = k;
            y0q[q] = y0;
            y1q[q] = y1;
            y2q[q] = y2;
            wq[q] = S2 ? k * (y0 * y1) : k * (y0 * y1) * y2;
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            if (r0 + q >= nr) break;
            const int r = r0 + q;
            const unsigned long long ix = ixq[q];
            const int nin = S2 ? 2 : static_cast<int>(ix & 0x7f);
            const int nout = S2 ? 2 : static_cast<int>((ix >> 8) & 0xff);
            const bool dist = S2 && (ix & kIdxDistinct);
            const int i0 = static_cast<int>((ix >> 16) & 0xff), i1 = static_cast<int>((ix >> 24) & 0xff),
                      i2 = static_cast<int>((ix >> 32) & 0xff);
            const int o0 = static_cast<int>((ix >> 40) & 0xff), o1 = static_cast<int>((ix >> 48) & 0xff),
                      o2 = static_cast<int>((ix >> 56) & 0xff);
            const double k = kq[q], y0 = y0q[q], y1 = y1q[q], y2 = y2q[q], w = wq[q];
            if (dist) {
                // four different species: load the four entries, then store them (one
                // shared-memory round trip instead of a chain of read-modify-writes)
                const double a0 = LI(W, i0), a1 = LI(W, i1), b0 = LI(W, o0), b1 = LI(W, o1);
                LI(W, i0) = a0 - w;
                LI(W, i1) = a1 - w;
                LI(W, o0) = b0 + w;
                LI(W, o1) = b1 + w;
            } else {
                LI(W, i0) -= w;
                if (nin > 1) LI(W, i1) -= w;
                if (!S2 && nin > 2) LI(W, i2) -= w;
                if (nout > 0) LI(W, o0) += w;
                if (nout > 1) LI(W, o1) += w;
                if (!S2 && nout > 2) LI(W, o2) += w;
            }
            double dHr = 0.0;
            if (ENERGY) {
                dHr = t.dH[r];
                fT -= dHr * w;
            }
            if (MODE == 1 && dist) {
                const double hk = hph * k;
                const double d2 = ENERGY ? hph * (k * (t.b[r] + t.th[r] * invT) * invT) * (y0 * y1) : 0.0;
                scatter22<double, 5, ENERGY>(M64, N, ns, i0, i1, o0, o1, hk * y1, hk * y0, d2,
                                             ENERGY ? dHr * invCV : 0.0, 1.0);
            } else if (MODE == 1) {
                // M = I - h J: a reactant row gains +h dw/dy_m, a product row -h dw/dy_m,
                // the T row +h (dH_r/C_V) dw/dy_m.
                const double hk = hph * k;
                const double q2 = ENERGY ? dHr * invCV : 0.0;
                auto col = [&](int m, double hd) {
                    LI(M64, i0 * N + m) += hd;
                    if (nin > 1) LI(M64, i1 * N + m) += hd;
                    if (!S2 && nin > 2) LI(M64, i2 * N + m) += hd;
                    if (nout > 0) LI(M64, o0 * N + m) -= hd;
                    if (nout > 1) LI(M64, o1 * N + m) -= hd;
                    if (!S2 && nout > 2) LI(M64, o2 * N + m) -= hd;
                    if (ENERGY) LI(M64, ns * N + m) += q2 * hd;
                };
                col(i0, S2 ? hk * y1 : hk * y1 * y2);
                if (nin > 1) col(i1, S2 ? hk * y0 : hk * y0 * y2);
                if (!S2 && nin > 2) col(i2, hk * (y0 * y1));
                if (ENERGY) {
                    const double dkh = hph * (k * (t.b[r] + t.th[r] * invT) * invT);
                    col(ns, S2 ? dkh * (y0 * y1) : dkh * (y0 * y1) * y2);
                }
            }
            if (MODE == 2 && doJ && dist) {
                const float kf = static_cast<float>(k);
                const float f0 = static_cast<float>(y0), f1 = static_cast<float>(y1);
                const float d2 = ENERGY ? kf * (t.bf[r] + t.thf[r] * invTf) *
                                              invTf * (f0 * f1)
                                        : 0.0f;
                scatter22<float, 6, ENERGY>(J32, N, ns, i0, i1, o0, o1, kf * f1, kf * f0, d2,
                                            ENERGY ? t.dHf[r] * invCVf : 0.0f, -1.0f);
            } else if (MODE == 2 && doJ) {
                const float kf = static_cast<float>(k);
                const float f0 = static_cast<float>(y0), f1 = static_cast<float>(y1),
                            f2 = static_cast<float>(y2);
                const float qf = ENERGY ? t.dHf[r] * invCVf : 0.0f;
                auto col = [&](int m, float d) {
                    LIS(J32, i0 * N + m, 6) -= d;
                    if (nin > 1) LIS(J32, i1 * N + m, 6) -= d;
                    if (!S2 && nin > 2) LIS(J32, i2 * N + m, 6) -= d;
                    if (nout > 0) LIS(J32, o0 * N + m, 6) += d;
                    if (nout > 1) LIS(J32, o1 * N + m, 6) += d;
                    if (!S2 && nout > 2) LIS(J32, o2 * N + m, 6) += d;
                    if (ENERGY) LIS(J32, ns * N + m, 6) -= qf * d;
                };
                col(i0, S2 ? kf * f1 : kf * f1 * f2);
                if (nin > 1) col(i1, S2 ? kf * f0 : kf * f0 * f2);
                if (!S2 && nin > 2) col(i2, kf * f0 * f1);
                if (ENERGY) {
                    const float dw = kf * (t.bf[r] + t.thf[r] * invTf) *
                                     invTf * (f0 * f1);
                    col(ns, S2 ? dw : dw * f2);
                }
            }
            if (MODE == 3 && doJ && dist) {
                // I - h J in FP32: reactant rows + h dw/dy_c, product rows - h dw/dy_c,
                // the T row + (dH_r / C_V) h dw/dy_c
                const float hk = hf * static_cast<float>(k);
                const float f0 = static_cast<float>(y0), f1 = static_cast<float>(y1);
                const float d2 = ENERGY ? hk * (t.bf[r] + t.thf[r] * invTf) *
                                              invTf * (f0 * f1)
                                        : 0.0f;
                scatter22<float, 5, ENERGY>(J32, N, ns, i0, i1, o0, o1, hk * f1, hk * f0, d2,
                                            ENERGY ? t.dHf[r] * invCVf : 0.0f, 1.0f);
            } else if (MODE == 3 && doJ) {
                const float hk = hf * static_cast<float>(k);
                const float f0 = static_cast<float>(y0), f1 = static_cast<float>(y1),
                            f2 = static_cast<float>(y2);
                const float qf = ENERGY ? t.dHf[r] * invCVf : 0.0f;
                auto col = [&](int m, float d) {
                    LIS(J32, i0 * N + m, 5) += d;
                    if (nin > 1) LIS(J32, i1 * N + m, 5) += d;
                    if (!S2 && nin > 2) LIS(J32, i2 * N + m, 5) += d;
                    if (nout > 0) LIS(J32, o0 * N + m, 5) -= d;
                    if (nout > 1) LIS(J32, o1 * N + m, 5) -= d;
                    if (!S2 && nout > 2) LIS(J32, o2 * N + m, 5) -= d;
                    if (ENERGY) LIS(J32, ns * N + m, 5) += qf * d;
                };
                col(i0, S2 ? hk * f1 : hk * f1 * f2);
                if (nin > 1) col(i1, S2 ? hk * f0 : hk * f0 * f2);
                if (!S2 && nin > 2) col(i2, hk * f0 * f1);
                if (ENERGY) {
                    const float dw = hk * (t.bf[r] + t.thf[r] * invTf) *
                                     invTf * (f0 * f1);
                    col(ns, S2 ? dw : dw * f2);
                }
            }
        }
    }
    if (ENERGY) LI(W, ns) = fT * invCV;
    if (MODE == 1) {
        for (int i = 0; i < N; ++i) LI(M64, i * N + i) += 1.0;
    }
    if (MODE == 3 && doJ) {
        for (int i = 0; i < N; ++i) LIS(J32, i * N + i, 5) += 1.0f;
    }
}

// Crout LU with implicit-scaled row pivoting (Algorithm lu-decomp).  V holds the
// inverse row maxima, then the inverse pivots (used by the back substitution).
// Returns false on a zero row or a zero pivot.  T is double or float.
template <typename T, int SH>
__device__ __forceinline__ bool crout_lu(T *M, T *V, int *P, int N)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T big = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T a = LIS(M, i * N + j, SH);
            big = a < T(0) ? (-a > big ? -a : big) : (a > big ? a : big);
        }
        ok = ok && (big > T(0));
        LIS(V, i, SH) = big > T(0) ? T(1) / big : T(1);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int kmax = i < j ? i : j;
            T s = LIS(M, i * N + j, SH);
#pragma unroll
            for (int k = 0; k < kmax; ++k) s -= LIS(M, i * N + k, SH) * LIS(M, k * N + j, SH);
            LIS(M, i * N + j, SH) = s;
        }
        int imax = j;
        T tmax = fabs(LIS(M, j * N + j, SH)) * LIS(V, j, SH);
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            const T tt = fabs(LIS(M, i * N + j, SH)) * LIS(V, i, SH);
            if (tt > tmax) {
                tmax = tt;
                imax = i;
            }
        }
        ok = ok && (tmax > T(0));
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T a = LIS(M, imax * N + k, SH), b = LIS(M, j * N + k, SH);
            LIS(M, imax * N + k, SH) = b;
            LIS(M, j * N + k, SH) = a;
        }
        const T va = LIS(V, imax, SH);
        LIS(V, imax, SH) = LIS(V, j, SH);
        LIS(V, j, SH) = va;
        LI(P, j) = imax;
        const T rinv = T(1) / LIS(M, j * N + j, SH);
#pragma unroll
        for (int i = j + 1; i < N; ++i) LIS(M, i * N + j, SH) *= rinv;
        LIS(V, j, SH) = rinv;
    }
    return ok;
}

// Solve with the factors: row swaps in order, unit-lower forward, upper backward.
template <typename T, int SH>
__device__ __forceinline__ void crout_solve(const T *M, const T *V, const int *P, T *x, int N)
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int p = LI(P, i);
        const T a = LIS(x, i, SH), b = LIS(x, p, SH);
        LIS(x, i, SH) = b;
        LIS(x, p, SH) = a;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T s = LIS(x, i, SH);
#pragma unroll
        for (int k = 0; k < i; ++k) s -= LIS(M, i * N + k, SH) * LIS(x, k, SH);
        LIS(x, i, SH) = s;
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        T s = LIS(x, i, SH);
#pragma unroll
        for (int k = i + 1; k < N; ++k) s -= LIS(M, i * N + k, SH) * LIS(x, k, SH);
        LIS(x, i, SH) = s * LIS(V, i, SH);
    }
}

// Crout LU of the lean layout: the same steps and operation order as crout_lu<float>
// at lane stride 32, with the inverse pivots stored on the diagonal (U's diagonal is
// not read again once its column is done), the row scales V in a scratch area and one
// pivot byte per row.  Returns false on a zero row or a zero pivot.
template <int NT>
__device__ __forceinline__ bool crout_lu_lean(float *M, float *V, unsigned char *P)
{
    constexpr int N = NT;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float big = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float a = LIS(M, i * N + j, 5);
            big = a < 0.0f ? (-a > big ? -a : big) : (a > big ? a : big);
        }
        ok = ok && (big > 0.0f);
        LIS(V, i, 5) = big > 0.0f ? 1.0f / big : 1.0f;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int kmax = i < j ? i : j;
            float s = LIS(M, i * N + j, 5);
#pragma unroll
            for (int k = 0; k < kmax; ++k) s -= LIS(M, i * N + k, 5) * LIS(M, k * N + j, 5);
            LIS(M, i * N + j, 5) = s;
        }
        int imax = j;
        float tmax = fabsf(LIS(M, j * N + j, 5)) * LIS(V, j, 5);
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            const float tt = fabsf(LIS(M, i * N + j, 5)) * LIS(V, i, 5);
            if (tt > tmax) {
                tmax = tt;
                imax = i;
            }
        }
        ok = ok && (tmax > 0.0f);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float a = LIS(M, imax * N + k, 5), b = LIS(M, j * N + k, 5);
            LIS(M, imax * N + k, 5) = b;
            LIS(M, j * N + k, 5) = a;
        }
        const float va = LIS(V, imax, 5);
        LIS(V, imax, 5) = LIS(V, j, 5);
        LIS(V, j, 5) = va;
        LIS(P, j, 5) = static_cast<unsigned char>(imax);
        const float rinv = 1.0f / LIS(M, j * N + j, 5);
#pragma unroll
        for (int i = j + 1; i < N; ++i) LIS(M, i * N + j, 5) *= rinv;
        LIS(M, j * N + j, 5) = rinv;
    }
    return ok;
}

// Solve with the lean factors, the right-hand side in registers: the row swaps in
// order (as selects, so every index stays a compile-time constant), unit-lower forward,
// upper backward times the stored inverse pivot.
template <int NT>
__device__ __forceinline__ void crout_solve_lean(const float *M, const unsigned char *P, float (&x)[NT])
{
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const int p = LIS(P, i, 5);
#pragma unroll
        for (int k = i + 1; k < NT; ++k) {
            if (k == p) {
                const float t = x[i];
                x[i] = x[k];
                x[k] = t;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        float s = x[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= LIS(M, i * NT + k, 5) * x[k];
        x[i] = s;
    }
#pragma unroll
    for (int i = NT - 1; i >= 0; --i) {
        float s = x[i];
#pragma unroll
        for (int k = i + 1; k < NT; ++k) s -= LIS(M, i * NT + k, 5) * x[k];
        x[i] = s * LIS(M, i * NT + i, 5);
    }
}

template <int NT, bool ENERGY, bool F32, bool PERSIST, bool MLPG, bool LEAN>
__global__ void __launch_bounds__(kMaxWarps * 32, 1) lane_kernel(const LaunchArgs a, const LaneLayout L)
{
    static_assert(!LEAN || (F32 && NT > 0 && !MLPG), "the lean layout is an FP32-LU, fixed-size variant");
    constexpr int NR = LEAN ? NT : 1;   // register vectors of the lean layout
    extern __shared__ __align__(16) unsigned char sm[];
    const NetView nv = a.nv;
    if (!stage_table(sm, a.blob, static_cast<unsigned>(nv.bytes),
                     reinterpret_cast<uint64_t *>(sm + nv.bytes), &a.scratch->error, kDevErrTma))
        return;
    const unsigned char *mlpP = sm + L.mlp_off;
    if (MLPG && !stage_table(sm + L.mlp_off, a.mlp, static_cast<unsigned>(MlpLayout::BYTES),
                             reinterpret_cast<uint64_t *>(sm + nv.bytes + 8), &a.scratch->error, kDevErrTma))
        return;
    const NetSmem t = net_smem(sm, nv);
    const DevOpts o = a.o;
    // N = ns + 1 with the energy equation, else ns
    const int N = NT > 0 ? NT : nv.N, ns = LEAN ? NT - (ENERGY ? 1 : 0) : nv.ns, ne = nv.ne, nr = nv.nr;
    const long long nc = a.ncells;
    const int lane = threadIdx.x & 31;
    unsigned char *wb = sm + L.base + (threadIdx.x >> 5) * L.warp_bytes;
    // y_n (Y) and f_n (FY): registers in the lean layout, shared memory otherwise
    LaneVec<LEAN, NR> Y, FY;
    Y.p = LEAN ? nullptr : reinterpret_cast<double *>(wb + L.off_Y) + lane;
    FY.p = LEAN ? nullptr : reinterpret_cast<double *>(wb + L.off_FY) + lane;
    double *YF = reinterpret_cast<double *>(wb + L.off_YF) + lane;
    double *YH = reinterpret_cast<double *>(wb + L.off_YH) + lane;
    double *Y2 = reinterpret_cast<double *>(wb + L.off_Y2) + lane;
    double *W = reinterpret_cast<double *>(wb + L.off_W) + lane;
    const bool s2 = nv.shape == 22;   // every reaction A + B -> C + D
    int *P = LEAN ? nullptr : reinterpret_cast<int *>(wb + L.off_P) + lane;
    // lean layout: FP32 matrix at lane stride 32, row scales over the rate slots, pivot bytes
    float *ML = LEAN ? reinterpret_cast<float *>(wb + L.off_M) + lane : nullptr;
    float *VL = LEAN ? reinterpret_cast<float *>(wb + L.off_W) + lane : nullptr;
    unsigned char *PL = LEAN ? wb + L.off_P + lane : nullptr;
    double *K = ENERGY ? nullptr : reinterpret_cast<double *>(wb + L.off_K) + lane;
    // C_V(T) of polynomial networks (Sec. 4.2): the cell's coefficients sum_s n0_s c_s,k,
    // five below t_mid then five from t_mid
    const bool CVP = ENERGY && nv.cvpoly != 0;
    double *CV = CVP ? reinterpret_cast<double *>(wb + L.off_CV) + lane : nullptr;
    const double *cvp = reinterpret_cast<const double *>(sm + nv.off_cvp);
    // FP64 matrix and scales; in the FP32 form they overlay the lane's own J32/M32 and
    // V32/X32 slots and serve the FP64 rescue of a failed FP32 solve
    double *M64 = LEAN ? nullptr : reinterpret_cast<double *>(wb + L.off_M) + lane;
    double *V64 = LEAN ? nullptr : reinterpret_cast<double *>(wb + L.off_V) + lane;
    float *J32 = nullptr, *M32 = nullptr, *V32 = nullptr, *X32 = nullptr;
    if (F32 && !LEAN) {
        J32 = reinterpret_cast<float *>(wb + L.off_J) + 2 * lane;
        M32 = J32 + 1;
        V32 = reinterpret_cast<float *>(wb + L.off_V) + 2 * lane;
        X32 = V32 + 1;
    }

    // ---- per-lane state
    int state = kNeed;
    long long cell = -1;
    if (!PERSIST) {
        cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
        if (cell >= nc) state = kDone;
    }
    double tt = 0.0, h = 0.0, facmax = 0.0, T_iso = 0.0, invCV = 0.0, atol_s = 0.0, dtc = a.dt;
    int phase = 0, it = 0, natt = 0, nacc = 0, nnew = 0, attempt = 0;
    bool last = false;
    // FP32 form: needJ -> assemble J32 at the current iterate; needF -> factorise;
    // rescue -> this solve runs full FP64 Newton from its starting guess
    bool needJ = false, needF = false, luok = true, rescue = false;
    int refresh = 0;
    float dprev = 0.0f, dprevr = 0.0f;
    // FP32 form caches: atY -> the current solve's iterate is the attempt's start
    // state Y (bit for bit); fyok -> FY holds f(Y); jY -> J32 holds J(Y).  Phase 1
    // starts from Y like phase 0, and a rejected attempt restarts from the same Y, so
    // these passes reuse f(Y) (and J(Y)) instead of recomputing them.
    bool atY = false, fyok = false, jY = false;
    // learned guess: needG -> the attempt's first solve wants the MLP's starting point;
    // usedG -> the current solve started from it (fall back to the plain start on failure)
    bool needG = false, usedG = false;
    double rho_c = 1.0;

    auto finish = [&]() { state = PERSIST ? kNeed : kDone; };

    // TR-BDF2 (o.scheme == KT_SCHEME_TRBDF2, uniform over the launch): phase 0 is the
    // trapezoidal stage (iterate YF), phase 1 the BDF2 stage (iterate Y2); YH holds the
    // stage's right-hand side r and FY the rate f_n of the step's start state: evaluated
    // on the cell's first step, afterwards the previous step's stage relation
    // f_{n+1} = (y_{n+1} - r)/(d h) (an evaluated f(y_n) would enter the error estimate
    // multiplied by h, which turns its rounding into noise in err on stiff components).
    const bool TR = LEAN || o.scheme == KT_SCHEME_TRBDF2;
    const TrCoef tr = tr_coef();

    // Pre-processing (Sec. 2.2.2): floors y >= 0 and T clamped to [t_min, t_max].
    auto load_pre = [&]() {
        fyok = false;
        jY = false;
#pragma unroll
        for (int s = 0; s < ns; ++s) {
            const double v = a.y_in[static_cast<long long>(s) * nc + cell];
            Y[s] = v > 0.0 ? v : 0.0;
        }
        const double Tin = a.T_in[cell];
        const double T0 = Tin < nv.t_min ? nv.t_min : (Tin > nv.t_max ? nv.t_max : Tin);
        T_iso = T0;
        if (ENERGY) Y[ns] = T0;
    };

    auto write_out = [&](int st) {
#pragma unroll
        for (int s = 0; s < ns; ++s) a.y_out[static_cast<long long>(s) * nc + cell] = Y[s];
        a.T_out[cell] = ENERGY ? Y[ns] : T_iso;
        if (a.status) a.status[cell] = st;
        if (a.nsub) a.nsub[cell] = st == KT_STATUS_REVERTED ? 0 : nacc;
        if (a.nnew) a.nnew[cell] = nnew;
    };

    auto begin_attempt = [&]() -> bool {
        if (natt >= o.max_substeps) return false;
        ++natt;
        last = false;
        if (tt + h >= dtc * (1.0 - 1e-12)) {
            h = dtc - tt;
            last = true;
        }
        phase = 0;
        it = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) LI(YF, i) = Y[i];
        atY = true;
        if (F32) {
            needJ = true;
            needF = true;
            refresh = 0;
            rescue = false;
        }
        needG = MLPG && o.guess == KT_GUESS_MLP;
        usedG = false;
        return true;
    };

    auto start_run = [&](double h0, double fmax) -> bool {
        tt = 0.0;
        h = h0;
        facmax = fmax;
        natt = 0;
        nacc = 0;
        return begin_attempt();
    };

    // A failed run: retry once from the pre-processed input with a smaller first step
    // and gentler growth, else revert to the pre-processed input (Sec. 2.2.3).
    auto run_fail = [&]() {
        if (attempt == 0 && o.retry) {
            attempt = 1;
            load_pre();
            if (start_run(o.h_init * o.retry_h_factor, o.retry_facmax)) return;
        }
        load_pre();
        write_out(KT_STATUS_REVERTED);
        finish();
    };

    // Post-processing (Sec. 2.2.3): clip negatives, then restore the element totals b0
    // of the pre-processed input by y_s -= y_s (N^T lambda)_s with
    // (N diag(y) N^T) lambda = N y - b0.
    auto post_process = [&]() -> bool {
        double b0[kMaxElements], r[kMaxElements], Mp[kMaxElements * kMaxElements];
        for (int e = 0; e < ne; ++e) b0[e] = 0.0;
        for (int s = 0; s < ns; ++s) {
            const double v = a.y_in[static_cast<long long>(s) * nc + cell];
            const double y0 = v > 0.0 ? v : 0.0;
            for (int e = 0; e < ne; ++e) b0[e] += t.cnt[s * ne + e] * y0;
        }
#pragma unroll
        for (int s = 0; s < ns; ++s)
            if (Y[s] < 0.0) Y[s] = 0.0;
        for (int e = 0; e < ne; ++e) {
            double tot = 0.0;
#pragma unroll
            for (int s = 0; s < ns; ++s) tot += t.cnt[s * ne + e] * Y[s];
            r[e] = tot - b0[e];
            for (int f = 0; f < ne; ++f) {
                double m = 0.0;
#pragma unroll
                for (int s = 0; s < ns; ++s) m += t.cnt[s * ne + e] * t.cnt[s * ne + f] * Y[s];
                Mp[e * ne + f] = m;
            }
        }
        for (int e = 0; e < ne; ++e) {
            if (Mp[e * ne + e] == 0.0) {
                if (r[e] != 0.0) return false;
                for (int f = 0; f < ne; ++f) Mp[e * ne + f] = Mp[f * ne + e] = 0.0;
                Mp[e * ne + e] = 1.0;
            }
        }
        for (int k = 0; k < ne; ++k) {   // Gaussian elimination, partial pivoting
            int p = k;
            for (int i = k + 1; i < ne; ++i)
                if (fabs(Mp[i * ne + k]) > fabs(Mp[p * ne + k])) p = i;
            if (!(fabs(Mp[p * ne + k]) > 0.0)) return false;
            if (p != k) {
                for (int j = 0; j < ne; ++j) {
                    const double x = Mp[k * ne + j];
                    Mp[k * ne + j] = Mp[p * ne + j];
                    Mp[p * ne + j] = x;
                }
                const double x = r[k];
                r[k] = r[p];
                r[p] = x;
            }
            for (int i = k + 1; i < ne; ++i) {
                const double l = Mp[i * ne + k] / Mp[k * ne + k];
                for (int j = k; j < ne; ++j) Mp[i * ne + j] -= l * Mp[k * ne + j];
                r[i] -= l * r[k];
            }
        }
        for (int i = ne - 1; i >= 0; --i) {
            double s = r[i];
            for (int j = i + 1; j < ne; ++j) s -= Mp[i * ne + j] * r[j];
            r[i] = s / Mp[i * ne + i];
        }
        bool ok = true;
#pragma unroll
        for (int s = 0; s < ns; ++s) {
            double corr = 0.0;
            for (int e = 0; e < ne; ++e) corr += t.cnt[s * ne + e] * r[e];
            ok = ok && (corr < 1.0);
            Y[s] -= Y[s] * corr;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) ok = ok && isfinite(Y[i]);
        return ok;
    };

    auto begin_cell = [&]() {
        dtc = a.dt_cell ? a.dt_cell[cell] : a.dt;
        rho_c = a.rho ? a.rho[cell] : 1.0;
        bool fin = isfinite(a.T_in[cell]) && dtc > 0.0 && isfinite(dtc);
        for (int s = 0; s < ns; ++s) fin = fin && isfinite(a.y_in[static_cast<long long>(s) * nc + cell]);
        if (!fin) {
            for (int s = 0; s < ns; ++s)
                a.y_out[static_cast<long long>(s) * nc + cell] = a.y_in[static_cast<long long>(s) * nc + cell];
            a.T_out[cell] = a.T_in[cell];
            if (a.status) a.status[cell] = KT_STATUS_NONFINITE;
            if (a.nsub) a.nsub[cell] = 0;
            if (a.nnew) a.nnew[cell] = 0;
            finish();
            return;
        }
        load_pre();
        double cvt = 0.0, b00 = 0.0;
#pragma unroll
        for (int s = 0; s < ns; ++s) {
            cvt += t.cv[s] * Y[s];
            b00 += t.cnt[s * ne] * Y[s];
        }
        invCV = ENERGY ? 1.0 / cvt : 0.0;
        if (CVP) {
            for (int k = 0; k < 10; ++k) {
                double c = 0.0;
#pragma unroll
                for (int s = 0; s < ns; ++s) c += Y[s] * cvp[s * 10 + k];
                LI(CV, k) = c;
            }
        }
        atol_s = (o.atol_mode == 1 && b00 > 0.0) ? o.atol * b00 : o.atol;
        if (!ENERGY) {
            const double lt = log_t(T_iso, nv.t_ref), invT = 1.0 / T_iso;
            for (int r = 0; r < nr; ++r) {
                double k, dk;
                arrhenius(t, r, lt, invT, k, dk);
                LI(K, r) = k;
            }
        }
        attempt = 0;
        nnew = 0;
        state = kRun;
        if (!start_run(o.h_init, o.facmax)) run_fail();
    };

    auto step_fail_newton = [&]() {
        h *= 0.5;
        if (h < o.h_min || !begin_attempt()) run_fail();
    };

    // starting point of the current solve (plain predictor / second half from the full step)
    auto restart_solve = [&]() {
        if (TR) {
            if (phase == 0) {
#pragma unroll
                for (int i = 0; i < N; ++i) LI(YF, i) = Y[i];
            } else {
                for (int i = 0; i < N; ++i) LI(Y2, i) = LI(YF, i);
            }
            atY = phase == 0;
            it = 0;
            return;
        }
        double *yt = phase == 0 ? YF : (phase == 1 ? YH : Y2);
        const double *g = phase == 2 ? (o.guess != KT_GUESS_PREV ? YF : YH) : Y.p;
        for (int i = 0; i < N; ++i) LI(yt, i) = LI(g, i);
        atY = phase != 2;
        it = 0;
    };

    // Newton did not converge: a solve that started from the learned guess restarts from
    // the plain predictor; an FP32 solve is redone in FP64; otherwise h halves.
    auto newton_fail = [&]() {
        if (usedG) {
            usedG = false;
            restart_solve();
            if (F32) {
                needJ = true;
                needF = true;
                refresh = 0;
                rescue = false;
            }
            return;
        }
        if (F32 && !LEAN && !rescue) {
            rescue = true;
            atomicAdd(&a.scratch->rescues, 1u);
            restart_solve();
            return;
        }
        step_fail_newton();
    };

    auto step_done = [&]() {
        // weighted RMS of the step-doubling difference
        double s2 = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double y = Y[i], y2 = LI(Y2, i);
            const double sc = (i < ns ? atol_s : 0.0) + o.rtol * fmax(fabs(y), fabs(y2));
            const double e = (y2 - LI(YF, i)) / sc;
            s2 += e * e;
        }
        const double err = sqrt(s2 / N);
        if (err <= 1.0) {
#pragma unroll
            for (int i = 0; i < N; ++i) Y[i] = LI(Y2, i);
            fyok = false;
            jY = false;
            ++nacc;
            if (last) {
                if (post_process()) {
                    write_out(attempt == 0 ? KT_STATUS_OK : KT_STATUS_RETRIED);
                    finish();
                } else {
                    run_fail();
                }
                return;
            }
            tt += h;
            double fac = err > 0.0 ? 0.9 / sqrt(err) : facmax;
            if (fac > facmax) fac = facmax;
            if (fac < 0.2) fac = 0.2;
            h *= fac;
            if (!begin_attempt()) run_fail();
        } else {
            double fac = 0.9 / sqrt(err);
            if (!(fac >= 0.2)) fac = 0.2;
            h *= fac;
            if (h < o.h_min || !begin_attempt()) run_fail();
        }
    };

    // end of a TR-BDF2 step: weighted RMS of the local error estimate, then accept
    // (growth 0.9 err^(-1/3)) or reject
    auto step_done_tr = [&]() {
        const double dh = tr.d * h, inv = 1.0 / dh, ce = 2.0 * tr.C * h;
        double s2 = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double yn = Y[i], y1 = LI(Y2, i), f0 = FY[i];
            const double fg = (LI(YF, i) - yn) * inv - f0;
            const double f1 = (y1 - LI(YH, i)) * inv;
            const double est = ce * (tr.a0 * f0 + tr.a1 * fg + tr.a2 * f1);
            const double sc = (i < ns ? atol_s : 0.0) + o.rtol * fmax(fabs(yn), fabs(y1));
            const double e = est / sc;
            s2 += e * e;
        }
        const double err = sqrt(s2 / N);
        if (err <= 1.0) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                FY[i] = (LI(Y2, i) - LI(YH, i)) * inv;   // first same as last
                Y[i] = LI(Y2, i);
            }
            fyok = true;
            jY = false;
            ++nacc;
            if (last) {
                if (post_process()) {
                    write_out(attempt == 0 ? KT_STATUS_OK : KT_STATUS_RETRIED);
                    finish();
                } else {
                    run_fail();
                }
                return;
            }
            tt += h;
            double fac = err > 0.0 ? 0.9 / cbrt(err) : facmax;
            if (fac > facmax) fac = facmax;
            if (fac < 0.2) fac = 0.2;
            h *= fac;
            if (!begin_attempt()) run_fail();
        } else {
            double fac = 0.9 / cbrt(err);
            if (!(fac >= 0.2)) fac = 0.2;
            h *= fac;
            if (h < o.h_min || !begin_attempt()) run_fail();
        }
    };

    auto phase_done = [&]() {
        usedG = false;
        if (F32 && rescue) {      // the FP64 rescue overwrote the FP32 factors
            rescue = false;
            needJ = true;
            needF = true;
            refresh = 0;
        }
        if (TR) {
            if (phase == 0) {       // BDF2 stage: r = w1 y_g - w0 y_n, start from y_g
                phase = 1;
                it = 0;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    LI(YH, i) = tr.w1 * LI(YF, i) - tr.w0 * Y[i];
                    LI(Y2, i) = LI(YF, i);
                }
                atY = false;
            } else {
                step_done_tr();
            }
            return;
        }
        if (phase == 0) {
            phase = 1;
            it = 0;
#pragma unroll
            for (int i = 0; i < N; ++i) LI(YH, i) = Y[i];
            atY = true;
            if (F32) { needF = true; }
        } else if (phase == 1) {
            phase = 2;
            it = 0;
            const double *g2 = o.guess != KT_GUESS_PREV ? YF : YH;
            for (int i = 0; i < N; ++i) LI(Y2, i) = LI(g2, i);
            atY = false;
        } else {
            step_done();
        }
    };

    const double natol_frac = o.newton_atol_frac;
    for (;;) {
        // ---- give every idle lane a cell
        for (;;) {
            const bool want = state == kNeed;
            if (PERSIST) {
                const unsigned m = __ballot_sync(kFull, want);
                if (!m) break;
                const int leader = __ffs(m) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&a.scratch->queue, static_cast<unsigned long long>(__popc(m)));
                base = __shfl_sync(kFull, base, leader);
                if (want) {
                    const long long q = static_cast<long long>(base + __popc(m & ((1u << lane) - 1u)));
                    if (q >= nc) {
                        state = kDone;
                    } else {
                        cell = a.order ? static_cast<long long>(a.order[q]) : q;
                        begin_cell();
                    }
                }
            } else {
                if (!__any_sync(kFull, want)) break;
                if (want) begin_cell();
            }
        }
        if (__all_sync(kFull, state == kDone)) break;

        // ---- learned starting point for lanes that begin an attempt (warp-wide MMA)
        if (MLPG) {
            const bool wantG = state == kRun && needG;
            if (__any_sync(kFull, wantG)) {
                const float *nrm = reinterpret_cast<const float *>(mlpP + MlpLayout::NORM);
                float x[kMlpIn];
#pragma unroll
                for (int k = 0; k < kMlpIn; ++k) x[k] = 0.0f;
                if (wantG) {
                    for (int k = 0; k < ns && k < kMlpIn; ++k)
                        x[k] = static_cast<float>((log(fmax(Y[k], 1e-30)) - nrm[k]) / nrm[16 + k]);
                    const double Tc = ENERGY ? Y[ns] : T_iso;
                    const double f3[3] = {log(Tc), log(rho_c), log(h)};
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int k = ns + q;
                        if (k < kMlpIn) x[k] = static_cast<float>((f3[q] - nrm[k]) / nrm[16 + k]);
                    }
                }
                uint32_t af[1][4];
                float dlo[kMlpOutTiles][4], dhi[kMlpOutTiles][4];
                gather_a(x, a.mlp_nin, 0, lane, af);
                mlp_forward16(mlpP, af, dlo, lane);
                gather_a(x, a.mlp_nin, 16, lane, af);
                mlp_forward16(mlpP, af, dhi, lane);
                float outv[kMlpOut];
#pragma unroll
                for (int q = 0; q < kMlpOut; ++q) {
                    const float vlo = scatter_out(dlo, q, 0, lane);
                    const float vhi = scatter_out(dhi, q, 16, lane);
                    outv[q] = lane < 16 ? vlo : vhi;
                }
                if (wantG) {
                    for (int i = 0; i < N && i < kMlpOut; ++i) {
                        const double dlog = nrm[32 + i] + nrm[48 + i] * static_cast<double>(outv[i]);
                        const double base = i < ns ? fmax(Y[i], 1e-30) : Y[i];
                        const double g = base * exp(fmin(dlog, 50.0));
                        LI(YF, i) = isfinite(g) ? g : Y[i];
                    }
                    needG = false;
                    usedG = true;
                    atY = false;
                }
            }
        }
        if (state != kRun) continue;

        // ---- one Newton iteration of the current backward-Euler solve
        const double *yb = TR ? YH : (phase == 2 ? YH : Y.p);
        double *yt = TR ? (phase == 0 ? YF : Y2) : (phase == 0 ? YF : (phase == 1 ? YH : Y2));
        const double hph = TR ? tr.d * h : (phase == 0 ? h : 0.5 * h);
        // TR-BDF2 stage 1 at its first iterate (y_n itself): f(y_n) -> FY, r1 = y_n + d h f(y_n)
        const bool trF0 = TR && phase == 0 && atY;
        ++nnew;
        const double T = ENERGY ? LI(yt, ns) : T_iso;
        const bool bad = !(T > 0.0);
        double lt = 0.0, invT = 0.0, invCVi = invCV, dcvr = 0.0;
        if (ENERGY) {
            const double Ts = bad ? 1.0 : T;
            lt = log_t(Ts, nv.t_ref);
            invT = 1.0 / Ts;
            if (CVP) {
                // C_V(T) and C_V'(T)/C_V(T) at this iterate (Horner in the range of T)
                const int o5 = Ts < nv.t_mid ? 5 : 0;
                const double c0 = LI(CV, 5 - o5), c1 = LI(CV, 6 - o5), c2 = LI(CV, 7 - o5),
                             c3 = LI(CV, 8 - o5), c4 = LI(CV, 9 - o5);
                const double cv = (((c4 * Ts + c3) * Ts + c2) * Ts + c1) * Ts + c0;
                const double dcv = ((4.0 * c4 * Ts + 3.0 * c3) * Ts + 2.0 * c2) * Ts + c1;
                invCVi = 1.0 / cv;
                dcvr = dcv * invCVi;
            }
        }
        float xr[NR];   // lean layout: the FP32 residual, then the Newton update
        if (!F32 || (!LEAN && rescue)) {
            if (s2)
                reaction_pass<NT, ENERGY, 1, true>(nv, t, yt, K, lt, invT, invCVi, hph, W, M64, nullptr, false);
            else
                reaction_pass<NT, ENERGY, 1, false>(nv, t, yt, K, lt, invT, invCVi, hph, W, M64, nullptr, false);
            // d f_T / d T of C_V(T): -f_T C_V'/C_V, i.e. +h f_T C_V'/C_V in I - h J
            if (CVP) LI(M64, ns * N + ns) += hph * LI(W, ns) * dcvr;
            if (F32) jY = false;   // the FP64 matrix overlays the FP32 Jacobian
            if (trF0) {
                if (!fyok) {
#pragma unroll
                    for (int i = 0; i < N; ++i) FY[i] = LI(W, i);
                    fyok = true;
                }
#pragma unroll
                for (int i = 0; i < N; ++i) LI(YH, i) = Y[i] + hph * FY[i];
            }
            for (int i = 0; i < N; ++i) LI(W, i) = -(LI(yt, i) - LI(yb, i) - hph * LI(W, i));
            luok = crout_lu<double, 5>(M64, V64, P, N);
            crout_solve<double, 5>(M64, V64, P, W, N);
        } else if constexpr (LEAN) {
            // the matrix is assembled at the current iterate whenever it is factorised
            // (the step's start, a refresh): there is no Jacobian copy to re-use
            const bool doM = needF;
            if (s2)
                reaction_pass<NT, ENERGY, 3, true>(nv, t, yt, K, lt, invT, invCVi, hph, W, nullptr, ML, doM);
            else
                reaction_pass<NT, ENERGY, 3, false>(nv, t, yt, K, lt, invT, invCVi, hph, W, nullptr, ML, doM);
            if (CVP && doM) LIS(ML, ns * N + ns, 5) += static_cast<float>(hph * LI(W, ns) * dcvr);
            if (atY && !fyok) {
#pragma unroll
                for (int i = 0; i < N; ++i) FY[i] = LI(W, i);
                fyok = true;
            }
            if (trF0) {
#pragma unroll
                for (int i = 0; i < N; ++i) LI(YH, i) = Y[i] + hph * FY[i];
            }
            // residual before the factorisation: the row scales reuse the rate slots
#pragma unroll
            for (int i = 0; i < N; ++i) xr[i] = static_cast<float>(-(LI(yt, i) - LI(YH, i) - hph * LI(W, i)));
            if (doM) {
                luok = crout_lu_lean<NT>(ML, VL, PL);
                needF = false;
            }
            needJ = false;
            crout_solve_lean<NT>(ML, PL, xr);
        } else {
            const bool doJ = needJ && !(atY && jY);
            if (atY && fyok && !doJ) {
#pragma unroll
                for (int i = 0; i < N; ++i) LI(W, i) = FY[i];
            } else {
                if (s2)
                    reaction_pass<NT, ENERGY, 2, true>(nv, t, yt, K, lt, invT, invCVi, hph, W, nullptr, J32, doJ);
                else
                    reaction_pass<NT, ENERGY, 2, false>(nv, t, yt, K, lt, invT, invCVi, hph, W, nullptr, J32, doJ);
                if (CVP && doJ) LIS(J32, ns * N + ns, 6) -= static_cast<float>(LI(W, ns) * dcvr);
                if (atY && !(TR && fyok)) {
#pragma unroll
                    for (int i = 0; i < N; ++i) FY[i] = LI(W, i);
                    fyok = true;
                }
                if (doJ) jY = atY;
            }
            if (trF0) {
#pragma unroll
                for (int i = 0; i < N; ++i) LI(YH, i) = Y[i] + hph * FY[i];
            }
            if (needF) {
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < N; ++j)
                        LIS(M32, i * N + j, 6) =
                            (i == j ? 1.0f : 0.0f) - static_cast<float>(hph) * LIS(J32, i * N + j, 6);
                luok = crout_lu<float, 6>(M32, V32, P, N);
                needF = false;
            }
            needJ = false;
            for (int i = 0; i < N; ++i)
                LIS(X32, i, 6) = static_cast<float>(-(LI(yt, i) - LI(yb, i) - hph * LI(W, i)));
            crout_solve<float, 6>(M32, V32, P, X32, N);
            for (int i = 0; i < N; ++i) LI(W, i) = static_cast<double>(LIS(X32, i, 6));
        }
        bool conv = !bad && luok;
        // contraction monitors of the FP32 form (FP32 is plenty): dmax = max |delta|/tol,
        // dmaxr = max |delta| / (newton_rtol |y|), the purely relative part
        float dmax = 0.0f, dmaxr = 0.0f;
        const double natol = (F32 ? natol_frac * kF32NewtonAtolScale : natol_frac) * atol_s;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double d = LEAN ? static_cast<double>(xr[i]) : LI(W, i);
            const double y = LI(yt, i) + d;
            LI(yt, i) = y;
            const double tol = (i < ns ? natol : 0.0) + o.newton_rtol * fabs(y);
            if (!(fabs(d) <= tol)) conv = false;
            if (F32) {
                // (lean: |delta| is the FP32 update itself and |y| is rounded once, which
                // spares two conversions and a multiply on the FP64 pipe)
                const float ad = LEAN ? fabsf(xr[i]) : static_cast<float>(fabs(d)), tf = static_cast<float>(tol);
                const float q = __fdiv_rn(ad, fmaxf(tf, 1e-37f));
                // the relative part newton_rtol |y| formed directly: as a difference
                // tf - natol in FP32 it rounds to an ulp of natol for trace species
                const float trl = LEAN ? static_cast<float>(o.newton_rtol) * fabsf(static_cast<float>(y))
                                       : static_cast<float>(o.newton_rtol * fabs(y));
                const float qr = __fdiv_rn(ad, fmaxf(trl, 1e-37f));
                dmax = q > dmax ? q : dmax;
                dmaxr = qr > dmaxr ? qr : dmaxr;
            }
        }
        atY = false;
        // FP32 form: stop on the contraction rate (Hairer & Wanner, Solving ODEs II,
        // Sec. IV.8): with theta = dmaxr / dprevr < 1/2 the error left after this update
        // is about theta / (1 - theta) * |delta|; accept when that is within
        // newton_rtol |y_i| for every component, one iteration before |delta| itself
        // is.  Only the relative part of the tolerance is used, so species below the
        // absolute tolerance still end as close to the root as the plain test leaves them.
        if (F32 && !(!LEAN && rescue) && !conv && !bad && luok && it > 0) {
            const float th = dmaxr / dprevr;
            if (th < 0.5f && th / (1.0f - th) * dmaxr <= 1.0f) conv = true;
        }

        // ---- control
        if (conv) {
            phase_done();
        } else if (!F32 || (!LEAN && rescue)) {
            if (bad || !luok || it + 1 >= o.max_newton) newton_fail();
            else ++it;
        } else {
            // simplified Newton: refresh J (at the current iterate) when the
            // contraction stalls or the iteration budget of this factor is spent
            const bool stalled = it > 0 && !(dmax < 0.5f * dprev);
            if (bad || !luok || !isfinite(dmax)) {
                newton_fail();
            } else if (stalled || it + 1 >= o.max_newton) {
                if (refresh < 2) {
                    ++refresh;
                    needJ = true;
                    needF = true;
                    it = 0;
                } else {
                    newton_fail();
                }
            } else {
                ++it;
            }
            dprev = dmax;
            dprevr = dmaxr;
        }
    }
}

template <int NT, bool ENERGY, bool F32, bool PERSIST, bool MLPG, bool LEAN = false>
int launch_t(const LaunchArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    const LaneLayout L = LEAN ? lane_layout_lean(a.nv.N, a.nv.nr, a.nv.energy, a.nv.bytes, a.nv.cvpoly)
                              : lane_layout(a.nv.N, a.nv.nr, a.nv.energy, F32 ? 1 : 0, a.nv.bytes,
                                            MLPG ? MlpLayout::BYTES : 0, a.nv.cvpoly);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int smem_optin = 0, nsm = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int warps = c.block_warps > 0 ? c.block_warps : kMaxWarps;
    if (warps > kMaxWarps) warps = kMaxWarps;
    while (warps > 1 && L.base + warps * L.warp_bytes > smem_optin) --warps;
    const size_t smem = static_cast<size_t>(L.base) + static_cast<size_t>(warps) * L.warp_bytes;
    if (smem > static_cast<size_t>(smem_optin)) return cudaErrorInvalidConfiguration;
    auto kern = lane_kernel<NT, ENERGY, F32, PERSIST, MLPG, LEAN>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int threads = warps * 32;
    long long blocks;
    if (PERSIST) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        if (c.blocks_per_sm > 0 && c.blocks_per_sm < per_sm) per_sm = c.blocks_per_sm;
        blocks = static_cast<long long>(per_sm) * nsm;
        const long long need = (a.ncells + threads - 1) / threads;
        if (blocks > need) blocks = need;
    } else {
        blocks = (a.ncells + threads - 1) / threads;
    }
    if (blocks < 1) return cudaSuccess;
    kern<<<static_cast<unsigned>(blocks), threads, smem, s>>>(a, L);
    return cudaGetLastError();
}

// Dispatch over the compile-time options for a fixed (or runtime, NT = 0) size and one
// form of the iteration matrix.
template <int NT, bool F32>
int launch_lane_form(const LaunchArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    const bool en = a.nv.energy != 0, per = c.persistent != 0;
    if constexpr (NT == 0 || NT <= kMlpOut) {
        if (a.mlp)   // the learned guess runs with the persistent queue only
            return en ? launch_t<NT, true, F32, true, true>(a, c, s) : launch_t<NT, false, F32, true, true>(a, c, s);
    } else {
        if (a.mlp) return cudaErrorInvalidValue;
    }
    if constexpr (F32 && NT > 0) {
        // TR-BDF2 with a compile-time size: the lean layout unless the caller asks for
        // the Jacobian-caching one
        if (a.o.scheme == KT_SCHEME_TRBDF2 && c.lane_variant != KT_LANE_JCACHE) {
            if (en)
                return per ? launch_t<NT, true, true, true, false, true>(a, c, s)
                           : launch_t<NT, true, true, false, false, true>(a, c, s);
            return per ? launch_t<NT, false, true, true, false, true>(a, c, s)
                       : launch_t<NT, false, true, false, false, true>(a, c, s);
        }
    }
    if (en) return per ? launch_t<NT, true, F32, true, false>(a, c, s) : launch_t<NT, true, F32, false, false>(a, c, s);
    return per ? launch_t<NT, false, F32, true, false>(a, c, s) : launch_t<NT, false, F32, false, false>(a, c, s);
}

}  // namespace

// Launchers of one size (3, 11 or any other N <= 16 as 0) and one form each, every
// one in its own translation unit (compile time).
int launch_lane_n3(const LaunchArgs &a, const LaunchCfg &c, void *stream);
int launch_lane_n11_f64(const LaunchArgs &a, const LaunchCfg &c, void *stream);
int launch_lane_n11_f32(const LaunchArgs &a, const LaunchCfg &c, void *stream);
int launch_lane_any_f64(const LaunchArgs &a, const LaunchCfg &c, void *stream);
int launch_lane_any_f32(const LaunchArgs &a, const LaunchCfg &c, void *stream);

}  // namespace kt

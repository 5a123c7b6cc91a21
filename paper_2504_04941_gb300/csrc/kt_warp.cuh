// kt_warp.cuh -- warp-per-cell fused integrator for larger networks (N <= 96 unknowns).
//
// One warp owns one cell (the paper's Sec. 2.3 gives a whole thread block to a cell;
// a warp keeps every exchange on shuffles and __syncwarp).  Inside the warp:
//   rates          lanes over reactions (modified Arrhenius, Sec. 2.2.1);
//   f and J rows   lanes over species rows, each walking its own list of
//                  (reaction, net coefficient) pairs, so every row is accumulated
//                  by one lane in a fixed order: deterministic, no atomics
//                  (mass-action and thermal-coupling partials, Eq. method-jacobian);
//   T row          lanes over columns: J_T,m = -sum_s h_s J_s,m / C_V;
//   LU             right-looking elimination with the implicit-scaled row pivoting of
//                  Algorithm lu-decomp: shuffle argmax for the pivot (ties to the
//                  smaller row), lanes over columns for the row swap and the
//                  trailing update (same factors as Crout's ordering, other rounding);
//   solve          the right-hand side lives in registers, 3 rows per lane, and each
//                  substitution step broadcasts the finished entry with a shuffle.
// The sub-step control (step doubling, Newton, retry / revert, projection) is the
// same sequence as the FP64 oracle, run warp-uniformly.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kt_exp.cuh"
#include "kt_internal.h"
#include "kt_tma.cuh"
#include "kt_trbdf2.cuh"

namespace kt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps = 8;
constexpr int kQ = 3;   // rows per lane (N <= 96)

struct NetS {
    const double *A, *b, *th, *h, *cv, *cnt, *ex;
    const unsigned long long *idx;
    const int *rp, *re;
};

__device__ __forceinline__ double wsum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return __shfl_sync(kFull, v, 0);
}

__device__ __forceinline__ bool wall(bool p) { return __all_sync(kFull, p) != 0; }

// x < -700 decided on the bit pattern (integer compare; same result as the FP64 compare
// for every non-NaN x): negative and |x| > 700.0 (0x4085E00000000000).
__device__ __forceinline__ bool below_m700(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 && (b & 0x7fffffffffffffffLL) > 0x4085E00000000000LL;
}

// log(T / T_ref), skipping the division when T_ref is 1 (the same value bit for bit).
__device__ __forceinline__ double log_t(double T, double t_ref)
{
    return log(t_ref == 1.0 ? T : T / t_ref);
}

__device__ __forceinline__ void arrhenius(const NetS &t, int r, double lt, double invT, double &k, double &dk)
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

// phi(tau) = (1 - e^-tau)/tau of Eq. photo-reaction-single and its derivative; below
// tau = 0.1 by their Taylor series (8 terms), where the closed forms cancel.
__device__ __forceinline__ void photo_phi(double tau, double &phi, double &dphi)
{
    if (tau < 0.1) {
        double p = 0.0, d = 0.0, pw = 1.0, pwm = 0.0, fact = 1.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            fact *= (k + 1);
            const double sg = (k & 1) ? -1.0 : 1.0;
            p += sg * pw / fact;
            if (k >= 1) d += sg * k * pwm / fact;
            pwm = pw;
            pw *= tau;
        }
        phi = p;
        dphi = d;
    } else {
        const double e = exp(-tau);
        phi = (1.0 - e) / tau;
        dphi = (e * (1.0 + tau) - 1.0) / (tau * tau);
    }
}

// Tabulated rate (Sec. 2.2.1 item 3) of table row tr at T (lT = ln T) for a cell whose
// density sits at weight w between density nodes iR and iR + 1: ln k linear in ln rho
// between those rows (the per-cell reduction of Sec. 2.2.2), then linear in ln T between
// the T nodes; dk/dT from that slope; constant beyond the grid.  Tables are in global
// memory (read-only path).
__device__ __forceinline__ void table_rate(const NetView &nv, const double *tab, int tr, int iR, double w,
                                           double T, double lT, double &k, double &dk)
{
    const int nT = nv.tab_nT;
    const double *r0 = tab + (static_cast<size_t>(tr) * nv.tab_nR + iR) * nT;
    const bool two = nv.tab_nR > 1;
    auto L = [&](int j) { return two ? (1.0 - w) * __ldg(r0 + j) + w * __ldg(r0 + nT + j) : __ldg(r0 + j); };
    const double v = (lT - nv.tab_lt0) / nv.tab_dlt;
    if (!(v > 0.0)) {
        k = exp(L(0));
        dk = 0.0;
        return;
    }
    if (v >= nT - 1) {
        k = exp(L(nT - 1));
        dk = 0.0;
        return;
    }
    int j = static_cast<int>(floor(v));
    if (j > nT - 2) j = nT - 2;
    const double fr = v - j, a = L(j), b = L(j + 1);
    k = exp(a + fr * (b - a));
    dk = k * ((b - a) / nv.tab_dlt) / T;
}

template <typename T>
__device__ __forceinline__ T bcast(const T (&x)[kQ], int j)
{
    const int slot = j >> 5;
    const T v = slot == 0 ? x[0] : (slot == 1 ? x[1] : x[2]);
    return __shfl_sync(kFull, v, j & 31);
}

// Right-looking LU with implicit-scaled partial pivoting on the row-major matrix M
// (row stride NP).  V: inverse row maxima, replaced by the inverse pivots; P: pivot
// rows; G: composed gather index for the right-hand side.  Warp-uniform result.
template <typename T>
__device__ bool warp_lu(T *M, T *V, int *P, int *G, int N, int NP, int lane)
{
    bool ok = true;
    for (int i = lane; i < N; i += 32) {
        T big = T(0);
        for (int m = 0; m < N; ++m) {
            const T a = fabs(M[i * NP + m]);
            big = a > big ? a : big;
        }
        ok = ok && big > T(0);
        V[i] = big > T(0) ? T(1) / big : T(1);
    }
    ok = wall(ok);
    __syncwarp();
    for (int j = 0; j < N; ++j) {
        // pivot: argmax_{i >= j} |a_ij| / rowmax_i, ties to the smaller i
        T best = T(-1);
        int bi = N;
        for (int i = j + lane; i < N; i += 32) {
            T tt = fabs(M[i * NP + j]) * V[i];
            if (!(tt == tt)) tt = T(-1);
            if (tt > best) {
                best = tt;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T ob = __shfl_xor_sync(kFull, best, o);
            const int oi = __shfl_xor_sync(kFull, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        best = __shfl_sync(kFull, best, 0);
        const int p = __shfl_sync(kFull, bi, 0);
        if (!(best > T(0)) || p >= N) return false;
        if (p != j) {
            for (int k = lane; k < N; k += 32) {
                const T a = M[j * NP + k];
                M[j * NP + k] = M[p * NP + k];
                M[p * NP + k] = a;
            }
        }
        __syncwarp();
        if (lane == 0) {
            const T v = V[j];
            V[j] = V[p];
            V[p] = v;
            P[j] = p;
        }
        const T rinv = T(1) / M[j * NP + j];
        for (int i = j + 1 + lane; i < N; i += 32) M[i * NP + j] *= rinv;
        __syncwarp();
        for (int k = j + 1 + lane; k < N; k += 32) {
            const T u = M[j * NP + k];
            for (int i = j + 1; i < N; ++i) M[i * NP + k] -= M[i * NP + j] * u;
        }
        __syncwarp();
        if (lane == 0) V[j] = rinv;
    }
    if (lane == 0) {
        for (int i = 0; i < N; ++i) G[i] = i;
        for (int i = 0; i < N; ++i) {
            const int q = P[i];
            const int g = G[i];
            G[i] = G[q];
            G[q] = g;
        }
    }
    __syncwarp();
    return ok;
}

// x <- M^-1 b for the factors of warp_lu; b gathered from Wb (smem) by G.
template <typename T, typename TB>
__device__ void warp_solve(const T *M, const T *V, const int *G, const TB *Wb, T (&x)[kQ], int N, int NP,
                           int lane)
{
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const int i = lane + 32 * q;
        x[q] = i < N ? static_cast<T>(Wb[G[i]]) : T(0);
    }
    for (int j = 0; j < N - 1; ++j) {
        const T xj = bcast(x, j);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int i = lane + 32 * q;
            if (i > j && i < N) x[q] -= M[i * NP + j] * xj;
        }
    }
    for (int j = N - 1; j >= 0; --j) {
        const T xj = bcast(x, j) * V[j];
        if ((j & 31) == lane) {
            const int slot = j >> 5;
            if (slot == 0) x[0] = xj;
            else if (slot == 1) x[1] = xj;
            else x[2] = xj;
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int i = lane + 32 * q;
            if (i < j) x[q] -= M[i * NP + j] * xj;
        }
    }
}

template <bool ENERGY, bool F32, bool PERSIST>
__global__ void __launch_bounds__(kMaxWarps * 32, 2) warp_kernel(const LaunchArgs a, const WarpLayout L)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const NetView nv = a.nv;
    if (!stage_table(sm, a.blob, static_cast<unsigned>(nv.bytes_warp),
                     reinterpret_cast<uint64_t *>(sm + nv.bytes_warp), &a.scratch->error, kDevErrTma))
        return;
    NetS t;
    t.A = reinterpret_cast<const double *>(sm + nv.off_A);
    t.b = reinterpret_cast<const double *>(sm + nv.off_b);
    t.th = reinterpret_cast<const double *>(sm + nv.off_th);
    t.h = reinterpret_cast<const double *>(sm + nv.off_h);
    t.cv = reinterpret_cast<const double *>(sm + nv.off_cv);
    t.cnt = reinterpret_cast<const double *>(sm + nv.off_cnt);
    t.idx = reinterpret_cast<const unsigned long long *>(sm + nv.off_idx);
    t.rp = reinterpret_cast<const int *>(sm + nv.off_rp);
    t.re = reinterpret_cast<const int *>(sm + nv.off_re);
    t.ex = reinterpret_cast<const double *>(sm + nv.off_exp);
    const DevOpts o = a.o;
    const int N = nv.N, ns = nv.ns, ne = nv.ne, nr = nv.nr, NP = L.NP;
    const long long nc = a.ncells;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *wb = sm + L.base + wid * L.warp_bytes;
    double *M64 = F32 ? nullptr : reinterpret_cast<double *>(wb + L.off_M);
    double *V64 = F32 ? nullptr : reinterpret_cast<double *>(wb + L.off_V);
    float *J32 = F32 ? reinterpret_cast<float *>(wb + L.off_J) : nullptr;
    float *M32 = F32 ? reinterpret_cast<float *>(wb + L.off_M) : nullptr;
    float *V32 = F32 ? reinterpret_cast<float *>(wb + L.off_V) : nullptr;
    int *P = reinterpret_cast<int *>(wb + L.off_P);
    int *G = reinterpret_cast<int *>(wb + L.off_G);
    double *Y = reinterpret_cast<double *>(wb + L.off_Y);
    double *YF = reinterpret_cast<double *>(wb + L.off_YF);
    double *YH = reinterpret_cast<double *>(wb + L.off_YH);
    double *Y2 = reinterpret_cast<double *>(wb + L.off_Y2);
    double *W = reinterpret_cast<double *>(wb + L.off_W);
    double *F0 = reinterpret_cast<double *>(wb + L.off_F0);
    double *K = reinterpret_cast<double *>(wb + L.off_K);
    double *DK = reinterpret_cast<double *>(wb + L.off_DK);
    double *RW = DK;   // the reaction rates of an iteration without a Jacobian (DK is not needed then)

    long long cell = 0;
    double T_iso = 0.0, invCV = 0.0, atol_s = 0.0, dtc = a.dt;
    // C_V(T) of polynomial networks (Sec. 4.2): the cell's coefficients sum_s n0_s c_s,k
    // (five below t_mid, five from t_mid), and C_V'/C_V at the current iterate
    const bool CVP = ENERGY && nv.cvpoly != 0;
    const double *cvp = reinterpret_cast<const double *>(sm + nv.off_cvp);
    double cvc[10];
    double dcvr = 0.0;
    // tabulated and photo rates: rate types, the cell's density weight in the tables,
    // its photo flux factor and path length, and phi'(tau) at the current iterate
    const int *rtype = reinterpret_cast<const int *>(sm + nv.off_rtype);
    const double *sigr = reinterpret_cast<const double *>(sm + nv.off_sigr);
    const double *sigs = reinterpret_cast<const double *>(sm + nv.off_sigs);
    const double *tabs = reinterpret_cast<const double *>(a.blob + nv.off_tab);
    int tab_iR = 0;
    double tab_w = 0.0, ph_F = 1.0, ph_dl = 0.0, ph_phi = 1.0, ph_dphi = 0.0;

    // k and dk/dT of reaction r at T (lt = ln(T/T_ref), lT = ln T); photo-reactions take
    // the current phi(tau) (dk/dT = 0)
    auto rate = [&](int r, double T, double lt, double lT, double invT, double &k, double &dk) {
        const int ty = nv.special ? rtype[r] : 0;
        if (ty == 0) {
            arrhenius(t, r, lt, invT, k, dk);
        } else if (ty == 2) {
            k = ph_F * sigr[r] * ph_phi;
            dk = 0.0;
        } else {
            table_rate(nv, tabs, ty >> 8, tab_iR, tab_w, T, lT, k, dk);
        }
    };
    int nnew = 0;

    auto yin = [&](int s) { return a.y_in[static_cast<long long>(s) * nc + cell]; };

    auto load_pre = [&]() {
        for (int s = lane; s < ns; s += 32) {
            const double v = yin(s);
            Y[s] = v > 0.0 ? v : 0.0;
        }
        const double Tin = a.T_in[cell];
        T_iso = Tin < nv.t_min ? nv.t_min : (Tin > nv.t_max ? nv.t_max : Tin);
        if (ENERGY && lane == 0) Y[ns] = T_iso;
        __syncwarp();
    };

    // species rows of f (into W) and, when wantJ, of J (into the FP64 or FP32 matrix),
    // then the temperature row; all at state yt with the coefficients in K / DK.
    auto rows = [&](const double *yt, bool wantJ) {
        if (!wantJ) {
            // f alone: each reaction's rate w_r = k_r n_i n_j (n_k) once, lanes over
            // reactions, then every species row adds +-w_r per list entry (every entry
            // has a coefficient of +-1), the sign applied on the bit pattern: one FP64
            // add per entry whatever the signs of the 32 rows a warp sums at once, and
            // about a quarter of the FP64 work of forming k n_i n_j in every row a
            // reaction appears in.
            for (int r = lane; r < nr; r += 32) {
                const unsigned long long ix = t.idx[r];
                const int nin = static_cast<int>(ix & 0x7f);
                const double y0 = yt[(ix >> 16) & 0xff];
                const double y1 = nin > 1 ? yt[(ix >> 24) & 0xff] : 1.0;
                const double y2 = nin > 2 ? yt[(ix >> 32) & 0xff] : 1.0;
                RW[r] = K[r] * (y0 * y1) * y2;
            }
            __syncwarp();
            for (int s = lane; s < ns; s += 32) {
                double f = 0.0;
                const int e1 = t.rp[s + 1];
                for (int e = t.rp[s]; e < e1; ++e) {
                    const int ent = t.re[e];
                    // -1 is stored as 0xff: its bit 7 becomes the sign bit of w_r
                    const long long sign = static_cast<long long>(ent & 0x80) << 56;
                    f += __longlong_as_double(__double_as_longlong(RW[ent >> 8]) ^ sign);
                }
                W[s] = f;
            }
        }
        for (int s = lane; wantJ && s < ns; s += 32) {
            double f = 0.0;
            if (wantJ) {
                if (F32) {
                    for (int m = 0; m < N; ++m) J32[s * NP + m] = 0.0f;
                } else {
                    for (int m = 0; m < N; ++m) M64[s * NP + m] = 0.0;
                }
            }
            const int e1 = t.rp[s + 1];
            double gph = 0.0;    // photo: sum over the row's photo reactions of nu F sigma_r n_i phi' dl
            for (int e = t.rp[s]; e < e1; ++e) {
                const int ent = t.re[e];
                const int r = ent >> 8;
                const double nu = static_cast<double>(static_cast<signed char>(ent & 0xff));
                const unsigned long long ix = t.idx[r];
                const int nin = static_cast<int>(ix & 0x7f);
                const int i0 = static_cast<int>((ix >> 16) & 0xff), i1 = static_cast<int>((ix >> 24) & 0xff),
                          i2 = static_cast<int>((ix >> 32) & 0xff);
                const double k = K[r];
                const double y0 = yt[i0];
                const double y1 = nin > 1 ? yt[i1] : 1.0;
                const double y2 = nin > 2 ? yt[i2] : 1.0;
                const double p01 = y0 * y1;
                f += nu * (k * p01 * y2);
                if (wantJ && nv.nphoto && rtype[r] == 2) gph += nu * (ph_F * sigr[r] * y0 * ph_dphi * ph_dl);
                if (wantJ) {
                    // two different reactants: the row entries i0, i1 (and T) differ, so
                    // they are loaded first and stored after (one shared-memory round trip
                    // instead of a chain of read-modify-writes); same updates either way
                    const bool two = nin == 2 && i0 != i1;
                    if (F32) {
                        float *row = J32 + s * NP;
                        if (two) {
                            const float a0 = row[i0], a1 = row[i1], aT = ENERGY ? row[ns] : 0.0f;
                            row[i0] = a0 + static_cast<float>(nu * (k * y1 * y2));
                            row[i1] = a1 + static_cast<float>(nu * (k * y0 * y2));
                            if (ENERGY) row[ns] = aT + static_cast<float>(nu * (DK[r] * p01 * y2));
                        } else {
                            row[i0] += static_cast<float>(nu * (k * y1 * y2));
                            if (nin > 1) row[i1] += static_cast<float>(nu * (k * y0 * y2));
                            if (nin > 2) row[i2] += static_cast<float>(nu * (k * p01));
                            if (ENERGY) row[ns] += static_cast<float>(nu * (DK[r] * p01 * y2));
                        }
                    } else {
                        double *row = M64 + s * NP;
                        if (two) {
                            const double a0 = row[i0], a1 = row[i1], aT = ENERGY ? row[ns] : 0.0;
                            row[i0] = a0 + nu * (k * y1 * y2);
                            row[i1] = a1 + nu * (k * y0 * y2);
                            if (ENERGY) row[ns] = aT + nu * (DK[r] * p01 * y2);
                        } else {
                            row[i0] += nu * (k * y1 * y2);
                            if (nin > 1) row[i1] += nu * (k * y0 * y2);
                            if (nin > 2) row[i2] += nu * (k * p01);
                            if (ENERGY) row[ns] += nu * (DK[r] * p01 * y2);
                        }
                    }
                }
            }
            // dw/dn_m of a photo rate through tau: + (sum) sigma_m for every absorber m
            if (wantJ && gph != 0.0) {
                for (int m = 0; m < ns; ++m) {
                    if (F32) J32[s * NP + m] += static_cast<float>(gph * sigs[m]);
                    else M64[s * NP + m] += gph * sigs[m];
                }
            }
            W[s] = f;
        }
        __syncwarp();
        if (ENERGY) {
            double q = 0.0;
            for (int s = lane; s < ns; s += 32) q += t.h[s] * W[s];
            q = wsum(q);
            if (wantJ) {
                for (int m = lane; m < N; m += 32) {
                    double c = 0.0;
                    if (F32) {
                        for (int s = 0; s < ns; ++s) c += t.h[s] * static_cast<double>(J32[s * NP + m]);
                        J32[ns * NP + m] = static_cast<float>(-c * invCV);
                    } else {
                        for (int s = 0; s < ns; ++s) c += t.h[s] * M64[s * NP + m];
                        M64[ns * NP + m] = -c * invCV;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                W[ns] = -q * invCV;
                // d f_T / d T of C_V(T): -f_T C_V'/C_V
                if (CVP && wantJ) {
                    if (F32) J32[ns * NP + ns] -= static_cast<float>(W[ns] * dcvr);
                    else M64[ns * NP + ns] -= W[ns] * dcvr;
                }
            }
            __syncwarp();
        }
    };

    auto coefficients = [&](double T, const double *yt) {
        if (nv.nphoto) {
            // optical depth tau = dl sum_s n_s sigma_s of the iterate, then phi(tau)
            double sg = 0.0;
            for (int s = lane; s < ns; s += 32) sg += yt[s] * sigs[s];
            photo_phi(ph_dl * wsum(sg), ph_phi, ph_dphi);
            if (!ENERGY) {
                for (int r = lane; r < nr; r += 32)
                    if (rtype[r] == 2) K[r] = ph_F * sigr[r] * ph_phi;
                __syncwarp();
            }
        }
        if (CVP) {
            const int o5 = T < nv.t_mid ? 0 : 5;
            const double cv = (((cvc[o5 + 4] * T + cvc[o5 + 3]) * T + cvc[o5 + 2]) * T + cvc[o5 + 1]) * T + cvc[o5];
            const double dcv = ((4.0 * cvc[o5 + 4] * T + 3.0 * cvc[o5 + 3]) * T + 2.0 * cvc[o5 + 2]) * T + cvc[o5 + 1];
            invCV = 1.0 / cv;
            dcvr = dcv * invCV;
        }
        if (ENERGY) {
            const double lt = log_t(T, nv.t_ref), invT = 1.0 / T;
            const double lT = nv.ntab ? log(T) : 0.0;
            for (int r = lane; r < nr; r += 32) {
                double k, dk;
                rate(r, T, lt, lT, invT, k, dk);
                K[r] = k;
                DK[r] = dk;
            }
            __syncwarp();
        }
    };

    // factor state of the FP32 form
    bool luok32 = false;
    double h_fact = -1.0;

    // One backward-Euler solve yt = yb + hph f(yt) by Newton from the guess in yt.
    // fmode (FP32 form): 2 assemble J at the guess and factor; 1 factor from the
    // stored J; 0 reuse the current factor.
    auto be_solve = [&](const double *yb, double *yt, double hph, int fmode) -> bool {
        int refresh = 0;
        bool doJ = F32 && fmode == 2, doF = F32 && fmode >= 1;
        float dprev = 0.0f, dprevr = 0.0f;
        for (int it = 0;; ++it) {
            ++nnew;
            const double T = ENERGY ? yt[ns] : T_iso;
            if (!(T > 0.0)) return false;
            coefficients(T, yt);
            bool luok;
            double x[kQ];
            if (!F32) {
                rows(yt, true);
                for (int i = lane; i < N; i += 32) {
                    double *row = M64 + i * NP;
                    for (int m = 0; m < N; ++m) row[m] = (i == m ? 1.0 : 0.0) - hph * row[m];
                    W[i] = -(yt[i] - yb[i] - hph * W[i]);
                }
                __syncwarp();
                luok = warp_lu<double>(M64, V64, P, G, N, NP, lane);
                if (!luok) return false;
                warp_solve<double, double>(M64, V64, G, W, x, N, NP, lane);
            } else {
                rows(yt, doJ);
                if (doF) {
                    for (int i = lane; i < N; i += 32)
                        for (int m = 0; m < N; ++m)
                            M32[i * NP + m] = (i == m ? 1.0f : 0.0f) - static_cast<float>(hph) * J32[i * NP + m];
                    __syncwarp();
                    luok32 = warp_lu<float>(M32, V32, P, G, N, NP, lane);
                    h_fact = hph;
                }
                doJ = false;
                doF = false;
                if (!luok32) return false;
                for (int i = lane; i < N; i += 32) W[i] = -(yt[i] - yb[i] - hph * W[i]);
                __syncwarp();
                float xf[kQ];
                warp_solve<float, double>(M32, V32, G, W, xf, N, NP, lane);
#pragma unroll
                for (int q = 0; q < kQ; ++q) x[q] = static_cast<double>(xf[q]);
            }
            bool conv = true;
            // contraction monitors (FP32 is plenty): dmax = max |delta|/tol, dmaxr =
            // max |delta| / (newton_rtol |y|), the purely relative part of the tolerance
            float dmax = 0.0f, dmaxr = 0.0f;
            const double natol = (F32 ? o.newton_atol_frac * kF32NewtonAtolScale : o.newton_atol_frac) * atol_s;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const int i = lane + 32 * q;
                if (i < N) {
                    const double y = yt[i] + x[q];
                    yt[i] = y;
                    const double tol = (i < ns ? natol : 0.0) + o.newton_rtol * fabs(y);
                    if (!(fabs(x[q]) <= tol)) conv = false;
                    if (F32) {
                        const float ad = static_cast<float>(fabs(x[q])), tf = static_cast<float>(tol);
                        const float r = __fdiv_rn(ad, fmaxf(tf, 1e-37f));
                        // the relative part newton_rtol |y| formed directly: as a difference
                        // tf - natol in FP32 it rounds to an ulp of natol for trace species
                        const float trl = static_cast<float>(o.newton_rtol * fabs(y));
                        const float rr = __fdiv_rn(ad, fmaxf(trl, 1e-37f));
                        dmax = r > dmax ? r : dmax;
                        dmaxr = rr > dmaxr ? rr : dmaxr;
                    }
                }
            }
            __syncwarp();
            conv = wall(conv);
            if (conv) return true;
            if (!F32) {
                if (it + 1 >= o.max_newton) return false;
            } else {
                for (int off = 16; off > 0; off >>= 1) {
                    dmax = fmaxf(dmax, __shfl_xor_sync(kFull, dmax, off));
                    dmaxr = fmaxf(dmaxr, __shfl_xor_sync(kFull, dmaxr, off));
                }
                dmax = __shfl_sync(kFull, dmax, 0);
                dmaxr = __shfl_sync(kFull, dmaxr, 0);
                if (!isfinite(dmax)) return false;
                // stop on the contraction rate (Hairer & Wanner, Solving ODEs II, Sec. IV.8):
                // with theta = dmaxr / dprevr < 1/2 the error left after this update is about
                // theta / (1 - theta) * |delta|; accept when that is within newton_rtol |y_i|
                // for every component (the relative part only: species below the absolute
                // tolerance end as close to the root as the plain test leaves them)
                if (it > 0) {
                    const float th = dmaxr / dprevr;
                    if (th < 0.5f && th / (1.0f - th) * dmaxr <= 1.0f) return true;
                }
                const bool stalled = it > 0 && !(dmax < 0.5f * dprev);
                if (stalled || it + 1 >= o.max_newton) {
                    if (refresh >= 2) return false;
                    ++refresh;
                    doJ = true;
                    doF = true;
                    it = -1;
                }
                dprev = dmax;
                dprevr = dmaxr;
            }
        }
    };

    // Sub-steps over [0, dtc] in either scheme; every Newton solve goes through the one
    // call of be_solve below (one inlined copy of the solver per kernel).
    //   backward Euler with step doubling: stage 0 the full step h from Y (-> YF),
    //     stage 1 the first half step from Y (-> YH), stage 2 the second from YH (-> Y2)
    //   TR-BDF2 (o.scheme == KT_SCHEME_TRBDF2): stage 0 trapezoidal, r = Y + d h f_n in
    //     YH (-> YF), stage 1 BDF2, r = w1 YF - w0 Y in YH (-> Y2); one FP32 factor of
    //     I - d h J serves both stages.  F0 holds f_n: f(Y) on the cell's first step,
    //     afterwards the previous step's stage relation (y_{n+1} - r)/(d h), which keeps
    //     the rounding of an evaluated rate (amplified by h k in the error estimate) out
    //     of the accept decision
    auto advance = [&](double h0, double fgrow, int &nacc) -> bool {
        const bool trs = o.scheme == KT_SCHEME_TRBDF2;
        const TrCoef tr = tr_coef();
        const int nst = trs ? 2 : 3;
        double tt = 0.0, h = h0;
        int natt = 0;
        bool f0ok = false;
        nacc = 0;
        for (;;) {
            if (natt >= o.max_substeps) return false;
            ++natt;
            bool last = false;
            if (tt + h >= dtc * (1.0 - 1e-12)) {
                h = dtc - tt;
                last = true;
            }
            const double dh = tr.d * h;
            bool ok = true;
            if (trs && !f0ok) {
                const double T = ENERGY ? Y[ns] : T_iso;
                ok = T > 0.0;
                if (ok) {
                    coefficients(T, Y);
                    rows(Y, false);
                    for (int i = lane; i < N; i += 32) F0[i] = W[i];
                    __syncwarp();
                    f0ok = true;
                }
            }
            for (int stg = 0; ok && stg < nst; ++stg) {
                const double *yb;
                double *yt;
                double hph;
                int fmode;
                if (trs) {
                    for (int i = lane; i < N; i += 32) {
                        if (stg == 0) {
                            YH[i] = Y[i] + dh * F0[i];
                            YF[i] = Y[i];
                        } else {
                            YH[i] = tr.w1 * YF[i] - tr.w0 * Y[i];
                            Y2[i] = YF[i];
                        }
                    }
                    yb = YH;
                    yt = stg == 0 ? YF : Y2;
                    hph = dh;
                    fmode = stg == 0 ? 2 : 0;
                } else {
                    const double *g = stg < 2 ? Y : (o.guess != KT_GUESS_PREV ? YF : YH);
                    yt = stg == 0 ? YF : (stg == 1 ? YH : Y2);
                    for (int i = lane; i < N; i += 32) yt[i] = g[i];
                    yb = stg == 2 ? YH : Y;
                    hph = stg == 0 ? h : 0.5 * h;
                    fmode = 2 - stg;
                }
                __syncwarp();
                ok = be_solve(yb, yt, hph, fmode);
            }
            if (!ok) {
                h *= 0.5;
                if (h < o.h_min) return false;
                continue;
            }
            double s2 = 0.0;
            if (trs) {
                // local error estimate 2 C h (a0 f_n + a1 f_g + a2 f_{n+1}), the stage
                // rates taken from the stage equations
                const double inv = 1.0 / dh, ce = 2.0 * tr.C * h;
                for (int i = lane; i < N; i += 32) {
                    const double yn = Y[i], y1 = Y2[i], f0 = F0[i];
                    const double fg = (YF[i] - yn) * inv - f0;
                    const double f1 = (y1 - YH[i]) * inv;
                    const double est = ce * (tr.a0 * f0 + tr.a1 * fg + tr.a2 * f1);
                    const double sc = (i < ns ? atol_s : 0.0) + o.rtol * fmax(fabs(yn), fabs(y1));
                    const double e = est / sc;
                    s2 += e * e;
                }
            } else {
                for (int i = lane; i < N; i += 32) {
                    const double y = Y[i], y2 = Y2[i];
                    const double sc = (i < ns ? atol_s : 0.0) + o.rtol * fmax(fabs(y), fabs(y2));
                    const double e = (y2 - YF[i]) / sc;
                    s2 += e * e;
                }
            }
            const double err = sqrt(wsum(s2) / N);
            if (err <= 1.0) {
                const double inv = trs ? 1.0 / dh : 0.0;
                for (int i = lane; i < N; i += 32) {
                    if (trs) F0[i] = (Y2[i] - YH[i]) * inv;    // first same as last
                    Y[i] = Y2[i];
                }
                __syncwarp();
                ++nacc;
                if (last) return true;
                tt += h;
                double fac = err > 0.0 ? 0.9 / (trs ? cbrt(err) : sqrt(err)) : fgrow;
                if (fac > fgrow) fac = fgrow;
                if (fac < 0.2) fac = 0.2;
                h *= fac;
            } else {
                double fac = 0.9 / (trs ? cbrt(err) : sqrt(err));
                if (!(fac >= 0.2)) fac = 0.2;
                h *= fac;
                if (h < o.h_min) return false;
            }
        }
    };

    // clip, then restore the element totals of the pre-processed input (Sec. 2.2.3)
    auto post_process = [&]() -> bool {
        double b0[kMaxElements], r[kMaxElements], Mp[kMaxElements * kMaxElements];
        for (int s = lane; s < ns; s += 32)
            if (Y[s] < 0.0) Y[s] = 0.0;
        __syncwarp();
        for (int e = 0; e < ne; ++e) {
            double pb = 0.0, pt = 0.0;
            for (int s = lane; s < ns; s += 32) {
                const double v = yin(s);
                pb += t.cnt[s * ne + e] * (v > 0.0 ? v : 0.0);
                pt += t.cnt[s * ne + e] * Y[s];
            }
            b0[e] = wsum(pb);
            r[e] = wsum(pt) - b0[e];
            for (int f = 0; f < ne; ++f) {
                double pm = 0.0;
                for (int s = lane; s < ns; s += 32) pm += t.cnt[s * ne + e] * t.cnt[s * ne + f] * Y[s];
                Mp[e * ne + f] = wsum(pm);
            }
        }
        for (int e = 0; e < ne; ++e) {
            if (Mp[e * ne + e] == 0.0) {
                if (r[e] != 0.0) return false;
                for (int f = 0; f < ne; ++f) Mp[e * ne + f] = Mp[f * ne + e] = 0.0;
                Mp[e * ne + e] = 1.0;
            }
        }
        for (int k = 0; k < ne; ++k) {
            int p = k;
            for (int i = k + 1; i < ne; ++i)
                if (fabs(Mp[i * ne + k]) > fabs(Mp[p * ne + k])) p = i;
            if (!(fabs(Mp[p * ne + k]) > 0.0)) return false;
            if (p != k) {
                for (int j = 0; j < ne; ++j) {
                    const double xx = Mp[k * ne + j];
                    Mp[k * ne + j] = Mp[p * ne + j];
                    Mp[p * ne + j] = xx;
                }
                const double xx = r[k];
                r[k] = r[p];
                r[p] = xx;
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
        for (int s = lane; s < ns; s += 32) {
            double corr = 0.0;
            for (int e = 0; e < ne; ++e) corr += t.cnt[s * ne + e] * r[e];
            ok = ok && corr < 1.0;
            Y[s] -= Y[s] * corr;
        }
        __syncwarp();
        for (int i = lane; i < N; i += 32) ok = ok && isfinite(Y[i]);
        return wall(ok);
    };

    auto write_out = [&](int st, int nsub) {
        for (int s = lane; s < ns; s += 32) a.y_out[static_cast<long long>(s) * nc + cell] = Y[s];
        if (lane == 0) {
            a.T_out[cell] = ENERGY ? Y[ns] : T_iso;
            if (a.status) a.status[cell] = st;
            if (a.nsub) a.nsub[cell] = nsub;
            if (a.nnew) a.nnew[cell] = nnew;
        }
    };

    auto process_cell = [&]() {
        dtc = a.dt_cell ? a.dt_cell[cell] : a.dt;
        bool fin = isfinite(a.T_in[cell]) && dtc > 0.0 && isfinite(dtc);
        for (int s = lane; s < ns; s += 32) fin = fin && isfinite(yin(s));
        if (!wall(fin)) {
            for (int s = lane; s < ns; s += 32) a.y_out[static_cast<long long>(s) * nc + cell] = yin(s);
            if (lane == 0) {
                a.T_out[cell] = a.T_in[cell];
                if (a.status) a.status[cell] = KT_STATUS_NONFINITE;
                if (a.nsub) a.nsub[cell] = 0;
                if (a.nnew) a.nnew[cell] = 0;
            }
            return;
        }
        load_pre();
        double cvt = 0.0, b00 = 0.0;
        for (int s = lane; s < ns; s += 32) {
            cvt += t.cv[s] * Y[s];
            b00 += t.cnt[s * ne] * Y[s];
        }
        cvt = wsum(cvt);
        b00 = wsum(b00);
        invCV = ENERGY ? 1.0 / cvt : 0.0;
        if (CVP) {
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                double c = 0.0;
                for (int s = lane; s < ns; s += 32) c += Y[s] * cvp[s * 10 + k];
                cvc[k] = wsum(c);
            }
        }
        atol_s = (o.atol_mode == 1 && b00 > 0.0) ? o.atol * b00 : o.atol;
        // pre-processing of tabulated and photo rates (Sec. 2.2.2): the cell's weight in
        // the density nodes of the tables, its flux factor and path length
        if (nv.special) {
            ph_F = a.flux ? a.flux[cell] : 1.0;
            ph_dl = a.path ? a.path[cell] : 0.0;
            ph_phi = 1.0;
            ph_dphi = 0.0;
            tab_iR = 0;
            tab_w = 0.0;
            if (nv.ntab && nv.tab_nR > 1) {
                const double rho_c = a.rho ? a.rho[cell] : 1.0;
                double u = (log(rho_c) - nv.tab_lr0) / nv.tab_dlr * (nv.tab_nR - 1);
                if (!(u > 0.0)) u = 0.0;
                if (u > nv.tab_nR - 1) u = nv.tab_nR - 1;
                tab_iR = static_cast<int>(floor(u));
                if (tab_iR > nv.tab_nR - 2) tab_iR = nv.tab_nR - 2;
                tab_w = u - tab_iR;
            }
        }
        if (!ENERGY) {
            const double lt = log_t(T_iso, nv.t_ref), invT = 1.0 / T_iso;
            const double lT = nv.ntab ? log(T_iso) : 0.0;
            for (int r = lane; r < nr; r += 32) {
                double k, dk;
                rate(r, T_iso, lt, lT, invT, k, dk);
                K[r] = k;
            }
            __syncwarp();
        }
        nnew = 0;
        int nacc = 0;
        bool ok = advance(o.h_init, o.facmax, nacc) && post_process();
        int st = KT_STATUS_OK;
        if (!ok && o.retry) {
            st = KT_STATUS_RETRIED;
            load_pre();
            ok = advance(o.h_init * o.retry_h_factor, o.retry_facmax, nacc) && post_process();
        }
        if (!ok) {
            load_pre();
            write_out(KT_STATUS_REVERTED, 0);
        } else {
            write_out(st, nacc);
        }
        __syncwarp();
    };

    if (PERSIST) {
        for (;;) {
            unsigned long long c = 0;
            if (lane == 0) c = atomicAdd(&a.scratch->queue, 1ULL);
            c = __shfl_sync(kFull, c, 0);
            if (c >= static_cast<unsigned long long>(nc)) break;
            cell = a.order ? static_cast<long long>(a.order[c]) : static_cast<long long>(c);
            process_cell();
        }
    } else {
        cell = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + wid;
        if (cell < nc) process_cell();
    }
    (void)h_fact;
}

template <bool ENERGY, bool F32, bool PERSIST>
int launch_t(const LaunchArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    const WarpLayout L = warp_layout(a.nv.N, a.nv.nr, a.nv.energy, F32 ? 1 : 0, a.nv.bytes_warp,
                                     F32 && a.o.scheme == KT_SCHEME_TRBDF2);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int smem_optin = 0, nsm = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int warps = c.block_warps > 0 ? c.block_warps : 4;
    if (warps > kMaxWarps) warps = kMaxWarps;
    while (warps > 1 && L.base + warps * L.warp_bytes > smem_optin) --warps;
    const size_t smem = static_cast<size_t>(L.base) + static_cast<size_t>(warps) * L.warp_bytes;
    if (smem > static_cast<size_t>(smem_optin)) return cudaErrorInvalidConfiguration;
    auto kern = warp_kernel<ENERGY, F32, PERSIST>;
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
        const long long need = (a.ncells + warps - 1) / warps;
        if (blocks > need) blocks = need;
    } else {
        blocks = (a.ncells + warps - 1) / warps;
    }
    if (blocks < 1) return cudaSuccess;
    kern<<<static_cast<unsigned>(blocks), threads, smem, s>>>(a, L);
    return cudaGetLastError();
}

// Dispatch over the compile-time options for one form of the iteration matrix.
template <bool F32>
int launch_warp_form(const LaunchArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    const bool en = a.nv.energy != 0, per = c.persistent != 0;
    if (en) return per ? launch_t<true, F32, true>(a, c, s) : launch_t<true, F32, false>(a, c, s);
    return per ? launch_t<false, F32, true>(a, c, s) : launch_t<false, F32, false>(a, c, s);
}

}  // namespace

// One translation unit per form (compile time).
int launch_warp_f64(const LaunchArgs &a, const LaunchCfg &c, void *stream);
int launch_warp_f32(const LaunchArgs &a, const LaunchCfg &c, void *stream);

}  // namespace kt

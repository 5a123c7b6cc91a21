// kt_internal.h -- structures shared by the host side and the kernels of libkt.
#pragma once

#include <cstdint>
#include <cstddef>

#include "../../include/kt.h"

namespace kt {

constexpr int kMaxSide = 3;      // reactants / products per reaction
constexpr int kMaxElements = 8;
constexpr int kLaneMaxN = 16;    // unknowns per cell handled by the lane-per-cell kernels
constexpr int kIdxNone = 255;

// Byte layout of the device copy of a network ("blob").  Every section starts on a
// 16-byte boundary so the whole blob can be staged into shared memory by one bulk
// (TMA) copy and read back with the same offsets.
struct NetView {
    int ns, ne, nr, energy, N;
    int off_A, off_b, off_th, off_dH;     // double[nr]: prefactor, exponent, activation T, heat
    int off_h, off_cv, off_cnt;           // double[ns], double[ns], double[ns*ne]
    int off_idx;                          // uint8[nr*8]: nin, nout, in0..2, out0..2
    int bytes;                            // total, multiple of 16
    double t_ref, t_min, t_max;
};

// Device copy of the integration options (POD kernel parameter).
struct DevOpts {
    double rtol, atol, h_init, h_min, newton_rtol, newton_atol_frac;
    double facmax, retry_h_factor, retry_facmax;
    int max_substeps, max_newton, retry, atol_mode, guess;
};

// Scratch words of one integrate call (device memory, 16 B).
struct Scratch {
    unsigned long long queue;   // next cell of the persistent work queue
    int error;                  // KT_E* recorded by a kernel (0 = none)
    int pad;
};

enum DevError : int { kDevErrNone = 0, kDevErrTma = 1 };

struct LaunchArgs {
    NetView nv;
    const unsigned char *blob;   // device network blob
    DevOpts o;
    double dt;
    long long ncells;
    const double *y_in, *T_in;
    double *y_out, *T_out;
    int *status, *nsub, *nnew;
    Scratch *scratch;
};

struct LaunchCfg {
    int form;           // KT_FORM_*
    int persistent;
    int block_warps;    // 0 = auto
    int blocks_per_sm;  // 0 = auto
};

// Shared-memory layout of one warp of the lane-per-cell kernels.  Every per-cell
// array is lane-interleaved: element e of lane l sits at base[e * 32 + l], so a warp
// touching "the same element of its 32 cells" reads 32 consecutive words (no bank
// conflicts), even when the element index differs per lane (pivot rows).
struct LaneLayout {
    int off_M, off_J, off_V, off_P, off_X;         // matrix / factor / scale / perm / fp32 rhs
    int off_Y, off_YF, off_YH, off_Y2, off_W;      // fp64 vectors
    int off_K;                                     // per-cell rate coefficients (isothermal)
    int warp_bytes;                                // bytes per warp
    int base;                                      // byte offset of warp 0 (after blob + barrier)
};

inline LaneLayout lane_layout(int N, int nr, int energy, int fp32, int blob_bytes)
{
    LaneLayout L{};
    const int d = 32 * 8, f = 32 * 4;   // bytes per element of a double / 4-byte array
    int o = 0;
    if (fp32) {
        L.off_J = o; o += N * N * f;
        L.off_M = o; o += N * N * f;
        L.off_V = o; o += N * f;
        L.off_X = o; o += N * f;
    } else {
        L.off_J = -1;
        L.off_X = -1;
        L.off_M = o; o += N * N * d;
        L.off_V = o; o += N * d;
    }
    L.off_P = o; o += N * f;
    o = (o + 255) & ~255;
    L.off_Y = o; o += N * d;
    L.off_YF = o; o += N * d;
    L.off_YH = o; o += N * d;
    L.off_Y2 = o; o += N * d;
    L.off_W = o; o += N * d;
    if (!energy) { L.off_K = o; o += nr * d; } else { L.off_K = -1; }
    L.warp_bytes = (o + 255) & ~255;
    L.base = (blob_bytes + 16 + 255) & ~255;
    return L;
}

// Lane-per-cell kernels (N <= kLaneMaxN); returns a cudaError_t value.
int launch_lane(const LaunchArgs &a, const LaunchCfg &c, void *stream);

}  // namespace kt

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
constexpr int kIdxDistinct = 0x80;   // flag in the reactant-count byte: all species differ
constexpr int kExpTable = 256;       // entries 2^(j/256) of the table-driven exponential
// The FP32-LU form's simplified Newton converges linearly and stops with an error about
// as large as its last update, where full Newton (quadratic) stops far below it.  Its
// absolute Newton tolerance is therefore newton_atol_frac * atol scaled by this factor:
// trace species below atol then land on full Newton's root to ~1e-9 relative (measured
// 3e-5 without it on the 32-species network), and the error norm of the step control,
// weighted by atol, sees a Newton residue below 1e-8 of its weights, so accept/reject
// decisions agree with full Newton's except within ~1e-8 of the threshold.  The root
// itself does not change; the cost is ~2 % more iterations on that network.
constexpr double kF32NewtonAtolScale = 1e-6;

// Byte layout of the device copy of a network ("blob").  Every section starts on a
// 16-byte boundary so the whole blob can be staged into shared memory by one bulk
// (TMA) copy and read back with the same offsets.
struct NetView {
    int ns, ne, nr, energy, N;
    int off_A, off_b, off_th, off_dH;     // double[nr]: prefactor, exponent, activation T, heat
    int off_f32;                          // float[3][nr]: b, activation T and heat in FP32
    int off_h, off_cv, off_cnt;           // double[ns], double[ns], double[ns*ne]
    int off_idx;                          // uint8[nr*8]: nin (| kIdxDistinct), nout, in0..2, out0..2
    int off_exp;                          // double[kExpTable]: 2^(j/256) for the table-driven exp
    int off_rp, off_re, nent;             // per-species reaction lists (CSR): int32 row
                                          // pointers [ns+1]; entries (r << 8) | (nu & 0xff),
                                          // nu = +-1: a net stoichiometric coefficient of
                                          // magnitude m appears as m entries
    int shape;                            // 22: every reaction has 2 reactants and 2
                                          // products (straight-line rate code); 0: mixed
    int cvpoly, off_cvp;                  // heat capacities polynomial in T: double[ns*10],
                                          // cv_s(T) = sum_k c[10s+k] T^k below t_mid,
                                          // sum_k c[10s+5+k] T^k from t_mid (Sec. 4.2)
    int special, nphoto;                  // any tabulated or photo rates; photo count
    int off_rtype;                        // int32[nr]: 0 Arrhenius, 2 photo, 1 | (row << 8) table
    int off_sigr, off_sigs;               // double[nr] photo cross-sections, double[ns] the
                                          // species' absorption (sum over its photo reactions)
    int ntab, tab_nT, tab_nR, off_tab;    // tables: double[ntab][nR][nT] ln k after the staged
                                          // part (global memory)
    int bytes;                            // staged part (shared memory), multiple of 16
    int bytes_warp;                       // the prefix the warp-per-cell kernels stage
                                          // (no reaction heats; photo and table
                                          // descriptors only when the network has them)
    int bytes_total;                      // the whole blob, tables included
    double t_ref, t_min, t_max, t_mid;
    double tab_lt0, tab_dlt, tab_lr0, tab_dlr;   // ln T0, ln-T node spacing, ln rho0, ln(rho1/rho0)
};

// Device copy of the integration options (POD kernel parameter).
struct DevOpts {
    double rtol, atol, h_init, h_min, newton_rtol, newton_atol_frac;
    double facmax, retry_h_factor, retry_facmax;
    int max_substeps, max_newton, retry, atol_mode, guess, scheme;
};

// Scratch words of one integrate call (device memory, 16 B).
struct Scratch {
    unsigned long long queue;   // next cell of the persistent work queue
    int error;                  // KT_E* recorded by a kernel (0 = none)
    unsigned rescues;           // diagnostic: FP32-LU solves redone in FP64 during the call
};

enum DevError : int { kDevErrNone = 0, kDevErrTma = 1 };

struct LaunchArgs {
    NetView nv;
    const unsigned char *blob;   // device network blob
    DevOpts o;
    double dt;
    const double *dt_cell;       // per-cell dt (device, may be null: dt for every cell)
    const double *rho;           // per-cell density (device, may be null: 1)
    const unsigned char *mlp;    // packed MLP block for the learned guess (may be null)
    const double *flux, *path;   // per-cell photo flux factor and path length (may be null:
                                 // F = 1, dl = 0)
    int mlp_nin, mlp_nout;
    long long ncells;
    const double *y_in, *T_in;
    double *y_out, *T_out;
    int *status, *nsub, *nnew;
    Scratch *scratch;
    const int *order;            // persistent queue order (device, may be null: index order)
};

struct LaunchCfg {
    int form;           // KT_FORM_*
    int persistent;
    int block_warps;    // 0 = auto
    int blocks_per_sm;  // 0 = auto
    int cells_per_warp; // 32: lane-per-cell kernels, 1: warp-per-cell kernels
    int lane_variant;   // KT_LANE_*: storage of the FP32-LU lane kernels under TR-BDF2
};

// Shared-memory layout of one warp of the lane-per-cell kernels.  Every per-cell
// array is lane-interleaved: element e of lane l sits at base[e * 32 + l], so a warp
// touching "the same element of its 32 cells" reads 32 consecutive words (no bank
// conflicts), even when the element index differs per lane (pivot rows).
struct LaneLayout {
    int off_M, off_J, off_V, off_P, off_X;         // matrix / factor / scale / perm / fp32 rhs
    int off_Y, off_YF, off_YH, off_Y2, off_W;      // fp64 vectors
    int off_K;                                     // per-cell rate coefficients (isothermal)
    int off_FY;                                    // f at the attempt's start state
    int off_CV;                                    // C_V(T) of polynomial networks: the cell's
                                                   // 10 aggregated coefficients (-1: none)
    int warp_bytes;                                // bytes per warp
    int mlp_off;                                   // byte offset of the staged MLP block
    int base;                                      // byte offset of warp 0 (after blob, barriers, MLP)
};

inline LaneLayout lane_layout(int N, int nr, int energy, int fp32, int blob_bytes, int mlp_bytes = 0,
                              int cvpoly = 0)
{
    LaneLayout L{};
    const int d = 32 * 8, f = 32 * 4;   // bytes per element of a double / 4-byte array
    int o = 0;
    if (fp32) {
        // J32/M32 (and V32/X32) interleave per lane: element e of lane l at float
        // 64 e + 2 l (+1), so the lane's FP64 rescue matrix (double 32 e + l) overlays
        // exactly its own FP32 slots.
        L.off_J = o;
        L.off_M = o;
        o += N * N * d;
        L.off_V = o;
        L.off_X = o;
        o += N * d;
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
    L.off_FY = o; o += N * d;      // f at the attempt's start state (FP32 form; TR-BDF2)
    if (!energy) { L.off_K = o; o += nr * d; } else { L.off_K = -1; }
    if (cvpoly) { L.off_CV = o; o += 10 * d; } else { L.off_CV = -1; }
    L.warp_bytes = (o + 255) & ~255;
    L.mlp_off = (blob_bytes + 16 + 255) & ~255;
    L.base = (L.mlp_off + mlp_bytes + 255) & ~255;
    return L;
}

// Shared-memory layout of one warp of the lean FP32-LU lane kernels (TR-BDF2 only;
// the step's start state y_n and its rate f_n live in registers): the FP32 iteration
// matrix I - d h J, assembled directly and factorised in place (inverse pivots on its
// diagonal); the rate vector f (FP64), whose slots the LU's FP32 row scales reuse once
// the Newton residual has been formed from it; one pivot byte per row; the stage
// iterates and the stage right-hand side.  11 unknowns: 27,136 bytes per warp.
inline LaneLayout lane_layout_lean(int N, int nr, int energy, int blob_bytes, int cvpoly)
{
    LaneLayout L{};
    const int d = 32 * 8, f = 32 * 4;
    int o = 0;
    L.off_M = o; o += N * N * f;
    L.off_W = o; o += N * d;
    L.off_V = L.off_W;
    L.off_P = o; o += N * 32;
    o = (o + 255) & ~255;
    L.off_YF = o; o += N * d;
    L.off_YH = o; o += N * d;
    L.off_Y2 = o; o += N * d;
    L.off_J = L.off_X = L.off_Y = L.off_FY = -1;
    if (!energy) { L.off_K = o; o += nr * d; } else { L.off_K = -1; }
    if (cvpoly) { L.off_CV = o; o += 10 * d; } else { L.off_CV = -1; }
    L.warp_bytes = (o + 255) & ~255;
    L.mlp_off = (blob_bytes + 16 + 255) & ~255;
    L.base = L.mlp_off;
    return L;
}

// Shared-memory layout of one warp of the warp-per-cell kernels (one cell per warp).
// Matrices are row-major with an odd row stride NP (conflict-free column reads).
struct WarpLayout {
    int NP;
    int off_M, off_J, off_V, off_P, off_G;   // matrix, fp32 Jacobian, scales, pivots, gather
    int off_Y, off_YF, off_YH, off_Y2, off_W;
    int off_F0;                              // TR-BDF2: f at the step's start state
    int off_K, off_DK;                       // rate coefficients and dk/dT (or the rates) per reaction
    int warp_bytes, base;
};

// share_jm (FP32 form under TR-BDF2): the FP32 Jacobian is assembled in the storage of
// the iteration matrix and turned into I - d h J in place, since TR-BDF2 factorises
// once per step attempt from a freshly assembled Jacobian and never re-uses it.
inline WarpLayout warp_layout(int N, int nr, int energy, int fp32, int blob_bytes, bool share_jm = false)
{
    WarpLayout L{};
    L.NP = N | 1;
    const int NN = N * L.NP;
    int o = 0;
    auto take = [&](int bytes) { int r = o; o = (o + bytes + 15) & ~15; return r; };
    if (fp32) {
        L.off_J = take(NN * 4);
        L.off_M = share_jm ? L.off_J : take(NN * 4);
        L.off_V = take(N * 4);
    } else {
        L.off_J = -1;
        L.off_M = take(NN * 8);
        L.off_V = take(N * 8);
    }
    L.off_P = take(N * 4);
    L.off_G = take(N * 4);
    L.off_Y = take(N * 8);
    L.off_YF = take(N * 8);
    L.off_YH = take(N * 8);
    L.off_Y2 = take(N * 8);
    L.off_W = take(N * 8);
    L.off_F0 = take(N * 8);
    L.off_K = take(nr * 8);
    L.off_DK = take(nr * 8);   // dk/dT; in iterations without a Jacobian, the reaction rates
    L.warp_bytes = (o + 127) & ~127;
    L.base = (blob_bytes + 16 + 127) & ~127;
    return L;
}

constexpr int kWarpMaxN = 96;   // unknowns per cell handled by the warp-per-cell kernels

// Thread-local error message shared by every entry point of the library.
void set_error(const char *msg);

// Entry j of the 2^(j/32) table of the table-driven exponential.
double exp2_table(int j);

// Device copy of an MLP's packed parameter block (null if m is null).
const unsigned char *mlp_device_block(const kt_mlp *m, int *nin, int *nout, int *device);

// Launch arguments of an integrate call without its device tables and scratch (the
// caller supplies both); validates like the allocating entry points.  Used by the
// entry point that allocates nothing.
int prepare_launch(const kt_network *net, int64_t ncells, const double *y_in, const double *T_in,
                   const double *rho, double dt, const kt_options *opts, double *y_out, double *T_out,
                   int32_t *status, int32_t *n_substeps, int32_t *n_newton, LaunchArgs *a, LaunchCfg *c,
                   const unsigned char **host_blob);

// Orthonormal basis Vr [ns][rank] of the element matrix's row space (rank <= 8).
int network_element_basis(const kt_network *net, double *Vr, int *ns, int *rank);

// Longest-first queue order from per-cell cost counts (kt_sched.cu): work holds
// 2 * kSchedBuckets unsigned words, order receives a permutation of 0..ncells-1 with the
// cells of the largest counts first.  Returns a cudaError_t value.
constexpr int kSchedBuckets = 128;
int launch_schedule(const int *count, long long ncells, unsigned *work, int *order, void *stream);

// Lane-per-cell kernels (N <= kLaneMaxN); returns a cudaError_t value.
int launch_lane(const LaunchArgs &a, const LaunchCfg &c, void *stream);
// Warp-per-cell kernels (N <= kWarpMaxN); returns a cudaError_t value.
int launch_warp(const LaunchArgs &a, const LaunchCfg &c, void *stream);

}  // namespace kt

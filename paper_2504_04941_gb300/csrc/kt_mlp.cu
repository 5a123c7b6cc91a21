// kt_mlp.cu -- training and batch inference of the learned-guess MLP.
//
// Parameters live twice: FP32 master weights (Adam state beside them) and the packed
// BF16 block of kt_mlp.cuh that the tensor-core kernels read.  One training step:
//   train_fb   one warp per 16-sample tile: forward (storing the BF16 activations h_l
//              and SiLU derivatives s_l), MSE loss gradient, backward through the
//              layers (dz_l = (dz_{l+1} W_{l+1}) * s_l), storing dz_l;
//   train_dw   one warp per 16-row block of a weight matrix: dW_l = dz_l^T h_{l-1}
//              summed over the whole batch in a fixed order (deterministic);
//   train_db   bias gradients, fixed-order sums;
//   adam       FP32 Adam on the master weights, then the BF16 repack.
// All products are mma.sync m16n8k16 BF16 x BF16 -> FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <fstream>
#include <random>
#include <string>
#include <vector>

#include "kt_internal.h"
#include "kt_mlp.cuh"

namespace kt {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// FP32 master parameter offsets (floats), unpadded [out][in].
struct Master {
    static constexpr int W1 = 0;                         // [128][16]
    static constexpr int W2 = W1 + kMlpH * kMlpIn;       // [128][128]
    static constexpr int W3 = W2 + kMlpH * kMlpH;
    static constexpr int W4 = W3 + kMlpH * kMlpH;        // [16][128]
    static constexpr int B1 = W4 + kMlpOut * kMlpH;
    static constexpr int B2 = B1 + kMlpH;
    static constexpr int B3 = B2 + kMlpH;
    static constexpr int B4 = B3 + kMlpH;
    static constexpr int N = B4 + kMlpOut;
};

__device__ __forceinline__ float bf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16 *p0, const __nv_bfloat16 *p1)
{
    __nv_bfloat162 v;
    v.x = *p0;
    v.y = *p1;
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// store the 16x(8*NT) accumulator tile as bf16 rows [m][ld]
template <int NT>
__device__ __forceinline__ void store_tile_bf16(__nv_bfloat16 *dst, int ld, const float (&v)[NT][4], int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        *reinterpret_cast<uint32_t *>(dst + g * ld + nt * 8 + 2 * t) = pack_bf16(v[nt][0], v[nt][1]);
        *reinterpret_cast<uint32_t *>(dst + (g + 8) * ld + nt * 8 + 2 * t) = pack_bf16(v[nt][2], v[nt][3]);
    }
}

// dh = dz W for W [n][k] with n the reduction index: B fragment (n pair, column k).
template <int KCN, int NTK>
__device__ __forceinline__ void back_data(const __nv_bfloat16 *W, int kp, int nvalid, const uint32_t (&a)[KCN][4],
                                          float (&acc)[NTK][4], int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NTK; ++nt) {
        acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
        const int k = nt * 8 + g;
#pragma unroll
        for (int kc = 0; kc < KCN; ++kc) {
            const int n0 = kc * 16 + 2 * t, n1 = n0 + 8;
            const __nv_bfloat16 z = __float2bfloat16(0.0f);
            const uint32_t b0 = pack2(n0 < nvalid ? W + n0 * kp + k : &z, n0 + 1 < nvalid ? W + (n0 + 1) * kp + k : &z);
            const uint32_t b1 = pack2(n1 < nvalid ? W + n1 * kp + k : &z, n1 + 1 < nvalid ? W + (n1 + 1) * kp + k : &z);
            mma_bf16(acc[nt], a[kc], b0, b1);
        }
    }
}

template <int NT>
__device__ __forceinline__ void repack(const float (&v)[NT][4], uint32_t (&a)[NT / 2][4])
{
#pragma unroll
    for (int j = 0; j < NT / 2; ++j) {
        a[j][0] = pack_bf16(v[2 * j][0], v[2 * j][1]);
        a[j][1] = pack_bf16(v[2 * j][2], v[2 * j][3]);
        a[j][2] = pack_bf16(v[2 * j + 1][0], v[2 * j + 1][1]);
        a[j][3] = pack_bf16(v[2 * j + 1][2], v[2 * j + 1][3]);
    }
}

struct TrainBufs {
    const unsigned char *P;          // packed bf16 parameters
    const float *X, *Tg;             // [B][16], [B][16]
    __nv_bfloat16 *H0, *H1, *H2, *H3;  // activations: H0 [B][16], H1..H3 [B][128]
    __nv_bfloat16 *S1, *S2, *S3;     // SiLU derivatives [B][128]
    __nv_bfloat16 *D1, *D2, *D3, *D4;  // dz: D1..D3 [B][128], D4 [B][16]
    double *loss;
    int B, nout;
};

// forward + backward-data of one 16-sample tile per warp
__global__ void __launch_bounds__(128) train_fb(const TrainBufs tb)
{
    const int lane = threadIdx.x & 31;
    const long long tile = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const long long m0 = tile * 16;
    if (m0 >= tb.B) return;
    const int g = lane >> 2, t = lane & 3;
    const float invB = 1.0f / static_cast<float>(tb.B);
    // input fragment straight from X (rows beyond B are zero)
    auto xin = [&](long long m, int k) -> float { return m < tb.B ? tb.X[m * kMlpIn + k] : 0.0f; };
    uint32_t a0[1][4];
    a0[0][0] = pack_bf16(xin(m0 + g, 2 * t), xin(m0 + g, 2 * t + 1));
    a0[0][1] = pack_bf16(xin(m0 + g + 8, 2 * t), xin(m0 + g + 8, 2 * t + 1));
    a0[0][2] = pack_bf16(xin(m0 + g, 8 + 2 * t), xin(m0 + g, 9 + 2 * t));
    a0[0][3] = pack_bf16(xin(m0 + g + 8, 8 + 2 * t), xin(m0 + g + 8, 9 + 2 * t));
    {   // H0 = bf16(X)
        __nv_bfloat16 *h0 = tb.H0 + m0 * kMlpIn;
        *reinterpret_cast<uint32_t *>(h0 + g * kMlpIn + 2 * t) = a0[0][0];
        *reinterpret_cast<uint32_t *>(h0 + (g + 8) * kMlpIn + 2 * t) = a0[0][1];
        *reinterpret_cast<uint32_t *>(h0 + g * kMlpIn + 8 + 2 * t) = a0[0][2];
        *reinterpret_cast<uint32_t *>(h0 + (g + 8) * kMlpIn + 8 + 2 * t) = a0[0][3];
    }
    uint32_t a1[8][4], a2[8][4], a3[8][4];
    float acc[16][4], sg[16][4];
    // layer 1
    mlp_hidden<1>(tb.P, MlpLayout::W1, MlpLayout::B1, kMlpKP1, a0, a1, acc, lane);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) sg[nt][i] = silu_grad_f(acc[nt][i]);
    store_tile_bf16<16>(tb.S1 + m0 * kMlpH, kMlpH, sg, lane);
    // layer 2
    mlp_hidden<8>(tb.P, MlpLayout::W2, MlpLayout::B2, kMlpKP, a1, a2, acc, lane);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) sg[nt][i] = silu_grad_f(acc[nt][i]);
    store_tile_bf16<16>(tb.S2 + m0 * kMlpH, kMlpH, sg, lane);
    // layer 3
    mlp_hidden<8>(tb.P, MlpLayout::W3, MlpLayout::B3, kMlpKP, a2, a3, acc, lane);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) sg[nt][i] = silu_grad_f(acc[nt][i]);
    store_tile_bf16<16>(tb.S3 + m0 * kMlpH, kMlpH, sg, lane);
    // activations h1..h3 (the A fragments) to memory, row-major [m][128]
    auto store_a = [&](__nv_bfloat16 *dst, const uint32_t (&a)[8][4]) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            *reinterpret_cast<uint32_t *>(dst + g * kMlpH + 16 * j + 2 * t) = a[j][0];
            *reinterpret_cast<uint32_t *>(dst + (g + 8) * kMlpH + 16 * j + 2 * t) = a[j][1];
            *reinterpret_cast<uint32_t *>(dst + g * kMlpH + 16 * j + 8 + 2 * t) = a[j][2];
            *reinterpret_cast<uint32_t *>(dst + (g + 8) * kMlpH + 16 * j + 8 + 2 * t) = a[j][3];
        }
    };
    store_a(tb.H1 + m0 * kMlpH, a1);
    store_a(tb.H2 + m0 * kMlpH, a2);
    store_a(tb.H3 + m0 * kMlpH, a3);
    // output and loss gradient dz4 = (out - t) / B (rows beyond B and columns beyond nout: 0)
    float d[kMlpOutTiles][4];
    mlp_out(tb.P, a3, d, lane);
    float dz4[kMlpOutTiles][4];
    double lsum = 0.0;
#pragma unroll
    for (int nt = 0; nt < kMlpOutTiles; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long long m = m0 + g + (i >= 2 ? 8 : 0);
            const int o = nt * 8 + 2 * t + (i & 1);
            float r = 0.0f;
            if (m < tb.B && o < tb.nout) r = d[nt][i] - tb.Tg[m * kMlpOut + o];
            lsum += 0.5 * static_cast<double>(r) * r;
            dz4[nt][i] = r * invB;
        }
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(kFull, lsum, off);
    if (lane == 0) atomicAdd(tb.loss, lsum / tb.B);
    store_tile_bf16<kMlpOutTiles>(tb.D4 + m0 * kMlpOut, kMlpOut, dz4, lane);
    // backward: dh3 = dz4 W4 (reduction over the 16 outputs: one K chunk)
    uint32_t ad4[1][4];
    ad4[0][0] = pack_bf16(dz4[0][0], dz4[0][1]);
    ad4[0][1] = pack_bf16(dz4[0][2], dz4[0][3]);
    ad4[0][2] = pack_bf16(dz4[1][0], dz4[1][1]);
    ad4[0][3] = pack_bf16(dz4[1][2], dz4[1][3]);
    const __nv_bfloat16 *W4 = reinterpret_cast<const __nv_bfloat16 *>(tb.P + MlpLayout::W4);
    const __nv_bfloat16 *W3 = reinterpret_cast<const __nv_bfloat16 *>(tb.P + MlpLayout::W3);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(tb.P + MlpLayout::W2);
    back_data<1, 16>(W4, kMlpKP, kMlpOut, ad4, acc, lane);
    auto times_s = [&](const __nv_bfloat16 *S) {
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            acc[nt][0] *= bf(S + g * kMlpH + nt * 8 + 2 * t);
            acc[nt][1] *= bf(S + g * kMlpH + nt * 8 + 2 * t + 1);
            acc[nt][2] *= bf(S + (g + 8) * kMlpH + nt * 8 + 2 * t);
            acc[nt][3] *= bf(S + (g + 8) * kMlpH + nt * 8 + 2 * t + 1);
        }
    };
    times_s(tb.S3 + m0 * kMlpH);                       // dz3
    store_tile_bf16<16>(tb.D3 + m0 * kMlpH, kMlpH, acc, lane);
    repack<16>(acc, a1);
    back_data<8, 16>(W3, kMlpKP, kMlpH, a1, acc, lane);   // dh2
    times_s(tb.S2 + m0 * kMlpH);                       // dz2
    store_tile_bf16<16>(tb.D2 + m0 * kMlpH, kMlpH, acc, lane);
    repack<16>(acc, a1);
    back_data<8, 16>(W2, kMlpKP, kMlpH, a1, acc, lane);   // dh1
    times_s(tb.S1 + m0 * kMlpH);                       // dz1
    store_tile_bf16<16>(tb.D1 + m0 * kMlpH, kMlpH, acc, lane);
}

// dW[n][k] = sum_m D[m][n] H[m][k] for a 16-row block of n per warp; fixed order.
// D: [B][ldd] bf16, H: [B][ldh] bf16; W output fp32 [nrows][ncols] (unpadded).
template <int NTK>
__device__ void dw_block(const __nv_bfloat16 *D, int ldd, int nrows, const __nv_bfloat16 *H, int ldh, int B,
                         float *G, int ncols, int n0, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    float acc[NTK][4];
#pragma unroll
    for (int nt = 0; nt < NTK; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    auto dget = [&](int m, int n) -> const __nv_bfloat16 * { return (m < B && n < nrows) ? D + static_cast<long long>(m) * ldd + n : &zero; };
    auto hget = [&](int m, int k) -> const __nv_bfloat16 * { return (m < B && k < ncols) ? H + static_cast<long long>(m) * ldh + k : &zero; };
    for (int m0 = 0; m0 < B; m0 += 16) {
        uint32_t a[4];
        a[0] = pack2(dget(m0 + 2 * t, n0 + g), dget(m0 + 2 * t + 1, n0 + g));
        a[1] = pack2(dget(m0 + 2 * t, n0 + g + 8), dget(m0 + 2 * t + 1, n0 + g + 8));
        a[2] = pack2(dget(m0 + 8 + 2 * t, n0 + g), dget(m0 + 9 + 2 * t, n0 + g));
        a[3] = pack2(dget(m0 + 8 + 2 * t, n0 + g + 8), dget(m0 + 9 + 2 * t, n0 + g + 8));
        const uint32_t(&af)[4] = a;
#pragma unroll
        for (int nt = 0; nt < NTK; ++nt) {
            const int k = nt * 8 + g;
            const uint32_t b0 = pack2(hget(m0 + 2 * t, k), hget(m0 + 2 * t + 1, k));
            const uint32_t b1 = pack2(hget(m0 + 8 + 2 * t, k), hget(m0 + 9 + 2 * t, k));
            mma_bf16(acc[nt], af, b0, b1);
        }
    }
#pragma unroll
    for (int nt = 0; nt < NTK; ++nt) {
        const int k = nt * 8 + 2 * t;
        const int r0 = n0 + g, r1 = n0 + g + 8;
        if (r0 < nrows && k < ncols) G[r0 * ncols + k] = acc[nt][0];
        if (r0 < nrows && k + 1 < ncols) G[r0 * ncols + k + 1] = acc[nt][1];
        if (r1 < nrows && k < ncols) G[r1 * ncols + k] = acc[nt][2];
        if (r1 < nrows && k + 1 < ncols) G[r1 * ncols + k + 1] = acc[nt][3];
    }
}

struct DwArgs {
    const __nv_bfloat16 *H0, *H1, *H2, *H3, *D1, *D2, *D3, *D4;
    float *grad;   // Master layout
    int B;
};

// blocks 0..7: W1 rows; 8..15: W2; 16..23: W3; 24: W4 (one warp each)
__global__ void __launch_bounds__(32) train_dw(const DwArgs a)
{
    const int lane = threadIdx.x;
    const int blk = blockIdx.x;
    if (blk < 8) {
        dw_block<2>(a.D1, kMlpH, kMlpH, a.H0, kMlpIn, a.B, a.grad + Master::W1, kMlpIn, blk * 16, lane);
    } else if (blk < 16) {
        dw_block<16>(a.D2, kMlpH, kMlpH, a.H1, kMlpH, a.B, a.grad + Master::W2, kMlpH, (blk - 8) * 16, lane);
    } else if (blk < 24) {
        dw_block<16>(a.D3, kMlpH, kMlpH, a.H2, kMlpH, a.B, a.grad + Master::W3, kMlpH, (blk - 16) * 16, lane);
    } else {
        dw_block<16>(a.D4, kMlpOut, kMlpOut, a.H3, kMlpH, a.B, a.grad + Master::W4, kMlpH, 0, lane);
    }
}

// bias gradients: db_l[n] = sum_m dz_l[m][n], one thread per n, fixed order
__global__ void train_db(const DwArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const __nv_bfloat16 *D;
    int ld, n, off;
    if (i < kMlpH) { D = a.D1; ld = kMlpH; n = i; off = Master::B1; }
    else if (i < 2 * kMlpH) { D = a.D2; ld = kMlpH; n = i - kMlpH; off = Master::B2; }
    else if (i < 3 * kMlpH) { D = a.D3; ld = kMlpH; n = i - 2 * kMlpH; off = Master::B3; }
    else if (i < 3 * kMlpH + kMlpOut) { D = a.D4; ld = kMlpOut; n = i - 3 * kMlpH; off = Master::B4; }
    else return;
    float s = 0.0f;
    for (int m = 0; m < a.B; ++m) s += __bfloat162float(D[static_cast<long long>(m) * ld + n]);
    a.grad[off + n] = s;
}

// Adam on the FP32 masters, then refresh the packed BF16 block; rows of W1 beyond
// the input width and of W4 / b4 beyond nout stay zero.
__global__ void adam(float *p, float *m, float *v, const float *g, unsigned char *P, int step, float lr, int nin,
                     int nout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Master::N) return;
    bool frozen = false;
    if (i < Master::W2) frozen = (i % kMlpIn) >= nin;
    else if (i >= Master::W4 && i < Master::B1) frozen = (i - Master::W4) / kMlpH >= nout;
    else if (i >= Master::B4) frozen = (i - Master::B4) >= nout;
    if (!frozen) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / (1.0f - powf(b1, static_cast<float>(step)));
        const float vh = vi / (1.0f - powf(b2, static_cast<float>(step)));
        p[i] -= lr * mh / (sqrtf(vh) + eps);
    }
    const float x = p[i];
    __nv_bfloat16 *Wb;
    if (i < Master::W2) {
        Wb = reinterpret_cast<__nv_bfloat16 *>(P + MlpLayout::W1) + (i / kMlpIn) * kMlpKP1 + i % kMlpIn;
        *Wb = __float2bfloat16(x);
    } else if (i < Master::W3) {
        const int j = i - Master::W2;
        reinterpret_cast<__nv_bfloat16 *>(P + MlpLayout::W2)[(j / kMlpH) * kMlpKP + j % kMlpH] = __float2bfloat16(x);
    } else if (i < Master::W4) {
        const int j = i - Master::W3;
        reinterpret_cast<__nv_bfloat16 *>(P + MlpLayout::W3)[(j / kMlpH) * kMlpKP + j % kMlpH] = __float2bfloat16(x);
    } else if (i < Master::B1) {
        const int j = i - Master::W4;
        reinterpret_cast<__nv_bfloat16 *>(P + MlpLayout::W4)[(j / kMlpH) * kMlpKP + j % kMlpH] = __float2bfloat16(x);
    } else if (i < Master::B2) {
        reinterpret_cast<float *>(P + MlpLayout::B1)[i - Master::B1] = x;
    } else if (i < Master::B3) {
        reinterpret_cast<float *>(P + MlpLayout::B2)[i - Master::B2] = x;
    } else if (i < Master::B4) {
        reinterpret_cast<float *>(P + MlpLayout::B3)[i - Master::B3] = x;
    } else {
        reinterpret_cast<float *>(P + MlpLayout::B4)[i - Master::B4] = x;
    }
}

// batch inference: X [n][16] -> out [n][8], one warp per 16 rows
__global__ void __launch_bounds__(128) infer(const unsigned char *P, const float *X, float *out, long long n)
{
    const int lane = threadIdx.x & 31;
    const long long m0 = ((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 16;
    if (m0 >= n) return;
    const int g = lane >> 2, t = lane & 3;
    auto xin = [&](long long m, int k) -> float { return m < n ? X[m * kMlpIn + k] : 0.0f; };
    uint32_t a0[1][4];
    a0[0][0] = pack_bf16(xin(m0 + g, 2 * t), xin(m0 + g, 2 * t + 1));
    a0[0][1] = pack_bf16(xin(m0 + g + 8, 2 * t), xin(m0 + g + 8, 2 * t + 1));
    a0[0][2] = pack_bf16(xin(m0 + g, 8 + 2 * t), xin(m0 + g, 9 + 2 * t));
    a0[0][3] = pack_bf16(xin(m0 + g + 8, 8 + 2 * t), xin(m0 + g + 8, 9 + 2 * t));
    float d[kMlpOutTiles][4];
    mlp_forward16(P, a0, d, lane);
    const long long r0 = m0 + g, r1 = m0 + g + 8;
#pragma unroll
    for (int nt = 0; nt < kMlpOutTiles; ++nt) {
        if (r0 < n) {
            out[r0 * kMlpOut + nt * 8 + 2 * t] = d[nt][0];
            out[r0 * kMlpOut + nt * 8 + 2 * t + 1] = d[nt][1];
        }
        if (r1 < n) {
            out[r1 * kMlpOut + nt * 8 + 2 * t] = d[nt][2];
            out[r1 * kMlpOut + nt * 8 + 2 * t + 1] = d[nt][3];
        }
    }
}

}  // namespace
}  // namespace kt

// ------------------------------------------------------------------ host side

namespace {

int mfail(int code, const char *msg)
{
    kt::set_error(msg);
    return code;
}

int mcuda(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    kt::set_error(m.c_str());
    return KT_ECUDA;
}

}  // namespace

struct kt_mlp {
    int nin = 0, nout = 0, device = 0;
    unsigned long long seed = 0;
    int step = 0;
    unsigned char *P = nullptr;                   // packed bf16 block (MlpLayout)
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // masters, Adam, grads
    int cap = 0;                                  // batch capacity of the buffers below
    __nv_bfloat16 *act = nullptr;                 // H0..H3, S1..S3, D1..D4
    double *loss = nullptr;
    std::vector<float> norm = std::vector<float>(kt::MlpLayout::NNORM, 0.0f);

    ~kt_mlp()
    {
        cudaFree(P);
        cudaFree(p);
        cudaFree(m);
        cudaFree(v);
        cudaFree(g);
        cudaFree(act);
        cudaFree(loss);
    }

    int ensure(int B)
    {
        if (B <= cap) return KT_OK;
        cudaFree(act);
        act = nullptr;
        const int Bp = (B + 15) & ~15;
        const size_t per = static_cast<size_t>(kt::kMlpIn) + 3 * kt::kMlpH + 3 * kt::kMlpH + 3 * kt::kMlpH + kt::kMlpOut;
        cudaError_t e = cudaMalloc(&act, per * Bp * sizeof(__nv_bfloat16));
        if (e != cudaSuccess) return mfail(KT_ENOMEM, "kt_mlp: activation buffers");
        cap = Bp;
        return KT_OK;
    }

    kt::TrainBufs bufs(const float *X, const float *T, int B)
    {
        kt::TrainBufs tb{};
        const size_t c = static_cast<size_t>(cap);
        __nv_bfloat16 *q = act;
        tb.H0 = q; q += c * kt::kMlpIn;
        tb.H1 = q; q += c * kt::kMlpH;
        tb.H2 = q; q += c * kt::kMlpH;
        tb.H3 = q; q += c * kt::kMlpH;
        tb.S1 = q; q += c * kt::kMlpH;
        tb.S2 = q; q += c * kt::kMlpH;
        tb.S3 = q; q += c * kt::kMlpH;
        tb.D1 = q; q += c * kt::kMlpH;
        tb.D2 = q; q += c * kt::kMlpH;
        tb.D3 = q; q += c * kt::kMlpH;
        tb.D4 = q;
        tb.P = P;
        tb.X = X;
        tb.Tg = T;
        tb.loss = loss;
        tb.B = B;
        tb.nout = nout;
        return tb;
    }

    // repack the masters into the bf16 block (adam with lr = 0 and no state change)
    int repack_all(cudaStream_t s)
    {
        std::vector<float> h(kt::Master::N);
        cudaError_t e = cudaMemcpy(h.data(), p, h.size() * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return mcuda(e, "kt_mlp repack");
        std::vector<unsigned char> blk(kt::MlpLayout::BYTES, 0);
        auto putw = [&](int off, int kp, int rows, int cols, int moff) {
            for (int r = 0; r < rows; ++r)
                for (int c = 0; c < cols; ++c) {
                    __nv_bfloat16 b = __float2bfloat16(h[moff + r * cols + c]);
                    std::memcpy(blk.data() + off + 2 * (r * kp + c), &b, 2);
                }
        };
        putw(kt::MlpLayout::W1, kt::kMlpKP1, kt::kMlpH, kt::kMlpIn, kt::Master::W1);
        putw(kt::MlpLayout::W2, kt::kMlpKP, kt::kMlpH, kt::kMlpH, kt::Master::W2);
        putw(kt::MlpLayout::W3, kt::kMlpKP, kt::kMlpH, kt::kMlpH, kt::Master::W3);
        putw(kt::MlpLayout::W4, kt::kMlpKP, kt::kMlpOut, kt::kMlpH, kt::Master::W4);
        std::memcpy(blk.data() + kt::MlpLayout::B1, h.data() + kt::Master::B1, 4 * kt::kMlpH);
        std::memcpy(blk.data() + kt::MlpLayout::B2, h.data() + kt::Master::B2, 4 * kt::kMlpH);
        std::memcpy(blk.data() + kt::MlpLayout::B3, h.data() + kt::Master::B3, 4 * kt::kMlpH);
        std::memcpy(blk.data() + kt::MlpLayout::B4, h.data() + kt::Master::B4, 4 * kt::kMlpOut);
        std::memcpy(blk.data() + kt::MlpLayout::NORM, norm.data(), 4 * norm.size());
        e = cudaMemcpyAsync(P, blk.data(), blk.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return mcuda(e, "kt_mlp repack upload");
        return KT_OK;
    }
};

namespace kt {
const unsigned char *mlp_device_block(const kt_mlp *m, int *nin, int *nout, int *device)
{
    if (!m) return nullptr;
    *nin = m->nin;
    *nout = m->nout;
    *device = m->device;
    return m->P;
}
}  // namespace kt

extern "C" {

int kt_mlp_sizes(int *n_master, int *packed_bytes)
{
    if (n_master) *n_master = kt::Master::N;
    if (packed_bytes) *packed_bytes = kt::MlpLayout::BYTES;
    return KT_OK;
}

int kt_mlp_create(int n_in, int n_out, unsigned long long seed, kt_mlp **out)
{
    if (!out || n_in < 1 || n_in > kt::kMlpIn || n_out < 1 || n_out > kt::kMlpOut)
        return mfail(KT_EINVAL, "kt_mlp_create: n_in must be 1..16 and n_out 1..16");
    *out = nullptr;
    kt_mlp *m = new (std::nothrow) kt_mlp();
    if (!m) return mfail(KT_ENOMEM, "kt_mlp_create: out of memory");
    m->nin = n_in;
    m->nout = n_out;
    m->seed = seed;
    cudaGetDevice(&m->device);
    cudaError_t e = cudaMalloc(&m->P, kt::MlpLayout::BYTES);
    if (e == cudaSuccess) e = cudaMalloc(&m->p, kt::Master::N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, kt::Master::N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, kt::Master::N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, kt::Master::N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, kt::Master::N * 4);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, kt::Master::N * 4);
    if (e != cudaSuccess) {
        delete m;
        return mfail(KT_ENOMEM, "kt_mlp_create: device allocation failed");
    }
    // PyTorch-style initialisation U(-1/sqrt(fan_in), 1/sqrt(fan_in)); padding stays 0
    std::vector<float> h(kt::Master::N, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int rows, int cols, int fan_in, int vrows, int vcols) {
        const float bnd = 1.0f / std::sqrt(static_cast<float>(fan_in));
        std::uniform_real_distribution<float> U(-bnd, bnd);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) {
                const float x = U(rng);
                h[off + r * cols + c] = (r < vrows && c < vcols) ? x : 0.0f;
            }
    };
    fill(kt::Master::W1, kt::kMlpH, kt::kMlpIn, n_in, kt::kMlpH, n_in);
    fill(kt::Master::W2, kt::kMlpH, kt::kMlpH, kt::kMlpH, kt::kMlpH, kt::kMlpH);
    fill(kt::Master::W3, kt::kMlpH, kt::kMlpH, kt::kMlpH, kt::kMlpH, kt::kMlpH);
    fill(kt::Master::W4, kt::kMlpOut, kt::kMlpH, kt::kMlpH, n_out, kt::kMlpH);
    fill(kt::Master::B1, 1, kt::kMlpH, n_in, 1, kt::kMlpH);
    fill(kt::Master::B2, 1, kt::kMlpH, kt::kMlpH, 1, kt::kMlpH);
    fill(kt::Master::B3, 1, kt::kMlpH, kt::kMlpH, 1, kt::kMlpH);
    fill(kt::Master::B4, 1, kt::kMlpOut, kt::kMlpH, 1, n_out);
    for (int i = 0; i < 16; ++i) m->norm[16 + i] = 1.0f;
    for (int i = 0; i < 16; ++i) m->norm[48 + i] = 1.0f;
    e = cudaMemcpy(m->p, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete m;
        return mcuda(e, "kt_mlp_create: upload");
    }
    int rc = m->repack_all(nullptr);
    if (rc) {
        delete m;
        return rc;
    }
    *out = m;
    return KT_OK;
}

void kt_mlp_free(kt_mlp *m) { delete m; }

int kt_mlp_set_norm(kt_mlp *m, const float *mu_in, const float *sd_in, const float *mu_out, const float *sd_out)
{
    if (!m || !mu_in || !sd_in || !mu_out || !sd_out) return mfail(KT_EINVAL, "kt_mlp_set_norm: NULL argument");
    for (int i = 0; i < m->nin; ++i) {
        if (!(sd_in[i] > 0)) return mfail(KT_EINVAL, "kt_mlp_set_norm: sd_in must be > 0");
        m->norm[i] = mu_in[i];
        m->norm[16 + i] = sd_in[i];
    }
    for (int i = 0; i < m->nout; ++i) {
        if (!(sd_out[i] > 0)) return mfail(KT_EINVAL, "kt_mlp_set_norm: sd_out must be > 0");
        m->norm[32 + i] = mu_out[i];
        m->norm[48 + i] = sd_out[i];
    }
    cudaError_t e = cudaMemcpy(m->P + kt::MlpLayout::NORM, m->norm.data(), 4 * m->norm.size(), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? KT_OK : mcuda(e, "kt_mlp_set_norm");
}

static int fwd_bwd(kt_mlp *m, const float *X, const float *T, int B, cudaStream_t s)
{
    int rc = m->ensure(B);
    if (rc) return rc;
    kt::TrainBufs tb = m->bufs(X, T, B);
    cudaError_t e = cudaMemsetAsync(m->loss, 0, sizeof(double), s);
    if (e != cudaSuccess) return mcuda(e, "kt_mlp: memset");
    const int tiles = (B + 15) / 16;
    kt::train_fb<<<(tiles + 3) / 4, 128, 0, s>>>(tb);
    kt::DwArgs da{tb.H0, tb.H1, tb.H2, tb.H3, tb.D1, tb.D2, tb.D3, tb.D4, m->g, B};
    kt::train_dw<<<25, 32, 0, s>>>(da);
    kt::train_db<<<(3 * kt::kMlpH + kt::kMlpOut + 127) / 128, 128, 0, s>>>(da);
    e = cudaGetLastError();
    return e == cudaSuccess ? KT_OK : mcuda(e, "kt_mlp: train kernels");
}

int kt_mlp_train_step(kt_mlp *m, const float *X, const float *T, int B, float lr, double *loss, void *stream)
{
    if (!m || !X || !T || B < 1 || !(lr >= 0)) return mfail(KT_EINVAL, "kt_mlp_train_step: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = fwd_bwd(m, X, T, B, s);
    if (rc) return rc;
    ++m->step;
    kt::adam<<<(kt::Master::N + 255) / 256, 256, 0, s>>>(m->p, m->m, m->v, m->g, m->P, m->step, lr, m->nin, m->nout);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mcuda(e, "kt_mlp: adam");
    if (loss) {
        e = cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return mcuda(e, "kt_mlp: loss readback");
    }
    return KT_OK;
}

int kt_mlp_gradients(kt_mlp *m, const float *X, const float *T, int B, float *grads, double *loss, void *stream)
{
    if (!m || !X || !T || B < 1 || !grads) return mfail(KT_EINVAL, "kt_mlp_gradients: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = fwd_bwd(m, X, T, B, s);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(grads, m->g, kt::Master::N * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? KT_OK : mcuda(e, "kt_mlp_gradients");
}

int kt_mlp_forward(const kt_mlp *m, const float *X, float *out, int64_t n, void *stream)
{
    if (!m || !X || !out || n < 0) return mfail(KT_EINVAL, "kt_mlp_forward: bad argument");
    if (n == 0) return KT_OK;
    const long long tiles = (n + 15) / 16;
    kt::infer<<<static_cast<unsigned>((tiles + 3) / 4), 128, 0, static_cast<cudaStream_t>(stream)>>>(m->P, X, out, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KT_OK : mcuda(e, "kt_mlp_forward");
}

int kt_mlp_get_params(const kt_mlp *m, float *master)
{
    if (!m || !master) return mfail(KT_EINVAL, "kt_mlp_get_params: NULL argument");
    cudaError_t e = cudaMemcpy(master, m->p, kt::Master::N * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? KT_OK : mcuda(e, "kt_mlp_get_params");
}

int kt_mlp_set_params(kt_mlp *m, const float *master)
{
    if (!m || !master) return mfail(KT_EINVAL, "kt_mlp_set_params: NULL argument");
    cudaError_t e = cudaMemcpy(m->p, master, kt::Master::N * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mcuda(e, "kt_mlp_set_params");
    return m->repack_all(nullptr);
}

// File: "KTMLP2\0\0", int32 nin, nout, hidden, layers, uint64 seed, int32 step, dtype tag
// (1 = float32 masters), float norm[64], float masters[N].
int kt_mlp_save(const kt_mlp *m, const char *path)
{
    if (!m || !path) return mfail(KT_EINVAL, "kt_mlp_save: NULL argument");
    std::vector<float> h(kt::Master::N);
    cudaError_t e = cudaMemcpy(h.data(), m->p, h.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mcuda(e, "kt_mlp_save");
    std::ofstream f(path, std::ios::binary);
    if (!f) return mfail(KT_EINVAL, "kt_mlp_save: cannot open file");
    const char magic[8] = {'K', 'T', 'M', 'L', 'P', '2', 0, 0};
    const int32_t hdr[4] = {m->nin, m->nout, kt::kMlpH, 4};
    const int32_t tail[2] = {m->step, 1};
    f.write(magic, 8);
    f.write(reinterpret_cast<const char *>(hdr), sizeof hdr);
    f.write(reinterpret_cast<const char *>(&m->seed), 8);
    f.write(reinterpret_cast<const char *>(tail), sizeof tail);
    f.write(reinterpret_cast<const char *>(m->norm.data()), m->norm.size() * 4);
    f.write(reinterpret_cast<const char *>(h.data()), h.size() * 4);
    return f ? KT_OK : mfail(KT_EINVAL, "kt_mlp_save: write failed");
}

int kt_mlp_load_file(const char *path, kt_mlp **out)
{
    if (!path || !out) return mfail(KT_EINVAL, "kt_mlp_load_file: NULL argument");
    *out = nullptr;
    std::ifstream f(path, std::ios::binary);
    if (!f) return mfail(KT_EINVAL, "kt_mlp_load_file: cannot open file");
    char magic[8];
    int32_t hdr[4], tail[2];
    unsigned long long seed = 0;
    std::vector<float> norm(kt::MlpLayout::NNORM), h(kt::Master::N);
    f.read(magic, 8);
    f.read(reinterpret_cast<char *>(hdr), sizeof hdr);
    f.read(reinterpret_cast<char *>(&seed), 8);
    f.read(reinterpret_cast<char *>(tail), sizeof tail);
    f.read(reinterpret_cast<char *>(norm.data()), norm.size() * 4);
    f.read(reinterpret_cast<char *>(h.data()), h.size() * 4);
    if (!f || std::memcmp(magic, "KTMLP2", 6) != 0 || hdr[2] != kt::kMlpH || hdr[3] != 4 || tail[1] != 1)
        return mfail(KT_EPARSE, "kt_mlp_load_file: not a KTMLP2 file of this architecture");
    kt_mlp *m = nullptr;
    int rc = kt_mlp_create(hdr[0], hdr[1], seed, &m);
    if (rc) return rc;
    m->step = tail[0];
    m->norm = norm;
    rc = kt_mlp_set_params(m, h.data());
    if (rc) {
        delete m;
        return rc;
    }
    *out = m;
    return KT_OK;
}

}  // extern "C"

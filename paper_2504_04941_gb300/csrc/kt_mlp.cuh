// kt_mlp.cuh -- the learned-guess MLP: layout and warp-level BF16 tensor-core forward.
//
// Network: in (<= 16 features) -> 128 -> 128 -> 128 -> out (<= 16), SiLU between
// layers.  Weights W_l [n][k] (output-major, the reference convention z = h W^T + b)
// in bfloat16, biases in float; accumulation in float.  Every matrix product is
// mma.sync.m16n8k16 (BF16 in, FP32 accumulate) over 16-row tiles; the accumulator
// fragment of one layer is exactly the A fragment of the next (two adjacent 8-column
// tiles form one 16-wide K chunk), so activations never leave registers.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace kt {

constexpr int kMlpIn = 16;     // padded input width (one K chunk)
constexpr int kMlpH = 128;     // hidden width
constexpr int kMlpOut = 16;    // padded output width (two N tiles)
constexpr int kMlpKP1 = kMlpIn + 8;   // row stride (bf16) of W1: conflict-free B loads
constexpr int kMlpKP = kMlpH + 8;     // row stride (bf16) of W2, W3, W4

// Byte offsets of the packed parameter block (identical in global and shared memory).
struct MlpLayout {
    static constexpr int W1 = 0;                                   // bf16 [128][24]
    static constexpr int W2 = W1 + kMlpH * kMlpKP1 * 2;            // bf16 [128][136]
    static constexpr int W3 = W2 + kMlpH * kMlpKP * 2;             // bf16 [128][136]
    static constexpr int W4 = W3 + kMlpH * kMlpKP * 2;             // bf16 [16][136]
    static constexpr int B1 = W4 + kMlpOut * kMlpKP * 2;           // float [128]
    static constexpr int B2 = B1 + kMlpH * 4;
    static constexpr int B3 = B2 + kMlpH * 4;
    static constexpr int B4 = B3 + kMlpH * 4;                      // float [16]
    static constexpr int NORM = B4 + kMlpOut * 4;                  // float [16 mu][16 sigma][16 mu][16 sigma]
    static constexpr int NNORM = 64;
    static constexpr int BYTES = ((NORM + NNORM * 4) + 15) & ~15;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

// B fragment of W (row stride kp, bf16) for output tile nt and K chunk kc.
__device__ __forceinline__ void b_frag(const __nv_bfloat16 *W, int kp, int nt, int kc, int lane, uint32_t &b0,
                                       uint32_t &b1)
{
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *p = W + (nt * 8 + g) * kp + kc * 16 + 2 * t;
    b0 = *reinterpret_cast<const uint32_t *>(p);
    b1 = *reinterpret_cast<const uint32_t *>(p + 8);
}

// A hidden layer on a 16-row tile: a_in [KC][4] (A fragments over the layer input),
// result: SiLU activations repacked as A fragments a_out [8][4] (128 wide); the
// pre-activations z are returned in acc when the caller wants them.
template <int KC>
__device__ __forceinline__ void mlp_hidden(const unsigned char *P, int woff, int boff, int kp,
                                           const uint32_t (&a_in)[KC][4], uint32_t (&a_out)[8][4],
                                           float (&acc)[16][4], int lane)
{
    const __nv_bfloat16 *W = reinterpret_cast<const __nv_bfloat16 *>(P + woff);
    const float *bias = reinterpret_cast<const float *>(P + boff);
    const int t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const float bl = bias[nt * 8 + 2 * t], bh = bias[nt * 8 + 2 * t + 1];
        acc[nt][0] = bl;
        acc[nt][1] = bh;
        acc[nt][2] = bl;
        acc[nt][3] = bh;
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
            uint32_t b0, b1;
            b_frag(W, kp, nt, kc, lane, b0, b1);
            mma_bf16(acc[nt], a_in[kc], b0, b1);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        a_out[j][0] = pack_bf16(silu_f(acc[2 * j][0]), silu_f(acc[2 * j][1]));
        a_out[j][1] = pack_bf16(silu_f(acc[2 * j][2]), silu_f(acc[2 * j][3]));
        a_out[j][2] = pack_bf16(silu_f(acc[2 * j + 1][0]), silu_f(acc[2 * j + 1][1]));
        a_out[j][3] = pack_bf16(silu_f(acc[2 * j + 1][2]), silu_f(acc[2 * j + 1][3]));
    }
}

constexpr int kMlpOutTiles = kMlpOut / 8;

// Output layer: d = a W4^T + b4 as two 16x8 accumulator fragments (16 outputs).
__device__ __forceinline__ void mlp_out(const unsigned char *P, const uint32_t (&a)[8][4],
                                        float (&d)[kMlpOutTiles][4], int lane)
{
    const __nv_bfloat16 *W = reinterpret_cast<const __nv_bfloat16 *>(P + MlpLayout::W4);
    const float *bias = reinterpret_cast<const float *>(P + MlpLayout::B4);
    const int t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < kMlpOutTiles; ++nt) {
        d[nt][0] = bias[nt * 8 + 2 * t];
        d[nt][1] = bias[nt * 8 + 2 * t + 1];
        d[nt][2] = d[nt][0];
        d[nt][3] = d[nt][1];
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) {
            uint32_t b0, b1;
            b_frag(W, kMlpKP, nt, kc, lane, b0, b1);
            mma_bf16(d[nt], a[kc], b0, b1);
        }
    }
}

// Full forward of one 16-row tile from its input A fragment.
__device__ __forceinline__ void mlp_forward16(const unsigned char *P, const uint32_t (&a0)[1][4],
                                              float (&d)[kMlpOutTiles][4], int lane)
{
    uint32_t a1[8][4], a2[8][4];
    float acc[16][4];
    mlp_hidden<1>(P, MlpLayout::W1, MlpLayout::B1, kMlpKP1, a0, a1, acc, lane);
    mlp_hidden<8>(P, MlpLayout::W2, MlpLayout::B2, kMlpKP, a1, a2, acc, lane);
    mlp_hidden<8>(P, MlpLayout::W3, MlpLayout::B3, kMlpKP, a2, a1, acc, lane);
    mlp_out(P, a1, d, lane);
}

// A fragment of a 16-row tile whose row r's features x[0..nf) live in lane
// (row0 + r); every lane passes its own features.
__device__ __forceinline__ void gather_a(const float (&x)[kMlpIn], int nf, int row0, int lane, uint32_t (&a)[1][4])
{
    const int g = lane >> 2, t = lane & 3;
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.0f;
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) {
        if (k >= nf) break;
        const float lo = __shfl_sync(0xffffffffu, x[k], row0 + g);
        const float hi = __shfl_sync(0xffffffffu, x[k], row0 + g + 8);
        // a0: (g, 2t..2t+1)  a1: (g+8, 2t..2t+1)  a2: (g, 8+2t..)  a3: (g+8, 8+2t..)
        if (k == 2 * t) { v[0] = lo; v[2] = hi; }
        if (k == 2 * t + 1) { v[1] = lo; v[3] = hi; }
        if (k == 8 + 2 * t) { v[4] = lo; v[6] = hi; }
        if (k == 9 + 2 * t) { v[5] = lo; v[7] = hi; }
    }
    a[0][0] = pack_bf16(v[0], v[1]);
    a[0][1] = pack_bf16(v[2], v[3]);
    a[0][2] = pack_bf16(v[4], v[5]);
    a[0][3] = pack_bf16(v[6], v[7]);
}

// Output o (< 16) of row r of the output fragments, delivered to lane row0 + r.
__device__ __forceinline__ float scatter_out(const float (&d)[kMlpOutTiles][4], int o, int row0, int lane)
{
    const int r = lane - row0;
    const int rr = r & 7;
    const int oo = o & 7, nt = o >> 3;
    const int src = rr * 4 + (oo >> 1);
    const float lo = __shfl_sync(0xffffffffu, (oo & 1) ? d[nt][1] : d[nt][0], src);
    const float hi = __shfl_sync(0xffffffffu, (oo & 1) ? d[nt][3] : d[nt][2], src);
    return r < 8 ? lo : hi;
}

}  // namespace kt

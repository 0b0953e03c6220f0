// The learned stand-in for the Ewald real-space force factor
// c(r) = erfc(beta r) + 2 beta r / sqrt(pi) exp(-beta^2 r^2) (Sec. 3.2):
// a multilayer perceptron 1 -> 32 -> 32 -> 1 with SiLU hidden layers.
//
// Parameters (FP32, 1153): W1[32], b1[32], W2[32][32] (row = output unit),
// b2[32], W3[32], b3; input x = (r - c0) * c1 maps [r_min, r_max] to [-1, 1].
//
// Tensor-core evaluation of a tile of 64 distances by one warp: layer 1 and
// the SiLUs on the FP32 pipes, layer 2 (64 x 32 times 32 x 32) as
// mma.sync m16n8k16 BF16 products with FP32 accumulation, layer 3 as FP32
// dot products reduced over the 4 lanes of a quad.  Activations and W2 are
// split into BF16 hi + lo parts and the three products hi*hi + lo*hi +
// hi*lo are accumulated, so the result carries about 16 significant bits
// per operand instead of 8.
//
// Fragment layout (m16n8k16, row.col): lane = 4 g + q.  M-tile t of a
// 64-row tile holds rows 16 t + g and 16 t + 8 + g in lane group g; the
// lane's 8 hidden units (in both layers) are mlp_hidden(m, q), m = 0..7,
// which is exactly the set of A columns (layer 2 inputs) and C columns
// (layer 2 outputs) the lane holds.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace nbc {

constexpr int kMlpH = 32;
constexpr int kMlpW1 = 0, kMlpB1 = 32, kMlpW2 = 64, kMlpB2 = 64 + 32 * 32, kMlpW3 = kMlpB2 + 32,
              kMlpB3 = kMlpW3 + 32;
constexpr int kMlpParams = kMlpB3 + 1;   // 1153

// A network in the per-lane layout of the tile evaluator.
struct MlpTC {
    uint4 bfrag[8][32];   // [u * 2 + s][lane]: W2 fragments {hi b0, hi b1, lo b0, lo b1} of n-tile u, k-step s
    float4 lanec[8][32];  // [c][lane]: c 0,1: W1; 2,3: b1; 4,5: b2; 6,7: W3 of the lane's hidden units m = 0..7
    float b3, c0, c1, pad;
};

// Hidden unit held in slot m (0..7) by a lane with quad position q.
__host__ __device__ constexpr int mlp_hidden(int m, int q) { return (m >> 1) * 8 + 2 * q + (m & 1); }

// SiLU z * logistic(z) = h + h tanh(h), h = z / 2 (the logistic is
// (1 + tanh(z / 2)) / 2), with the hardware's approximate tanh: one
// special-function instruction instead of an exponential and a reciprocal.
// Its relative error (about 2^-11) is below the BF16 hi + lo rounding the
// activations go through next; the force error against the FP64 oracle is
// unchanged (tested).
__device__ __forceinline__ float mlp_silu(float z) {
    float t;
    const float h = 0.5f * z;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
    return *reinterpret_cast<const uint32_t*>(&v);
}

// (a, b) -> packed BF16 pairs hi = bf16(a, b) and lo = bf16(a - hi_a, b - hi_b).
__device__ __forceinline__ void mlp_split(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    hi = bf16x2_bits(h);
    lo = bf16x2_bits(__floats2bfloat162_rn(a - hf.x, b - hf.y));
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Evaluate the network on one m-tile (16 rows) of a 64-row tile: x0 is the
// normalised input of row g (g = lane / 4) and x1 that of row g + 8; on
// return o0, o1 hold the network's values for those rows in all four lanes
// of the quad.  Whole warp, converged.  Callers loop over the four m-tiles
// without unrolling, which bounds the registers live at once.
__device__ __forceinline__ void mlp_mtile(const MlpTC& P, int lane, float x0, float x1, float& o0, float& o1) {
    const unsigned full = 0xffffffffu;
    // A fragments of the two k-steps: regs {row g: m, m+1}, {row g+8: m, m+1},
    // {row g: m+2, m+3}, {row g+8: m+2, m+3} with m = 4 s
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float4 w1 = P.lanec[s][lane], b1 = P.lanec[2 + s][lane];
        mlp_split(mlp_silu(fmaf(w1.x, x0, b1.x)), mlp_silu(fmaf(w1.y, x0, b1.y)), ah[s][0], al[s][0]);
        mlp_split(mlp_silu(fmaf(w1.x, x1, b1.x)), mlp_silu(fmaf(w1.y, x1, b1.y)), ah[s][1], al[s][1]);
        mlp_split(mlp_silu(fmaf(w1.z, x0, b1.z)), mlp_silu(fmaf(w1.w, x0, b1.w)), ah[s][2], al[s][2]);
        mlp_split(mlp_silu(fmaf(w1.z, x1, b1.z)), mlp_silu(fmaf(w1.w, x1, b1.w)), ah[s][3], al[s][3]);
    }
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 b2 = P.lanec[4 + (u >> 1)][lane];
        const float4 w3 = P.lanec[6 + (u >> 1)][lane];
        const float b2a = (u & 1) ? b2.z : b2.x, b2b = (u & 1) ? b2.w : b2.y;
        const float w3a = (u & 1) ? w3.z : w3.x, w3b = (u & 1) ? w3.w : w3.y;
        float d[4] = {b2a, b2b, b2a, b2b};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const uint4 B = P.bfrag[u * 2 + s][lane];
            mma_bf16_16816(d, ah[s][0], ah[s][1], ah[s][2], ah[s][3], B.x, B.y);
            mma_bf16_16816(d, al[s][0], al[s][1], al[s][2], al[s][3], B.x, B.y);
            mma_bf16_16816(d, ah[s][0], ah[s][1], ah[s][2], ah[s][3], B.z, B.w);
        }
        s0 = fmaf(w3a, mlp_silu(d[0]), fmaf(w3b, mlp_silu(d[1]), s0));
        s1 = fmaf(w3a, mlp_silu(d[2]), fmaf(w3b, mlp_silu(d[3]), s1));
    }
    s0 += __shfl_xor_sync(full, s0, 1);
    s1 += __shfl_xor_sync(full, s1, 1);
    s0 += __shfl_xor_sync(full, s0, 2);
    s1 += __shfl_xor_sync(full, s1, 2);
    o0 = s0 + P.b3;
    o1 = s1 + P.b3;
}

}  // namespace nbc

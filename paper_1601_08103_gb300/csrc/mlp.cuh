// mlp.cuh -- device code of the boundary network (include/lee_mlp.h): 16 -> 64 -> 64 -> 1 with
// GELU, BF16 operands on the tensor cores (mma.sync m16n8k16, FP32 accumulation).
//
// One warp owns 16 rows.  Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4):
//   A (16 x 16): reg0 = A[g][2t..2t+1], reg1 = A[g+8][2t..2t+1], reg2 = A[g][2t+8..2t+9],
//                reg3 = A[g+8][2t+8..2t+9]           (two BF16 per 32-bit register, low = first)
//   B (16 x 8):  reg0 = B[2t..2t+1][g],  reg1 = B[2t+8..2t+9][g]
//   C (16 x 8):  c0, c1 = C[g][2t..2t+1],  c2, c3 = C[g+8][2t..2t+1]
// The C fragments of two adjacent 8-column tiles are exactly the A fragment of the next layer's
// 16-wide K chunk, so activations never leave registers between layers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lee {

constexpr int kMlpIn = 16, kMlpHid = 64;
constexpr int kMlpNParam = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1;  // 5313
constexpr int kOffW1 = 0, kOffB1 = 1024, kOffW2 = 1088, kOffB2 = 5184, kOffW3 = 5248, kOffB3 = 5312;

// Packed device weights (one allocation, kMlpPackedBytes).
//   w1[64][16], w2[64][64] (out x in), w2t[64][64] (w2t[n][k] = W2[k][n]), w3[8][64] (row 0 = W3,
//   rows 1..7 zero) in BF16; b1[64], b2[64], b3[1] in FP32.
constexpr int kPkW1 = 0, kPkW2 = 2048, kPkW2T = 10240, kPkW3 = 18432, kPkB1 = 19456, kPkB2 = 19712, kPkB3 = 19968;
constexpr int kMlpPackedBytes = 20480;

struct MlpDev {
    const __nv_bfloat16 *w1, *w2, *w2t, *w3;
    const float *b1, *b2, *b3;
};

inline MlpDev mlp_dev(const void *packed) {
    const char *p = static_cast<const char *>(packed);
    MlpDev d;
    d.w1 = reinterpret_cast<const __nv_bfloat16 *>(p + kPkW1);
    d.w2 = reinterpret_cast<const __nv_bfloat16 *>(p + kPkW2);
    d.w2t = reinterpret_cast<const __nv_bfloat16 *>(p + kPkW2T);
    d.w3 = reinterpret_cast<const __nv_bfloat16 *>(p + kPkW3);
    d.b1 = reinterpret_cast<const float *>(p + kPkB1);
    d.b2 = reinterpret_cast<const float *>(p + kPkB2);
    d.b3 = reinterpret_cast<const float *>(p + kPkB3);
    return d;
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// Two consecutive BF16 values of a weight row as one 32-bit word (generic address: the weights
// may sit in global or in shared memory).
__device__ __forceinline__ uint32_t ldw(const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned int *>(p); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Forward pass of one warp's 16 rows.  ax: A fragment of the input (BF16).  Outputs the two
// rows' results in lanes with t == 0 (y_lo for row g, y_hi for row g + 8), plus, when the
// pointers are given, the FP32 pre-activations z1, z2 in C-fragment layout.
struct MlpFwd {
    float z1[8][4];
    float z2[8][4];
    uint32_t h1[8][2];  // BF16 pairs: [tile][0] = row g, [tile][1] = row g + 8 (cols 8j+2t..)
    uint32_t h2[8][2];
    float y_lo, y_hi;
};

__device__ __forceinline__ void mlp_forward_warp(const MlpDev &W, const uint32_t (&ax)[4], MlpFwd &F) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        F.z1[j][0] = F.z1[j][1] = F.z1[j][2] = F.z1[j][3] = 0.f;
        const __nv_bfloat16 *w = W.w1 + (8 * j + g) * kMlpIn + 2 * t;
        mma16816(F.z1[j], ax, ldw(w), ldw(w + 8));
        const float bb0 = W.b1[8 * j + 2 * t], bb1 = W.b1[8 * j + 2 * t + 1];
        F.z1[j][0] += bb0;
        F.z1[j][1] += bb1;
        F.z1[j][2] += bb0;
        F.z1[j][3] += bb1;
        F.h1[j][0] = pack_bf16(gelu(F.z1[j][0]), gelu(F.z1[j][1]));
        F.h1[j][1] = pack_bf16(gelu(F.z1[j][2]), gelu(F.z1[j][3]));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        F.z2[j][0] = F.z2[j][1] = F.z2[j][2] = F.z2[j][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint32_t a[4] = {F.h1[2 * kk][0], F.h1[2 * kk][1], F.h1[2 * kk + 1][0], F.h1[2 * kk + 1][1]};
            const __nv_bfloat16 *w = W.w2 + (8 * j + g) * kMlpHid + 16 * kk + 2 * t;
            mma16816(F.z2[j], a, ldw(w), ldw(w + 8));
        }
        const float bb0 = W.b2[8 * j + 2 * t], bb1 = W.b2[8 * j + 2 * t + 1];
        F.z2[j][0] += bb0;
        F.z2[j][1] += bb1;
        F.z2[j][2] += bb0;
        F.z2[j][3] += bb1;
        F.h2[j][0] = pack_bf16(gelu(F.z2[j][0]), gelu(F.z2[j][1]));
        F.h2[j][1] = pack_bf16(gelu(F.z2[j][2]), gelu(F.z2[j][3]));
    }
    float z3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t a[4] = {F.h2[2 * kk][0], F.h2[2 * kk][1], F.h2[2 * kk + 1][0], F.h2[2 * kk + 1][1]};
        const __nv_bfloat16 *w = W.w3 + g * kMlpHid + 16 * kk + 2 * t;
        mma16816(z3, a, ldw(w), ldw(w + 8));
    }
    const float b3 = W.b3[0];
    F.y_lo = z3[0] + b3;  // column 0 lives in lanes with t == 0
    F.y_hi = z3[2] + b3;
}

// Copies the forward weights (w1, w2, w3 and the biases: packed bytes [0, kPkW2T) and
// [kPkW3, kMlpPackedBytes)) into a block's shared memory and returns views of them.  All threads
// of the block must call it; it ends with a barrier.
__device__ __forceinline__ MlpDev stage_forward_weights(const MlpDev &G, unsigned char *smem) {
    const uint4 *src0 = reinterpret_cast<const uint4 *>(G.w1);  // w1 | w2 are contiguous
    uint4 *dst0 = reinterpret_cast<uint4 *>(smem);
    for (int k = threadIdx.x; k < kPkW2T / 16; k += blockDim.x) dst0[k] = src0[k];
    const uint4 *src1 = reinterpret_cast<const uint4 *>(G.w3);  // w3 | b1 | b2 | b3 are contiguous
    uint4 *dst1 = reinterpret_cast<uint4 *>(smem + kPkW2T);
    for (int k = threadIdx.x; k < (kMlpPackedBytes - kPkW3) / 16; k += blockDim.x) dst1[k] = src1[k];
    __syncthreads();
    MlpDev S;
    S.w1 = reinterpret_cast<const __nv_bfloat16 *>(smem + kPkW1);
    S.w2 = reinterpret_cast<const __nv_bfloat16 *>(smem + kPkW2);
    S.w2t = G.w2t;  // not used by the forward pass
    S.w3 = reinterpret_cast<const __nv_bfloat16 *>(smem + kPkW2T);
    S.b1 = reinterpret_cast<const float *>(smem + kPkW2T + (kPkB1 - kPkW3));
    S.b2 = reinterpret_cast<const float *>(smem + kPkW2T + (kPkB2 - kPkW3));
    S.b3 = reinterpret_cast<const float *>(smem + kPkW2T + (kPkB3 - kPkW3));
    return S;
}
// Shared memory that stage_forward_weights needs.
constexpr int kStagedWeightBytes = kPkW2T + (kMlpPackedBytes - kPkW3);

// A fragment of 16 rows x 16 inputs held in a row-major FP32 tile in shared memory.
__device__ __forceinline__ void a_frag_from_tile(const float (*tile)[kMlpIn], uint32_t (&a)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    a[0] = pack_bf16(tile[g][2 * t], tile[g][2 * t + 1]);
    a[1] = pack_bf16(tile[g + 8][2 * t], tile[g + 8][2 * t + 1]);
    a[2] = pack_bf16(tile[g][2 * t + 8], tile[g][2 * t + 9]);
    a[3] = pack_bf16(tile[g + 8][2 * t + 8], tile[g + 8][2 * t + 9]);
}

}  // namespace lee

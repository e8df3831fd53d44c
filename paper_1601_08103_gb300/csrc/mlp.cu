// mlp.cu -- the learned boundary network (include/lee_mlp.h): packing, inference, fused
// forward + backward on the tensor cores, deterministic gradient reduction, Adam, and the edge
// strips of the solver state that feed it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/lee_mlp.h"
#include "handles.cuh"
#include "mlp.cuh"
#include "step_launch.cuh"

namespace lee {

constexpr int kMlpWarps = 4;                 // warps per block in the network kernels
constexpr int kChunkRows = 16 * kMlpWarps;   // rows per block and training chunk
constexpr int kMaxTrainBlocks = 128;

// ---------------------------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------------------------

// FP32 parameter vector -> packed BF16 weights + FP32 biases.
__global__ void k_mlp_pack(const float *__restrict__ p, char *__restrict__ packed) {
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(packed + kPkW1);
    __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(packed + kPkW2);
    __nv_bfloat16 *w2t = reinterpret_cast<__nv_bfloat16 *>(packed + kPkW2T);
    __nv_bfloat16 *w3 = reinterpret_cast<__nv_bfloat16 *>(packed + kPkW3);
    float *b1 = reinterpret_cast<float *>(packed + kPkB1);
    float *b2 = reinterpret_cast<float *>(packed + kPkB2);
    float *b3 = reinterpret_cast<float *>(packed + kPkB3);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpNParam + 7 * 64; i += gridDim.x * blockDim.x) {
        if (i >= kMlpNParam) {
            w3[64 + (i - kMlpNParam)] = __float2bfloat16_rn(0.f);  // zero rows 1..7 of the padded W3
            continue;
        }
        const float v = p[i];
        if (i < kOffB1) {
            w1[i - kOffW1] = __float2bfloat16_rn(v);
        } else if (i < kOffW2) {
            b1[i - kOffB1] = v;
        } else if (i < kOffB2) {
            const int r = (i - kOffW2) / kMlpHid, c = (i - kOffW2) % kMlpHid;
            w2[r * kMlpHid + c] = __float2bfloat16_rn(v);
            w2t[c * kMlpHid + r] = __float2bfloat16_rn(v);
        } else if (i < kOffW3) {
            b2[i - kOffB2] = v;
        } else if (i < kOffB3) {
            w3[i - kOffW3] = __float2bfloat16_rn(v);
        } else {
            b3[0] = v;
        }
    }
}

cudaError_t mlp_pack(const float *params_dev, void *packed, cudaStream_t st) {
    k_mlp_pack<<<8, 256, 0, st>>>(params_dev, static_cast<char *>(packed));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// inference on given inputs
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_forward(MlpDev WG, const float *__restrict__ x, long long rows,
                                                                float *__restrict__ y) {
    __shared__ __align__(16) unsigned char wsm[kStagedWeightBytes];
    __shared__ float tile[kMlpWarps][16][kMlpIn];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row0 = ((long long)blockIdx.x * kMlpWarps + warp) * 16;
    for (int e = lane; e < 16 * kMlpIn; e += 32) {
        const long long r = row0 + e / kMlpIn;
        tile[warp][e / kMlpIn][e % kMlpIn] = r < rows ? x[r * kMlpIn + e % kMlpIn] : 0.f;
    }
    const MlpDev W = stage_forward_weights(WG, wsm);  // ends with a block barrier
    uint32_t ax[4];
    a_frag_from_tile(tile[warp], ax);
    MlpFwd F;
    mlp_forward_warp(W, ax, F);
    const int g = lane >> 2, t = lane & 3;
    if (t == 0) {
        if (row0 + g < rows) y[row0 + g] = F.y_lo;
        if (row0 + g + 8 < rows) y[row0 + g + 8] = F.y_hi;
    }
}

// ---------------------------------------------------------------------------------------------
// training: fused forward + backward, per-block partial gradients
// ---------------------------------------------------------------------------------------------
struct TrainSmem {
    __nv_bfloat16 xq[kChunkRows][kMlpIn];
    __nv_bfloat16 h1q[kChunkRows][kMlpHid];
    __nv_bfloat16 dz1q[kChunkRows][kMlpHid];
    __nv_bfloat16 dz2q[kChunkRows][kMlpHid];
    float xin[kMlpWarps][16][kMlpIn];
    // per-warp accumulators (summed in warp order at the end: deterministic)
    float db1[kMlpWarps][kMlpHid], db2[kMlpWarps][kMlpHid], dw3[kMlpWarps][kMlpHid];
    float db3[kMlpWarps], loss[kMlpWarps];
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Sum over the 8 lane groups (lanes with equal t) of a warp.
__device__ __forceinline__ float group_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_train(MlpDev W, const float *__restrict__ x,
                                                              const float *__restrict__ tgt, long long rows,
                                                              float *__restrict__ partial, float *__restrict__ partial_loss) {
    __shared__ TrainSmem sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int i = threadIdx.x; i < kMlpWarps * kMlpHid; i += blockDim.x)
        sm.db1[i / kMlpHid][i % kMlpHid] = sm.db2[i / kMlpHid][i % kMlpHid] = sm.dw3[i / kMlpHid][i % kMlpHid] = 0.f;
    if (threadIdx.x < kMlpWarps) sm.db3[threadIdx.x] = sm.loss[threadIdx.x] = 0.f;
    float accW2[8][4], accW1[2][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) accW2[j][0] = accW2[j][1] = accW2[j][2] = accW2[j][3] = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j) accW1[j][0] = accW1[j][1] = accW1[j][2] = accW1[j][3] = 0.f;
    const float dscale = 2.0f / (float)rows;
    const long long nchunks = (rows + kChunkRows - 1) / kChunkRows;
    __syncthreads();

    for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const long long row0 = chunk * kChunkRows + warp * 16;
        const int lr0 = warp * 16;  // first row of this warp inside the block tile
        // ---- inputs
        for (int e = lane; e < 16 * kMlpIn; e += 32) {
            const long long r = row0 + e / kMlpIn;
            const float v = r < rows ? x[r * kMlpIn + e % kMlpIn] : 0.f;
            sm.xin[warp][e / kMlpIn][e % kMlpIn] = v;
            sm.xq[lr0 + e / kMlpIn][e % kMlpIn] = __float2bfloat16_rn(v);
        }
        __syncwarp();
        uint32_t ax[4];
        a_frag_from_tile(sm.xin[warp], ax);
        // ---- forward
        MlpFwd F;
        mlp_forward_warp(W, ax, F);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            *reinterpret_cast<uint32_t *>(&sm.h1q[lr0 + g][8 * j + 2 * t]) = F.h1[j][0];
            *reinterpret_cast<uint32_t *>(&sm.h1q[lr0 + g + 8][8 * j + 2 * t]) = F.h1[j][1];
        }
        // ---- loss and dy (row g in y_lo, row g + 8 in y_hi of the t == 0 lane of the group)
        const float ylo = __shfl_sync(0xffffffffu, F.y_lo, lane & ~3);
        const float yhi = __shfl_sync(0xffffffffu, F.y_hi, lane & ~3);
        const bool vlo = row0 + g < rows, vhi = row0 + g + 8 < rows;
        const float rlo = vlo ? ylo - tgt[row0 + g] : 0.f;
        const float rhi = vhi ? yhi - tgt[row0 + g + 8] : 0.f;
        const float dylo = dscale * rlo, dyhi = dscale * rhi;
        {
            float l = (t == 0) ? rlo * rlo + rhi * rhi : 0.f;
            l = group_sum(l);
            if (lane == 0) sm.loss[warp] += l;
            float d3 = (t == 0) ? dylo + dyhi : 0.f;
            d3 = group_sum(d3);
            if (lane == 0) sm.db3[warp] += d3;
        }
        // ---- layer 3 weights, dz2 = dy W3 * GELU'(z2) rounded to BF16
        uint32_t dz2p[8][2];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int col = 8 * j + 2 * t + e;
                const float h2lo = e ? bf16_hi(F.h2[j][0]) : bf16_lo(F.h2[j][0]);
                const float h2hi = e ? bf16_hi(F.h2[j][1]) : bf16_lo(F.h2[j][1]);
                const float dw = group_sum(dylo * h2lo + dyhi * h2hi);
                if (g == 0) sm.dw3[warp][col] += dw;
            }
            const float w3a = __bfloat162float(W.w3[8 * j + 2 * t]);
            const float w3b = __bfloat162float(W.w3[8 * j + 2 * t + 1]);
            dz2p[j][0] = pack_bf16(dylo * w3a * gelu_grad(F.z2[j][0]), dylo * w3b * gelu_grad(F.z2[j][1]));
            dz2p[j][1] = pack_bf16(dyhi * w3a * gelu_grad(F.z2[j][2]), dyhi * w3b * gelu_grad(F.z2[j][3]));
            *reinterpret_cast<uint32_t *>(&sm.dz2q[lr0 + g][8 * j + 2 * t]) = dz2p[j][0];
            *reinterpret_cast<uint32_t *>(&sm.dz2q[lr0 + g + 8][8 * j + 2 * t]) = dz2p[j][1];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float v = e ? bf16_hi(dz2p[j][0]) + bf16_hi(dz2p[j][1]) : bf16_lo(dz2p[j][0]) + bf16_lo(dz2p[j][1]);
                const float s = group_sum(v);
                if (g == 0) sm.db2[warp][8 * j + 2 * t + e] += s;
            }
        }
        // ---- dh1 = dz2 W2 (B[k][n] = W2[k][n] = w2t[n][k]); dz1 = dh1 * GELU'(z1) rounded to BF16
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float dh[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t a[4] = {dz2p[2 * kk][0], dz2p[2 * kk][1], dz2p[2 * kk + 1][0], dz2p[2 * kk + 1][1]};
                const __nv_bfloat16 *w = W.w2t + (8 * j + g) * kMlpHid + 16 * kk + 2 * t;
                mma16816(dh, a, ldw(w), ldw(w + 8));
            }
            const uint32_t lo = pack_bf16(dh[0] * gelu_grad(F.z1[j][0]), dh[1] * gelu_grad(F.z1[j][1]));
            const uint32_t hi = pack_bf16(dh[2] * gelu_grad(F.z1[j][2]), dh[3] * gelu_grad(F.z1[j][3]));
            *reinterpret_cast<uint32_t *>(&sm.dz1q[lr0 + g][8 * j + 2 * t]) = lo;
            *reinterpret_cast<uint32_t *>(&sm.dz1q[lr0 + g + 8][8 * j + 2 * t]) = hi;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float v = e ? bf16_hi(lo) + bf16_hi(hi) : bf16_lo(lo) + bf16_lo(hi);
                const float s = group_sum(v);
                if (g == 0) sm.db1[warp][8 * j + 2 * t + e] += s;
            }
        }
        __syncthreads();
        // ---- weight gradients over the block's 64 rows: warp w owns output rows 16w .. 16w + 15
        //      dW2[n][k] = sum_r dz2[r][n] h1[r][k],  dW1[n][k] = sum_r dz1[r][n] x[r][k]
        const int m0 = 16 * warp;
#pragma unroll
        for (int s = 0; s < kChunkRows / 16; ++s) {
            const int r0 = 16 * s;
            uint32_t a2[4], a1[4];
            a2[0] = pack2(sm.dz2q[r0 + 2 * t][m0 + g], sm.dz2q[r0 + 2 * t + 1][m0 + g]);
            a2[1] = pack2(sm.dz2q[r0 + 2 * t][m0 + g + 8], sm.dz2q[r0 + 2 * t + 1][m0 + g + 8]);
            a2[2] = pack2(sm.dz2q[r0 + 2 * t + 8][m0 + g], sm.dz2q[r0 + 2 * t + 9][m0 + g]);
            a2[3] = pack2(sm.dz2q[r0 + 2 * t + 8][m0 + g + 8], sm.dz2q[r0 + 2 * t + 9][m0 + g + 8]);
            a1[0] = pack2(sm.dz1q[r0 + 2 * t][m0 + g], sm.dz1q[r0 + 2 * t + 1][m0 + g]);
            a1[1] = pack2(sm.dz1q[r0 + 2 * t][m0 + g + 8], sm.dz1q[r0 + 2 * t + 1][m0 + g + 8]);
            a1[2] = pack2(sm.dz1q[r0 + 2 * t + 8][m0 + g], sm.dz1q[r0 + 2 * t + 9][m0 + g]);
            a1[3] = pack2(sm.dz1q[r0 + 2 * t + 8][m0 + g + 8], sm.dz1q[r0 + 2 * t + 9][m0 + g + 8]);
#pragma unroll
            for (int jn = 0; jn < 8; ++jn) {
                const uint32_t b0 = pack2(sm.h1q[r0 + 2 * t][8 * jn + g], sm.h1q[r0 + 2 * t + 1][8 * jn + g]);
                const uint32_t b1 = pack2(sm.h1q[r0 + 2 * t + 8][8 * jn + g], sm.h1q[r0 + 2 * t + 9][8 * jn + g]);
                mma16816(accW2[jn], a2, b0, b1);
            }
#pragma unroll
            for (int jn = 0; jn < 2; ++jn) {
                const uint32_t b0 = pack2(sm.xq[r0 + 2 * t][8 * jn + g], sm.xq[r0 + 2 * t + 1][8 * jn + g]);
                const uint32_t b1 = pack2(sm.xq[r0 + 2 * t + 8][8 * jn + g], sm.xq[r0 + 2 * t + 9][8 * jn + g]);
                mma16816(accW1[jn], a1, b0, b1);
            }
        }
        __syncthreads();
    }

    // ---- this block's partial gradient, every parameter written exactly once
    float *out = partial + (long long)blockIdx.x * kMlpNParam;
    const int m0 = 16 * warp;
#pragma unroll
    for (int jn = 0; jn < 8; ++jn) {
        out[kOffW2 + (m0 + g) * kMlpHid + 8 * jn + 2 * t] = accW2[jn][0];
        out[kOffW2 + (m0 + g) * kMlpHid + 8 * jn + 2 * t + 1] = accW2[jn][1];
        out[kOffW2 + (m0 + g + 8) * kMlpHid + 8 * jn + 2 * t] = accW2[jn][2];
        out[kOffW2 + (m0 + g + 8) * kMlpHid + 8 * jn + 2 * t + 1] = accW2[jn][3];
    }
#pragma unroll
    for (int jn = 0; jn < 2; ++jn) {
        out[kOffW1 + (m0 + g) * kMlpIn + 8 * jn + 2 * t] = accW1[jn][0];
        out[kOffW1 + (m0 + g) * kMlpIn + 8 * jn + 2 * t + 1] = accW1[jn][1];
        out[kOffW1 + (m0 + g + 8) * kMlpIn + 8 * jn + 2 * t] = accW1[jn][2];
        out[kOffW1 + (m0 + g + 8) * kMlpIn + 8 * jn + 2 * t + 1] = accW1[jn][3];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kMlpHid; i += blockDim.x) {
        float a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int w = 0; w < kMlpWarps; ++w) {
            a1 += sm.db1[w][i];
            a2 += sm.db2[w][i];
            a3 += sm.dw3[w][i];
        }
        out[kOffB1 + i] = a1;
        out[kOffB2 + i] = a2;
        out[kOffW3 + i] = a3;
    }
    if (threadIdx.x == 0) {
        float b = 0.f, l = 0.f;
        for (int w = 0; w < kMlpWarps; ++w) {
            b += sm.db3[w];
            l += sm.loss[w];
        }
        out[kOffB3] = b;
        partial_loss[blockIdx.x] = l;
    }
}

// grad[i] = sum over blocks of partial[b][i], in block order; loss = sum / rows.
__global__ void k_mlp_grad_reduce(const float *__restrict__ partial, const float *__restrict__ partial_loss, int nblocks,
                                  long long rows, float *__restrict__ grad, float *__restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpNParam) {
        float a = 0.f;
        for (int b = 0; b < nblocks; ++b) a += partial[(long long)b * kMlpNParam + i];
        grad[i] = a;
    }
    if (i == 0 && loss) {
        float l = 0.f;
        for (int b = 0; b < nblocks; ++b) l += partial_loss[b];
        *loss = l / (float)rows;
    }
}

// Adam (bias-corrected) on the FP32 master parameters.
__global__ void k_mlp_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ grad, float lr, float beta1, float beta2, float eps, float corr1,
                           float corr2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpNParam) return;
    const float gr = grad[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gr;
    const float vi = beta2 * v[i] + (1.f - beta2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * corr1) / (sqrtf(vi * corr2) + eps);
}

// ---------------------------------------------------------------------------------------------
// edge strips of D2Q5 population fields (library order 0 rest, 1 +x, 2 -x, 3 +y, 4 -y)
// ---------------------------------------------------------------------------------------------
// Canonical slots of edge e: rest, the velocity along the inward normal (entering), the opposite one
// (leaving), then the two tangential ones; canon(e, j) is the library velocity in slot j: edge 0
// {0,1,2,3,4}, edge 1 {0,2,1,4,3}, edge 2 {0,3,4,2,1}, edge 3 {0,4,3,1,2}.  Packed 3 bits per slot
// in a 16-bit field per edge, two edges per word, so that the lookup is register arithmetic.
constexpr unsigned canon_word(int a, int b, int c, int d, int e) {
    return (unsigned)(a | b << 3 | c << 6 | d << 9 | e << 12);
}
constexpr unsigned kCanon01 = canon_word(0, 1, 2, 3, 4) | canon_word(0, 2, 1, 4, 3) << 16;
constexpr unsigned kCanon23 = canon_word(0, 3, 4, 2, 1) | canon_word(0, 4, 3, 1, 2) << 16;
__host__ __device__ constexpr int canon(int e, int j) {
    return (int)(((e < 2 ? kCanon01 : kCanon23) >> (16 * (e & 1) + 3 * j)) & 7u);
}
// Inward normal of edge e: (1, 0), (-1, 0), (0, 1), (0, -1).
__host__ __device__ constexpr int normal_x(int e) { return (e == 0) - (e == 1); }
__host__ __device__ constexpr int normal_y(int e) { return (e == 2) - (e == 3); }
static_assert(canon(0, 4) == 4 && canon(1, 1) == 2 && canon(1, 3) == 4 && canon(2, 1) == 3 && canon(2, 4) == 1 &&
                  canon(3, 1) == 4 && canon(3, 2) == 3 && canon(3, 4) == 2,
              "canonical edge orders");

struct EdgeRow {
    int e, k, cx, cy;
};

// Row r of the region's border rows -> edge, position along it, and cell.
__device__ __forceinline__ EdgeRow edge_row(int r, int x0, int y0, int nx, int ny) {
    EdgeRow E;
    if (r < ny) { E.e = 0; E.k = r; E.cx = x0; E.cy = y0 + r; }
    else if (r < 2 * ny) { E.e = 1; E.k = r - ny; E.cx = x0 + nx - 1; E.cy = y0 + E.k; }
    else if (r < 2 * ny + nx) { E.e = 2; E.k = r - 2 * ny; E.cx = x0 + E.k; E.cy = y0; }
    else { E.e = 3; E.k = r - 2 * ny - nx; E.cx = x0 + E.k; E.cy = y0 + ny - 1; }
    return E;
}

// 1 / f* of D2Q5 (f* = 1/2 rest, 1/8 moving), exact.
__device__ __forceinline__ float inv_f(int i) { return i == 0 ? 2.f : 8.f; }
// f* itself; x / inv_f(i) == x * f_star(i) exactly (both are powers of two).
__device__ __forceinline__ float f_star(int i) { return i == 0 ? 0.5f : 0.125f; }

// Value k of the strip of border row E (depth d = k / 5 from the edge, canonical slot k % 5), in
// units of f* (x 1/f* for unscaled storage).
template <class T>
__device__ __forceinline__ float strip_value(const T *__restrict__ g, long long pitch, int NX, const EdgeRow &E,
                                             bool scaled, int k) {
    const int d = k / 5, i = canon(E.e, k - 5 * d);
    const int px = E.cx + d * normal_x(E.e), py = E.cy + d * normal_y(E.e);
    float h = (float)Store<T>::load(g[(long long)i * pitch + px + (long long)NX * py]);
    if (!scaled) h *= inv_f(i);
    return h;
}
// Scale of a strip from its 15 values xv[0..14] (slot k = 5 d + j: depth d, canonical slot j), and
// the values divided by it, in place (registers or shared memory); xv[15] = 0 pads the row to the
// mma's K.
__device__ __forceinline__ void strip_finish(float *xv, float &s) {
    float ss = 0.f;
#pragma unroll
    for (int k = 0; k < 15; ++k) ss += xv[k] * xv[k];
    s = fmaxf(sqrtf(ss / 15.f), 1e-30f);
    const float inv = 1.f / s;
#pragma unroll
    for (int k = 0; k < 15; ++k) xv[k] *= inv;
    xv[15] = 0.f;
}
// Strip inputs x[16] and scale s of one border row.
template <class T>
__device__ __forceinline__ void strip_inputs(const T *__restrict__ g, long long pitch, int NX, const EdgeRow &E, bool scaled,
                                             float (&xv)[kMlpIn], float &s) {
#pragma unroll
    for (int k = 0; k < 15; ++k) xv[k] = strip_value<T>(g, pitch, NX, E, scaled, k);
    strip_finish(xv, s);
}

// Training pairs from a batch: one thread per border row of one domain.
template <class T>
__global__ void k_edge_samples(const T *__restrict__ buf, const long long *__restrict__ offset,
                               const long long *__restrict__ pitch, const int *__restrict__ dnx, int ndom, int x0, int y0,
                               int nx, int ny, float *__restrict__ xo, float *__restrict__ to, float *__restrict__ so) {
    const int R = 2 * (nx + ny);
    const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (long long)ndom * R) return;
    const int d = (int)(row / R), r = (int)(row % R);
    const T *g = buf + offset[d];
    const EdgeRow E = edge_row(r, x0, y0, nx, ny);
    float xv[kMlpIn], s;
    strip_inputs<T>(g, pitch[d], dnx[d], E, Store<T>::scaled, xv, s);
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xo[row * kMlpIn + k] = xv[k];
    const int iin = canon(E.e, 1);
    const int ox = E.cx - normal_x(E.e), oy = E.cy - normal_y(E.e);
    float tv = (float)Store<T>::load(g[(long long)iin * pitch[d] + ox + (long long)dnx[d] * oy]);
    if (!Store<T>::scaled) tv *= inv_f(iin);
    to[row] = tv / s;
    if (so) so[row] = s;
}

// Inputs of the border of a single whole grid (no targets).
template <class T>
__global__ void k_edge_inputs(const T *__restrict__ g, long long pitch, int NX, int NY, float *__restrict__ xo,
                              float *__restrict__ so) {
    const int R = 2 * (NX + NY);
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= R) return;
    const EdgeRow E = edge_row(row, 0, 0, NX, NY);
    float xv[kMlpIn], s;
    strip_inputs<T>(g, pitch, NX, E, Store<T>::scaled, xv, s);
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xo[(long long)row * kMlpIn + k] = xv[k];
    if (so) so[row] = s;
}

// The learned boundary of one step: strips of the current post-collision state -> network ->
// entering populations ghost[4][L] (arithmetic type C of the storage).
//
// One block of 8 warps per group of 16 border rows.  The chain of three dependent layers is what
// bounds this work, so the hidden units are split over the warps: warp j computes hidden units
// 8j .. 8j+7 of layers 1 and 2 (one 8-column tile each).  The C fragment of a warp's tile is half
// of the A fragment of k-chunk j/2 of the next layer, and that per-lane layout is the same in
// every warp, so the fragments pass between warps through shared memory as they are.  Warp 0
// runs layer 3 over the four k-chunks in order and applies the passivity bound.  Every tile sees
// the same operations in the same order as in mlp_forward_warp, so the result is the same bit for
// bit.
constexpr int kBoundaryWarps = 8;  // warp j owns hidden units 8j .. 8j+7 of both hidden layers

// Read-only 32-bit load of two consecutive BF16 weights from global memory.
__device__ __forceinline__ uint32_t ldg_w(const __nv_bfloat16 *p) {
    return __ldg(reinterpret_cast<const unsigned int *>(p));
}

// The network over border rows row0 .. row0+15 of one grid; every thread of the block calls it.
// The critical path is one chain per warp: the strip loads (one value per thread: row tid / 16,
// slot tid % 16) and the strip scales (shuffles within the row's 16 lanes), a barrier, layer 1
// (one mma and 4 GELU per lane), a barrier, layer 2 (four mma, 4 GELU), a barrier, layer 3
// (warp 0).  The weight fragments come straight from global memory (L1/L2-resident, shared by
// every block) and are loaded while the strips load, so no staging copy precedes layer 1.
// Returns false in warps 1..7 once layer 2 is done; in warp 0 it returns true, and each lane
// with t = lane % 4 == 0 holds in v[h] the entering population of row row0 + lane/4 + 8h in
// stored units (network output x strip scale x passivity factor, times f* for unscaled storage),
// still in FP32; rows at or beyond 2 (NX + NY) hold 0.
template <class T>
__device__ __forceinline__ bool boundary_rows(const MlpDev &W, const T *__restrict__ g, long long pitch, int NX,
                                              int NY, int row0, float (&v)[2]) {
    static_assert(kBoundaryWarps * 32 == 16 * 16, "one thread per strip value of 16 rows");
    __shared__ float tile[16][kMlpIn];
    __shared__ float sc[16];
    // A fragments of layers 2 and 3: k-chunk kk (hidden units 16kk .. 16kk+15) from warps 2kk, 2kk+1
    __shared__ uint32_t afrag1[4][32][4], afrag2[4][32][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = 2 * (NX + NY);
    const int gq = lane >> 2, t = lane & 3;
    const int j = warp;
    const __nv_bfloat16 *w1p = W.w1 + (8 * j + gq) * kMlpIn + 2 * t;
    const uint32_t w1a = ldg_w(w1p), w1b = ldg_w(w1p + 8);
    uint32_t w2f[4][2];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const __nv_bfloat16 *w = W.w2 + (8 * j + gq) * kMlpHid + 16 * kk + 2 * t;
        w2f[kk][0] = ldg_w(w);
        w2f[kk][1] = ldg_w(w + 8);
    }
    const float b1a = __ldg(W.b1 + 8 * j + 2 * t), b1b = __ldg(W.b1 + 8 * j + 2 * t + 1);
    const float b2a = __ldg(W.b2 + 8 * j + 2 * t), b2b = __ldg(W.b2 + 8 * j + 2 * t + 1);
    {
        // row lr's 16 slots sit in 16 consecutive lanes; each of them sums the squares of the
        // row's values in slot order (strip_finish's arithmetic) and scales its own value
        const int lr = threadIdx.x >> 4, k = threadIdx.x & 15, r = row0 + lr;
        float h = 0.f;
        if (k < 15 && r < R) h = strip_value<T>(g, pitch, NX, edge_row(r, 0, 0, NX, NY), Store<T>::scaled, k);
        float ss = 0.f;
#pragma unroll
        for (int q = 0; q < 15; ++q) {
            const float x = __shfl_sync(0xffffffffu, h, (lane & 16) + q);
            ss += x * x;
        }
        const float s = fmaxf(sqrtf(ss / 15.f), 1e-30f);
        const float inv = 1.f / s;
        tile[lr][k] = h * inv;  // 0 in slot 15 and in rows past the border
        if (k == 0) sc[lr] = r < R ? s : 1.f;
    }
    __syncthreads();  // the scaled strips are in the tile
    // layer 1: tile j
    {
        uint32_t ax[4];
        a_frag_from_tile(tile, ax);
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(z, ax, w1a, w1b);
        z[0] += b1a;
        z[1] += b1b;
        z[2] += b1a;
        z[3] += b1b;
        afrag1[j >> 1][lane][2 * (j & 1)] = pack_bf16(gelu(z[0]), gelu(z[1]));
        afrag1[j >> 1][lane][2 * (j & 1) + 1] = pack_bf16(gelu(z[2]), gelu(z[3]));
    }
    __syncthreads();
    // layer 2: tile j, over the four k-chunks
    {
        float z[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint32_t a[4] = {afrag1[kk][lane][0], afrag1[kk][lane][1], afrag1[kk][lane][2], afrag1[kk][lane][3]};
            mma16816(z, a, w2f[kk][0], w2f[kk][1]);
        }
        z[0] += b2a;
        z[1] += b2b;
        z[2] += b2a;
        z[3] += b2b;
        afrag2[j >> 1][lane][2 * (j & 1)] = pack_bf16(gelu(z[0]), gelu(z[1]));
        afrag2[j >> 1][lane][2 * (j & 1) + 1] = pack_bf16(gelu(z[2]), gelu(z[3]));
    }
    __syncthreads();
    if (warp != 0) return false;
    float z3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t a[4] = {afrag2[kk][lane][0], afrag2[kk][lane][1], afrag2[kk][lane][2], afrag2[kk][lane][3]};
        const __nv_bfloat16 *w = W.w3 + gq * kMlpHid + 16 * kk + 2 * t;
        mma16816(z3, a, ldg_w(w), ldg_w(w + 8));
    }
    const float b3 = __ldg(W.b3);
    const float y_lo = z3[0] + b3, y_hi = z3[2] + b3;  // column 0 lives in lanes with t == 0
    // Passivity bound over the block's 16 border cells: the entering populations may carry at most
    // the weighted energy sum g^2 / f* of the outward populations leaving through the same cells
    // (canonical slot 2 at depth 0 of each strip; entering and leaving velocities share f*).  If
    // the network's predictions exceed it they are scaled down together.  The edge then never adds
    // weighted energy, so with tau >= 1/2 the whole step is L2-stable whatever the network predicts.
    float vin[2], ein = 0.f, eout = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int lr = gq + 8 * h;
        const bool ok = (t == 0) && (row0 + lr < R);
        const float hout = tile[lr][2] * sc[lr];
        vin[h] = ok ? sc[lr] * (h ? y_hi : y_lo) : 0.f;
        ein += vin[h] * vin[h];
        eout += ok ? hout * hout : 0.f;
    }
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
        ein += __shfl_xor_sync(0xffffffffu, ein, off);
        eout += __shfl_xor_sync(0xffffffffu, eout, off);
    }
    float factor = 1.f;
    if (ein > eout) factor = sqrtf(eout / ein);
    // the entering velocity (canonical slot 1) moves, so f* = 1/8 for it
    const float fs = Store<T>::scaled ? 1.f : f_star(canon(0, 1));
#pragma unroll
    for (int h = 0; h < 2; ++h) v[h] = vin[h] * factor * fs;
    return true;
}

// The learned edge's network for one grid: the entering populations ghost[e * L + k] of edge e at
// position k.  Block b takes border rows 16b .. 16b+15 (16 rows = the M of one mma tile).
template <class T>
__global__ void __launch_bounds__(32 * kBoundaryWarps)
    k_mlp_boundary(MlpDev W, const T *__restrict__ g, long long pitch, int NX, int NY,
                   typename Store<T>::C *__restrict__ ghost, int L) {
    using C = typename Store<T>::C;
    const int row0 = blockIdx.x * 16;
    float v[2];
    if (!boundary_rows<T>(W, g, pitch, NX, NY, row0, v)) return;
    const int lane = threadIdx.x & 31;
    if ((lane & 3) != 0) return;
    const int R = 2 * (NX + NY);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = row0 + (lane >> 2) + 8 * h;
        if (r < R) {
            const EdgeRow E = edge_row(r, 0, 0, NX, NY);
            ghost[E.e * L + E.k] = (C)v[h];
        }
    }
}

template <class Fn>
cudaError_t with_store(int storage, Fn &&fn) {
    switch (storage) {
    case LEE_STORE_F64: return fn((double *)nullptr);
    case LEE_STORE_F32: return fn((float *)nullptr);
    case LEE_STORE_F16: return fn((__half *)nullptr);
    case LEE_STORE_BF16: return fn((__nv_bfloat16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

// Called by lee_lbm_step for LEE_BC_OPEN_LEARNED.
cudaError_t launch_mlp_boundary(const void *packed, int storage, const void *g, long long pitch, int NX, int NY, void *ghost,
                                int L, cudaStream_t st) {
    const MlpDev W = mlp_dev(packed);
    const int R = 2 * (NX + NY);
    const int blocks = (R + 15) / 16;  // one block per 16 border rows
    return with_store(storage, [&](auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        using C = typename Store<T>::C;
        // the network's blocks take the SMs before the step's (the network is the longer chain)
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return cudaGetLastError();
        cudaLaunchConfig_t lc{};
        lc.gridDim = dim3(blocks);
        lc.blockDim = dim3(32 * kBoundaryWarps);
        lc.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributePriority;
        at[0].val.priority = hi;
        lc.attrs = at;
        lc.numAttrs = 1;
        return cudaLaunchKernelEx(&lc, k_mlp_boundary<T>, W, static_cast<const T *>(g), pitch, NX, NY,
                                  static_cast<C *>(ghost), L);
    });
}

// ---------------------------------------------------------------------------------------------
// one learned step in one launch
// ---------------------------------------------------------------------------------------------

// The in-grid pulls of border cell (x, y): pre[i] = the stored value of velocity i at (x - c_i),
// 0 where that cell is outside the grid (an entering population, which the network supplies).
template <class S, class T>
__device__ __forceinline__ void border_pulls(const T *__restrict__ src, const GridDesc &gd, int x, int y,
                                             typename Store<T>::C (&pre)[S::Q]) {
    using C = typename Store<T>::C;
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const int xs = x - S::c(i, 0), ys = y - S::c(i, 1);
        pre[i] = (xs >= 0 && xs < gd.nx && ys >= 0 && ys < gd.ny)
                     ? Store<T>::load(src[(long long)i * gd.pitch + (long long)ys * gd.nx + xs])
                     : C(0);
    });
}

// A load served by L2 (not L1, which is not coherent with other SMs' stores within a launch).
template <class C>
__device__ __forceinline__ C load_l2(const C *p) {
    static_assert(sizeof(C) == 8 || sizeof(C) == 4, "entering populations are FP64 or FP32");
    if constexpr (sizeof(C) == 8) {
        const unsigned long long b = __ldcg(reinterpret_cast<const unsigned long long *>(p));
        return __longlong_as_double((long long)b);
    } else {
        return __uint_as_float(__ldcg(reinterpret_cast<const unsigned int *>(p)));
    }
}

// Resident blocks per SM the fused kernel's registers are sized for: those of the one-step kernel
// over the same cells (5 at 48 registers; 3 for the 16-bit vector forms, which need about 72).
template <class T, int V>
constexpr int learned_min_blocks() {
    return sizeof(T) == 2 && V > 1 ? 3 : 5;
}

// One time step of an open 2D grid with the learned edge, in one launch (equal bit for bit to the
// network kernel, k_edge_fixup and the step over the interior cells):
//  - blocks 0 .. nnet-1 each run the network for 16 border rows (boundary_rows) and then write
//    those rows' border cells.  Lanes 16..31 of warp 0 own the cells: they load the cells' in-grid
//    pulls while the strips load, take the entering populations from lanes t == 0 by shuffle,
//    store them into ghost[] and collide (k_edge_fixup's arithmetic);
//  - a corner cell takes the entering populations of two rows, an x-edge one and a y-edge one,
//    possibly in two blocks.  Each of the two lanes swaps its value (FP32, with a flag bit) into
//    the corner's 64-bit slot; the lane that gets the other's value back (the second of the two)
//    empties the slot and writes the corner.  FP64 values do not fit beside the flag: there each
//    lane stores its value, fences and counts one arrival in the slot, and the second arrival of
//    the step (an odd count before it: two arrivals per step from zero) reads the other value
//    from L2.  Nothing waits;
//  - the other blocks run the one-step stream-collide chunks over the interior cells, leaving the
//    border unwritten (OpenEdge::skip_border).
// The network blocks come first in the grid, so they are dispatched first and their dependent
// chain overlaps the interior's memory traffic.
template <class S, class T, int V>
__global__ void __launch_bounds__(32 * kBoundaryWarps, learned_min_blocks<T, V>())
    k_learned_step(MlpDev W, const T *__restrict__ src, T *__restrict__ dst, GridDesc gd,
                   CollideCoef<typename Store<T>::C> cf, OpenEdge<typename Store<T>::C> ob,
                   typename Store<T>::C *__restrict__ ghost, int L, unsigned long long *__restrict__ corner, int nnet) {
    using C = typename Store<T>::C;
    static_assert(32 * kBoundaryWarps == 256, "the interior chunks take 256 threads per block");
    if ((int)blockIdx.x >= nnet) {
        stream_collide_chunk<S, T, V, true>(src, dst, gd, cf, ob,
                                            (long long)(blockIdx.x - nnet) * blockDim.x + threadIdx.x);
        return;
    }
    const int NX = gd.nx, NY = gd.ny, R = 2 * (NX + NY);
    const int row0 = blockIdx.x * 16;
    const int lane = threadIdx.x & 31, lr = (lane - 16) & 15;  // lanes 16..31: row row0 + lr
    const bool own = threadIdx.x >= 16 && threadIdx.x < 32 && row0 + lr < R;
    EdgeRow F{0, 0, 0, 0};
    C pre[S::Q];
    if (own) {
        F = edge_row(row0 + lr, 0, 0, NX, NY);
        border_pulls<S, T>(src, gd, F.cx, F.cy, pre);
    }
    float v[2];
    if (!boundary_rows<T>(W, src, gd.pitch, NX, NY, row0, v)) return;
    // row lr's value sits in lane 4 (lr % 8), slot lr / 8
    const float v0 = __shfl_sync(0xffffffffu, v[0], 4 * (lr & 7));
    const float v1 = __shfl_sync(0xffffffffu, v[1], 4 * (lr & 7));
    if (!own) return;
    const C gv = (C)(lr < 8 ? v0 : v1);
    ghost[F.e * L + F.k] = gv;
    auto pulled = [&](int i, int, int) -> C { return pre[i]; };
    const int kmax = (F.e < 2 ? NY : NX) - 1;
    if (F.k != 0 && F.k != kmax) {
        edge_fixup_cell_from<S, T>(dst, gd, cf, [&](int, int) -> C { return gv; }, pulled, F.cx, F.cy);
        return;
    }
    unsigned long long *slot = corner + (F.cx == 0 ? 0 : 1) + (F.cy == 0 ? 0 : 2);
    if constexpr (sizeof(C) == 4) {
        // the value travels in the exchange: flag bit 32 marks a deposited value
        const unsigned long long prev = atomicExch(slot, (1ULL << 32) | __float_as_uint(gv));
        if ((prev >> 32) == 0ULL) return;  // first of the two: the other row completes the corner
        *slot = 0ULL;                     // empty for the next step (only this lane touches it now)
        const C other = __uint_as_float((unsigned)prev);
        edge_fixup_cell_from<S, T>(dst, gd, cf, [&](int e, int) -> C { return e == F.e ? gv : other; }, pulled,
                                   F.cx, F.cy);
    } else {
        // FP64 values do not fit beside a flag: count arrivals, then read the other value from L2
        __threadfence();
        const unsigned long long before = atomicAdd(slot, 1ULL);
        if ((before & 1ULL) == 0ULL) return;  // the corner's other row completes it
        __threadfence();
        edge_fixup_cell_from<S, T>(
            dst, gd, cf, [&](int e, int k) -> C { return e == F.e ? gv : load_l2(ghost + e * L + k); }, pulled,
            F.cx, F.cy);
    }
}

template <class S, class T, int V>
cudaError_t launch_learned_v(const MlpDev &W, const StepLaunch &L, unsigned long long *corner) {
    using C = typename Store<T>::C;
    GridDesc gd;
    gd.nx = L.nx;
    gd.ny = L.ny;
    gd.nz = 1;
    gd.nxc = L.nx / V;
    gd.nchunks = (long long)gd.nxc * L.ny;
    gd.pitch = L.pitch;
    const CollideCoef<C> cf = make_coef<C>(L.omega, L.coefM, L.coefN);
    OpenEdge<C> ob;
    ob.sponge_w = L.sponge_w;
    ob.sponge_smax = (C)L.sponge_smax;
    ob.ghost = nullptr;  // interior cells never read the entering populations
    ob.ghost_L = 0;
    ob.skip_border = 1;
    const int nnet = (2 * (L.nx + L.ny) + 15) / 16;
    const long long blocks = nnet + (gd.nchunks + 255) / 256;
    k_learned_step<S, T, V><<<(unsigned)blocks, 32 * kBoundaryWarps, 0, L.stream>>>(
        W, static_cast<const T *>(L.src), static_cast<T *>(L.dst), gd, cf, ob, static_cast<C *>(const_cast<void *>(L.ghost)),
        L.ghost_L, corner, nnet);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_learned_s(const MlpDev &W, const StepLaunch &L, unsigned long long *corner) {
    return with_store(L.storage, [&](auto *tp) -> cudaError_t {
        using T = std::remove_pointer_t<decltype(tp)>;
        constexpr int V = vec_width<S, T>();
        if (!L.force_scalar && L.nx % V == 0) return launch_learned_v<S, T, V>(W, L, corner);
        return launch_learned_v<S, T, 1>(W, L, corner);
    });
}

// Called by lee_lbm_step for LEE_BC_OPEN_LEARNED (D2Q5): the whole step
// in one launch of k_learned_step, reading L.src and writing L.dst and the entering populations
// L.ghost[4][L.ghost_L]; corner = the 4 corner slots (zero at create and between launches, or
// even arrival counts for FP64 storage).
cudaError_t launch_learned_step(const void *packed, int set, const StepLaunch &L, unsigned long long *corner) {
    if (!L.ghost || !corner || L.nx < 3 || L.ny < 3 || L.nz != 1) return cudaErrorInvalidValue;
    const MlpDev W = mlp_dev(packed);
    if (set != LEE_D2Q5) return cudaErrorInvalidValue;  // the network is trained on this set only
    return launch_learned_s<D2Q5>(W, L, corner);
}

}  // namespace lee

using namespace lee;

struct lee_mlp {
    int device = 0;
    cudaStream_t st = nullptr;
    float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    void *packed = nullptr;
    float *partial = nullptr, *partial_loss = nullptr;
    long long adam_t = 0;
    bool poisoned = false;
    std::string err;
};

namespace {

#define MCK(mm, call)                                                      \
    do {                                                                   \
        cudaError_t e_ = lee::checked(call);                               \
        if (e_ != cudaSuccess) {                                           \
            (mm)->poisoned = true;                                         \
            (mm)->err = cudaGetErrorString(e_);                            \
            return e_ == cudaErrorMemoryAllocation ? LEE_ERR_OUT_OF_MEMORY : LEE_ERR_CUDA; \
        }                                                                  \
    } while (0)

lee_status menter(lee_mlp *m) {
    if (!m) return LEE_ERR_INVALID_ARGUMENT;
    if (m->poisoned) return LEE_ERR_POISONED;
    if (lee::checked(cudaSetDevice(m->device)) != cudaSuccess) {
        m->poisoned = true;
        m->err = "cudaSetDevice";
        return LEE_ERR_CUDA;
    }
    return LEE_OK;
}

}  // namespace

extern "C" {

lee_status lee_mlp_create(const float *params, void *cuda_stream, lee_mlp **out) {
    if (!out) return LEE_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    lee_mlp *m = new (std::nothrow) lee_mlp();
    if (!m) return LEE_ERR_OUT_OF_MEMORY;
    m->st = static_cast<cudaStream_t>(cuda_stream);
    const size_t pb = sizeof(float) * kMlpNParam;
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaMalloc(&m->p, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->packed, kMlpPackedBytes);
    if (e == cudaSuccess) e = cudaMalloc(&m->partial, pb * kMaxTrainBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&m->partial_loss, sizeof(float) * kMaxTrainBlocks);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, pb, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, pb, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, pb, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->packed, 0, kMlpPackedBytes, m->st);
    if (e == cudaSuccess) {
        if (params)
            e = cudaMemcpyAsync(m->p, params, pb, cudaMemcpyHostToDevice, m->st);
        else
            e = cudaMemsetAsync(m->p, 0, pb, m->st);
    }
    if (e == cudaSuccess) e = mlp_pack(m->p, m->packed, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) {
        lee_mlp_destroy(m);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LEE_ERR_OUT_OF_MEMORY : LEE_ERR_CUDA;
    }
    *out = m;
    return LEE_OK;
}

lee_status lee_mlp_get_params(lee_mlp *m, float *params) {
    lee_status s = menter(m);
    if (s != LEE_OK) return s;
    if (!params) return LEE_ERR_INVALID_ARGUMENT;
    MCK(m, cudaMemcpyAsync(params, m->p, sizeof(float) * kMlpNParam, cudaMemcpyDeviceToHost, m->st));
    MCK(m, cudaStreamSynchronize(m->st));
    return LEE_OK;
}

lee_status lee_mlp_set_params(lee_mlp *m, const float *params) {
    lee_status s = menter(m);
    if (s != LEE_OK) return s;
    if (!params) return LEE_ERR_INVALID_ARGUMENT;
    MCK(m, cudaMemcpyAsync(m->p, params, sizeof(float) * kMlpNParam, cudaMemcpyHostToDevice, m->st));
    MCK(m, mlp_pack(m->p, m->packed, m->st));
    MCK(m, cudaStreamSynchronize(m->st));
    return LEE_OK;
}

lee_status lee_mlp_forward(lee_mlp *m, const float *x, int64_t rows, float *y) {
    lee_status s = menter(m);
    if (s != LEE_OK) return s;
    if (!x || !y || rows < 0) return LEE_ERR_INVALID_ARGUMENT;
    if (rows == 0) return LEE_OK;
    const long long blocks = (rows + kChunkRows - 1) / kChunkRows;
    k_mlp_forward<<<(unsigned)blocks, 32 * kMlpWarps, 0, m->st>>>(mlp_dev(m->packed), x, rows, y);
    MCK(m, cudaGetLastError());
    return LEE_OK;
}

lee_status lee_mlp_loss_grad(lee_mlp *m, const float *x, const float *t, int64_t rows, float *grad, float *loss) {
    lee_status s = menter(m);
    if (s != LEE_OK) return s;
    if (!x || !t || rows < 1) return LEE_ERR_INVALID_ARGUMENT;
    const long long nchunks = (rows + kChunkRows - 1) / kChunkRows;
    const int blocks = (int)(nchunks < kMaxTrainBlocks ? nchunks : kMaxTrainBlocks);
    k_mlp_train<<<blocks, 32 * kMlpWarps, 0, m->st>>>(mlp_dev(m->packed), x, t, rows, m->partial, m->partial_loss);
    MCK(m, cudaGetLastError());
    k_mlp_grad_reduce<<<(kMlpNParam + 255) / 256, 256, 0, m->st>>>(m->partial, m->partial_loss, blocks, rows, m->grad, loss);
    MCK(m, cudaGetLastError());
    if (grad) MCK(m, cudaMemcpyAsync(grad, m->grad, sizeof(float) * kMlpNParam, cudaMemcpyDeviceToDevice, m->st));
    return LEE_OK;
}

lee_status lee_mlp_adam_step(lee_mlp *m, float lr, float beta1, float beta2, float eps) {
    lee_status s = menter(m);
    if (s != LEE_OK) return s;
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return LEE_ERR_INVALID_ARGUMENT;
    m->adam_t++;
    const float corr1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)m->adam_t)));
    const float corr2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)m->adam_t)));
    k_mlp_adam<<<(kMlpNParam + 255) / 256, 256, 0, m->st>>>(m->p, m->m, m->v, m->grad, lr, beta1, beta2, eps, corr1, corr2);
    MCK(m, cudaGetLastError());
    MCK(m, mlp_pack(m->p, m->packed, m->st));
    return LEE_OK;
}

lee_status lee_batch_edge_samples(lee_batch *b, int64_t x0, int64_t y0, int64_t nx, int64_t ny, float *x, float *t,
                                  float *s) {
    if (!b || !x || !t) return LEE_ERR_INVALID_ARGUMENT;
    if (b->poisoned) return LEE_ERR_POISONED;
    if (b->set != LEE_D2Q5) return LEE_ERR_UNSUPPORTED;
    if (nx < 3 || ny < 3 || x0 < 1 || y0 < 1) return LEE_ERR_INVALID_ARGUMENT;
    for (const auto &d : b->doms)
        if (x0 + nx + 1 > d.nx || y0 + ny + 1 > d.ny) return LEE_ERR_INVALID_ARGUMENT;
    cudaSetDevice(b->device);
    std::vector<long long> off(b->count), pit(b->count);
    std::vector<int> dnx(b->count);
    for (int d = 0; d < b->count; ++d) {
        off[d] = b->offset[d];
        pit[d] = b->pitch[d];
        dnx[d] = (int)b->doms[d].nx;
    }
    long long *doff = nullptr, *dpit = nullptr;
    int *ddnx = nullptr;
    cudaError_t e = cudaMallocAsync(&doff, sizeof(long long) * b->count, b->st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dpit, sizeof(long long) * b->count, b->st);
    if (e == cudaSuccess) e = cudaMallocAsync(&ddnx, sizeof(int) * b->count, b->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(doff, off.data(), sizeof(long long) * b->count, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dpit, pit.data(), sizeof(long long) * b->count, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ddnx, dnx.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice, b->st);
    const long long rows = (long long)b->count * 2 * (nx + ny);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((rows + 255) / 256);
        e = with_store(b->storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_edge_samples<T><<<blocks, 256, 0, b->st>>>(static_cast<const T *>(b->buf[b->cur]), doff, dpit, ddnx, b->count,
                                                         (int)x0, (int)y0, (int)nx, (int)ny, x, t, s);
            return cudaGetLastError();
        });
    }
    cudaFreeAsync(doff, b->st);
    cudaFreeAsync(dpit, b->st);
    cudaFreeAsync(ddnx, b->st);
    if (e != cudaSuccess) {
        b->poisoned = true;
        b->err = std::string("edge samples: ") + cudaGetErrorString(e);
        return LEE_ERR_CUDA;
    }
    return LEE_OK;
}

lee_status lee_lbm_edge_inputs(lee_lbm *h, float *x, float *s) {
    if (!h || !x) return LEE_ERR_INVALID_ARGUMENT;
    if (h->poisoned) return LEE_ERR_POISONED;
    if (h->cfg.set != LEE_D2Q5) return LEE_ERR_UNSUPPORTED;
    if (h->cfg.storage == LEE_STORE_SPLIT16 || h->cfg.storage == LEE_STORE_BFP16 || h->slab) return LEE_ERR_UNSUPPORTED;
    if (h->cfg.nx < 3 || h->cfg.ny < 3) return LEE_ERR_INVALID_ARGUMENT;
    cudaSetDevice(h->device);
    const int NX = (int)h->cfg.nx, NY = (int)h->cfg.ny;
    const int R = 2 * (NX + NY);
    cudaError_t e = with_store(h->cfg.storage, [&](auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        k_edge_inputs<T><<<(R + 255) / 256, 256, 0, h->st>>>(static_cast<const T *>(h->buf[h->cur]), h->pitch, NX, NY, x, s);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) {
        h->poisoned = true;
        h->err = std::string("edge inputs: ") + cudaGetErrorString(e);
        return LEE_ERR_CUDA;
    }
    return LEE_OK;
}

lee_status lee_mlp_destroy(lee_mlp *m) {
    if (!m) return LEE_OK;
    cudaSetDevice(m->device);
    if (m->st) cudaStreamSynchronize(m->st);
    cudaFree(m->p);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->packed);
    cudaFree(m->partial);
    cudaFree(m->partial_loss);
    delete m;
    cudaGetLastError();
    return LEE_OK;
}

}  // extern "C"

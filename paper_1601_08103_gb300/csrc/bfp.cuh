// bfp.cuh -- block floating-point storage of the populations (LEE_STORE_BFP16).
//
// The populations g are already deviations from the rest state (F = M (1 + eps g), Sec. 3), so
// they are small numbers that vary smoothly from cell to cell.  BFP16 stores them with 16-bit
// integer mantissas and one shared exponent per block of 8 consecutive cells of one velocity
// array (cells in the flat order x + nx (y + ny z); the pitch is a multiple of 64, so a block
// never straddles two velocity arrays):
//
//   value = (u - 32768) * 2^(e - 127),   u: uint16 (offset binary), e: uint8 per block;
//   e = 0: the whole block is zero;  e = 255: the block held a NaN or Inf and decodes to NaN.
//
// Encoding a block of FP32 values v_k: M = max_k |v_k| = (1 + m / 2^23) 2^(b - 127) (b its biased
// exponent, m its 23 mantissa bits), e = b - 14, plus 1 when m >= 8387840 (that is when
// M 2^(127 - e) would be 32766.5 or more), and e = 0 if that is below 1; then u_k = the
// nearest-even integer to v_k 2^(127 - e), plus 32768.  So M 2^(127 - e) lies in [16383.25, 32766.5)
// and every |u_k - 32768| <= 32766: no rounding overflows 16 bits, the largest value of a block
// keeps 15 bits, and the rounding error is at most 2^(e - 128) <= 2^-15 M (1 + 2^-14), against
// 2^-11 |v| per value for FP16.  Decoding is exact, and encoding decoded values gives them back.
// Both run without the conversion unit:
//   encode: t = fma(v, s, 2^23 + 2^15) rounds v s to an integer whose offset form sits in the low
//           16 bits of t (2^23 <= t < 2^24, spacing 1), s = 2^(127 - e) built from exponent bits;
//           two such halves are packed with one byte permute;
//   decode: f = float with bits 0x4B00'0000 | u = 2^23 + u (one byte permute), then
//           v = fma(f, d, -(2^23 + 2^15) d) = (u - 32768) d with d = 2^(e - 127) (exact).
// Memory: 2 bytes per value plus 1 byte per 8 values: 2.125 bytes, e.g. 29.75 B per D3Q7 lattice
// update against 28 for FP16 and 56 for FP32.  The exponents of a state copy follow its
// mantissas: [q * pitch] uint16, then [q * pitch / 8] uint8.
#pragma once

#include <stdint.h>

#include "kernels.cuh"

namespace lee {

struct Bfp16 {
    unsigned short u;
};
template <>
struct Store<Bfp16> {
    using C = float;
    static constexpr bool scaled = false;  // stores g itself; the exponent adapts per block
};

constexpr int kBfpBlock = 8;
constexpr float kBfpMagic = 8421376.0f;  // 2^23 + 2^15

// Exponent array of a state copy whose mantissas start at g.
template <int Q>
__host__ __device__ __forceinline__ const uint8_t *bfp_exps(const Bfp16 *g, long long pitch) {
    return reinterpret_cast<const uint8_t *>(g + (long long)Q * pitch);
}
template <int Q>
__host__ __device__ __forceinline__ uint8_t *bfp_exps(Bfp16 *g, long long pitch) {
    return reinterpret_cast<uint8_t *>(g + (long long)Q * pitch);
}

// d = 2^(e - 127) from the exponent byte (0 for e = 0, +Inf for e = 255) and -(2^23 + 2^15) d.
struct BfpDec {
    float d, nd;
};
__device__ __forceinline__ BfpDec bfp_dec(unsigned e) {
    const float d = __uint_as_float(e << 23);
    return BfpDec{d, -kBfpMagic * d};
}
// One value from its mantissa bits u (low 16 bits of `bits`, higher bits ignored).
__device__ __forceinline__ float bfp_val(unsigned bits, const BfpDec &k) {
    return fmaf(__uint_as_float(__byte_perm(bits, 0x4B00u, 0x5410u)), k.d, k.nd);
}
// The two values of a packed pair of mantissas (low half first).
__device__ __forceinline__ float bfp_lo(unsigned w, const BfpDec &k) {
    return fmaf(__uint_as_float(__byte_perm(w, 0x4B00u, 0x5410u)), k.d, k.nd);
}
__device__ __forceinline__ float bfp_hi(unsigned w, const BfpDec &k) {
    return fmaf(__uint_as_float(__byte_perm(w, 0x4B00u, 0x5432u)), k.d, k.nd);
}
// Both values of a packed pair with one packed f32x2 fma (each half rounds like fmaf: the same
// bits as bfp_lo / bfp_hi).
__device__ __forceinline__ float2 bfp_pair(unsigned w, const BfpDec &k) {
    const float2 f = make_float2(__uint_as_float(__byte_perm(w, 0x4B00u, 0x5410u)),
                                 __uint_as_float(__byte_perm(w, 0x4B00u, 0x5432u)));
    return __ffma2_rn(f, make_float2(k.d, k.d), make_float2(k.nd, k.nd));
}

// Exponent byte of a block from the largest |v| bit pattern of its values (non-negative floats,
// Inf and NaN order like their bit patterns as unsigned integers).
__device__ __forceinline__ unsigned bfp_exponent(unsigned maxbits) {
    if (maxbits >= 0x7F800000u) return 255u;
    // the biased exponent, plus 1 when the mantissa field is 8387840 or more (= 2^23 - 768: the
    // addition carries into the exponent field exactly then)
    const unsigned b = (maxbits + 768u) >> 23;
    return b > 14u ? b - 14u : 0u;
}
// Encoding scale 2^(127 - e) (0 for an all-zero or non-finite block: every u becomes 32768).
__device__ __forceinline__ float bfp_enc_scale(unsigned e) {
    return (e == 0u || e == 255u) ? 0.0f : __uint_as_float((254u - e) << 23);
}
__device__ __forceinline__ unsigned bfp_pack(float a, float b, float s) {
    const float2 t = __ffma2_rn(make_float2(a, b), make_float2(s, s), make_float2(kBfpMagic, kBfpMagic));
    return __byte_perm(__float_as_uint(t.x), __float_as_uint(t.y), 0x5410u);
}
__device__ __forceinline__ unsigned short bfp_one(float a, float s) {
    return (unsigned short)(__float_as_uint(fmaf(a, s, kBfpMagic)) & 0xFFFFu);
}

// Block exponent of V values per lane, 8 / V lanes per block (consecutive lanes, aligned): every
// lane of those groups must call it together (warp shuffles over the group).  A lane with `live`
// false (it owns no cells: past the grid) counts as zeros, like the cells past the grid that the
// writers of whole blocks pad with.
// The larger of |a| and |b| in magnitude (its sign bit is the xor of the signs), NaN if either is
// NaN: one max.NaN.xorsign.abs instruction.
__device__ __forceinline__ float bfp_maxmag(float a, float b) {
    float d;
    asm("max.NaN.xorsign.abs.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

template <int V>
__device__ __forceinline__ unsigned bfp_block_exponent(const float (&v)[V], bool live) {
    static_assert(V == 1 || V == 2 || V == 4 || V == 8, "8 / V lanes per block");
    float mm = v[0];
#pragma unroll
    for (int k = 1; k < V; ++k) mm = bfp_maxmag(mm, v[k]);
    unsigned m = __float_as_uint(mm) & 0x7FFFFFFFu;
    if (!live) m = 0u;
#pragma unroll
    for (int off = 1; off < kBfpBlock / V; off <<= 1) m = max(m, __shfl_xor_sync(kFull, m, off));
    return bfp_exponent(m);
}

// V decoded values of one lane from its aligned mantissas (p, V * 2 bytes aligned) and the
// exponent byte of their block.
template <int V>
__device__ __forceinline__ void bfp_load_vec(const Bfp16 *__restrict__ p, const uint8_t *__restrict__ ep, float (&out)[V]) {
    const BfpDec k = bfp_dec(__ldg(ep));
    auto put = [&](int j, unsigned w) {
        const float2 v = bfp_pair(w, k);
        out[2 * j] = v.x;
        out[2 * j + 1] = v.y;
    };
    if constexpr (V == 8) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
        put(0, w.x); put(1, w.y); put(2, w.z); put(3, w.w);
    } else if constexpr (V == 4) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        put(0, w.x); put(1, w.y);
    } else if constexpr (V == 2) {
        put(0, __ldg(reinterpret_cast<const unsigned *>(p)));
    } else {
        out[0] = bfp_val(__ldg(reinterpret_cast<const unsigned short *>(p)), k);
    }
}

// One decoded value at element index idx of a state copy (mantissas at g, exponents at ex).
__device__ __forceinline__ float bfp_load1(const Bfp16 *__restrict__ g, const uint8_t *__restrict__ ex, long long idx) {
    return bfp_val(__ldg(reinterpret_cast<const unsigned short *>(g + idx)), bfp_dec(__ldg(ex + (idx >> 3))));
}

// Encodes and stores V values of one lane (block exponent shared with the other 8 / V - 1 lanes
// of its group, all of which must call this together); `store` false for lanes that must take
// part in the shuffles but own no cells (their values count as zeros and are not stored).  The
// first lane of a group writes the exponent byte.
template <int V>
__device__ __forceinline__ void bfp_store_vec(Bfp16 *__restrict__ p, uint8_t *__restrict__ ep, const float (&v)[V],
                                              bool store) {
    const unsigned e = bfp_block_exponent<V>(v, store);
    const float s = bfp_enc_scale(e);
    const int lane = threadIdx.x & 31;
    if (!store) return;
    if constexpr (V == 8) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(bfp_pack(v[0], v[1], s), bfp_pack(v[2], v[3], s),
                                                   bfp_pack(v[4], v[5], s), bfp_pack(v[6], v[7], s));
    } else if constexpr (V == 4) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(bfp_pack(v[0], v[1], s), bfp_pack(v[2], v[3], s));
    } else if constexpr (V == 2) {
        *reinterpret_cast<unsigned *>(p) = bfp_pack(v[0], v[1], s);
    } else {
        *reinterpret_cast<unsigned short *>(p) = bfp_one(v[0], s);
    }
    if ((lane & (kBfpBlock / V - 1)) == 0) *ep = (uint8_t)e;
}

// Element access for the read-only auxiliary kernels: the value at element index idx of a state
// copy starting at g, in the arithmetic type (decoded for BFP16).
template <class S, class T>
__device__ __forceinline__ typename Store<T>::C load_elem(const T *__restrict__ g, long long pitch, long long idx) {
    if constexpr (std::is_same<T, Bfp16>::value) {
        return bfp_load1(g, bfp_exps<S::Q>(g, pitch), idx);
    } else {
        return Store<T>::load(g[idx]);
    }
}

// ---------------------------------------------------------------------------------------------
// one fused pull-stream + collide step on BFP16 storage
// ---------------------------------------------------------------------------------------------
// The FP32 one-step kernel's pulls and collision (stream_collide_chunk), with the loads decoded
// and the stores encoded: one step equals decoding the state, one FP32 step, and encoding the
// result, bit for bit.  V cells per lane: 8 (16-byte mantissa vectors, one block per lane) or 4
// for the 19-velocity set (two lanes per block) when nx is a multiple of 8, else 1 (eight lanes
// per block: chunk = flat cell index, so blocks of 8 cells are 8 aligned lanes).  All 32 lanes of
// a warp call this together; lanes past the grid compute on a clamped chunk and store nothing.
template <class S, int V, bool OPEN>
__device__ __forceinline__ void stream_collide_chunk_bfp(const Bfp16 *__restrict__ src, Bfp16 *__restrict__ dst,
                                                         const GridDesc &gd, const CollideCoef<float> &cf,
                                                         const OpenEdge<float> &ob, long long raw) {
    using C = float;
    const uint8_t *__restrict__ sx = bfp_exps<S::Q>(src, gd.pitch);
    uint8_t *__restrict__ dx = bfp_exps<S::Q>(dst, gd.pitch);
    const bool active = raw < gd.nchunks;
    const long long chunk = active ? raw : gd.nchunks - 1;
    const int lane = threadIdx.x & 31;
    int xc, y, z;
    chunk_coords(chunk, gd, xc, y, z);
    const int x0 = xc * V;
    const bool has_left = (lane > 0) && (xc > 0);
    const bool has_right = (lane < 31) && (xc < gd.nxc - 1);

    C pull[S::Q][V];
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = S::c(i, 0), cy = S::c(i, 1), cz = S::c(i, 2);
        int ys = y - cy, zs = z - cz;
        bool row_out = false;
        if constexpr (cy != 0) {
            if (ys < 0) { if constexpr (OPEN) row_out = true; else ys += gd.ny; }
            if (ys >= gd.ny) { if constexpr (OPEN) row_out = true; else ys -= gd.ny; }
        }
        if constexpr (cz != 0) {
            if (zs < 0) { if constexpr (OPEN) row_out = true; else zs += gd.nz; }
            if (zs >= gd.nz) { if constexpr (OPEN) row_out = true; else zs -= gd.nz; }
        }
        const long long rowi = (long long)i * gd.pitch + ((long long)zs * gd.ny + ys) * gd.nx;
        C v[V];
        if (!row_out) {
            bfp_load_vec<V>(src + rowi + x0, sx + ((rowi + x0) >> 3), v);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = C(0);
        }
        if constexpr (cx == 0) {
#pragma unroll
            for (int k = 0; k < V; ++k) pull[i][k] = v[k];
        } else if constexpr (cx == 1) {
            const C prev = __shfl_up_sync(kFull, v[V - 1], 1);
            C left;
            if (has_left) {
                left = prev;
            } else {
                int xs = x0 - 1;
                bool out = row_out;
                if (xs < 0) { if constexpr (OPEN) out = true; else xs += gd.nx; }
                left = out ? C(0) : bfp_load1(src, sx, rowi + xs);
            }
            pull[i][0] = left;
#pragma unroll
            for (int k = 1; k < V; ++k) pull[i][k] = v[k - 1];
        } else {
            const C next = __shfl_down_sync(kFull, v[0], 1);
            C right;
            if (has_right) {
                right = next;
            } else {
                int xs = x0 + V;
                bool out = row_out;
                if (xs >= gd.nx) { if constexpr (OPEN) out = true; else xs -= gd.nx; }
                right = out ? C(0) : bfp_load1(src, sx, rowi + xs);
            }
#pragma unroll
            for (int k = 0; k < V - 1; ++k) pull[i][k] = v[k + 1];
            pull[i][V - 1] = right;
        }
    });

    C post[S::Q][V];
    // one cell at a time: the packed f32x2 pairs (same bits) measured slower here (D3Q7 384^3:
    // 192 against 196 GLUPS; D3Q19 256^3: 32 against 51, from their registers)
    collide_chunk<S, false>(pull, post, cf);

    if constexpr (OPEN) {
        if (ob.sponge_w > 0) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const C damp = sponge_factor<C>(x0 + k, y, z, gd, S::D, ob.sponge_w, ob.sponge_smax);
#pragma unroll
                for (int i = 0; i < S::Q; ++i) post[i][k] *= damp;
            }
        }
    }

    const long long outi = ((long long)z * gd.ny + y) * gd.nx + x0;
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const long long e = (long long)i * gd.pitch + outi;
        bfp_store_vec<V>(dst + e, dx + (e >> 3), post[i], active);
    });
}

// One block of 256 threads per 2048 cells; three blocks per SM at 78 registers (D3Q7, 8 cells per
// lane).  The kernel is bound by instruction issue (four blocks per SM at 64 registers: the same
// time), so decoding and encoding cost it against FP16: D3Q7 384^3 at 196 GLUPS, 5.8 TB/s in
// algorithmic bytes, against 251 GLUPS for FP16.
template <class S, int V, bool OPEN>
__global__ void __launch_bounds__(256) k_stream_collide_bfp(const Bfp16 *__restrict__ src, Bfp16 *__restrict__ dst,
                                                            GridDesc gd, CollideCoef<float> cf, OpenEdge<float> ob) {
    stream_collide_chunk_bfp<S, V, OPEN>(src, dst, gd, cf, ob, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// K-level 2D tiles (tbk_tile) on BFP16 storage: level 1 decodes S(t) as it pulls it, levels 2 ..
// K-1 stay FP32 in shared memory, level K encodes S(t+K).  So a launch equals decoding the state,
// K FP32 steps and one encoding, bit for bit: the state is rounded to 16 bits once per K steps.
// A lane's 4 cells are half a block (lane pairs share the exponent; nx a multiple of 8).
template <int Q>
struct TileIoBfp {
    using Elem = Bfp16;
    struct Vec {
        uint2 m;     // four mantissas
        unsigned e;  // their block's exponent byte
    };
    struct One {
        unsigned u, e;
    };
    __device__ static __forceinline__ Vec ld4(const Bfp16 *__restrict__ base, long long pitch, long long idx) {
        return Vec{__ldg(reinterpret_cast<const uint2 *>(base + idx)), (unsigned)__ldg(bfp_exps<Q>(base, pitch) + (idx >> 3))};
    }
    __device__ static __forceinline__ One ld1(const Bfp16 *__restrict__ base, long long pitch, long long idx) {
        return One{(unsigned)__ldg(reinterpret_cast<const unsigned short *>(base + idx)),
                   (unsigned)__ldg(bfp_exps<Q>(base, pitch) + (idx >> 3))};
    }
    __device__ static __forceinline__ void cvt4(const Vec &t, float (&v)[4]) {
        const BfpDec k = bfp_dec(t.e);
        const float2 a = bfp_pair(t.m.x, k), b = bfp_pair(t.m.y, k);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ static __forceinline__ float cvt1(const One &t) { return bfp_val(t.u, bfp_dec(t.e)); }
    __device__ static __forceinline__ void st4(Bfp16 *__restrict__ base, long long pitch, long long idx, const float (&v)[4],
                                               bool store) {
        bfp_store_vec<4>(base + idx, bfp_exps<Q>(base, pitch) + (idx >> 3), v, store);
    }
};

}  // namespace lee

// tb3d.cuh -- two time steps per launch (temporal blocking) in 3D for the axis-aligned
// seven-velocity sets (D3Q7 and diatomic D3Q7, Sec. 8.3), periodic grids with nx % 4 == 0.
// The solver uses it for FP32 storage, and for BFP16 storage (bfp.cuh; level 1 then stays in FP32,
// so a launch rounds to the storage once) when LEE_TB_STEPS=2 asks for it: with FP16/BF16, and with
// BFP16's decoding and encoding, this latency-bound tile measured slower than the one-step kernel
// (below; BFP16 on D3Q7 384^3: 124 against 196 GLUPS).
//
// A block of W = TY + 2 warps owns a tile of 128 columns x TY rows and marches through planes
// z0 .. z0 + HZ - 1.  Warp w works on row y = y0 - 1 + w at both levels, lane L on the four
// cells x0 + 4L .. x0 + 4L + 3.  Iteration k:
//   level 1: S(t+1) on plane p1 = z0 - 1 + k, rows y0-1 .. y0+TY (all warps) and the halo
//            columns x0-1 and x0+128 (lanes 0 and 1, one cell each), pulled from S(t) in global
//            memory (each population read once, as in the one-step kernel) and rounded to the
//            storage type, so that it equals a stored state;
//   barrier;
//   level 2: S(t+2) on plane p2 = p1 - 1, rows y0 .. y0+TY-1 (warps 1 .. TY), stored.
// Level 2 at (x, y, p2) pulls each velocity from S(t+1) at (x, y, p2) - c_i.  With only axis
// directions, every pull but +-y comes from the warp's own row:
//   rest, +x, -x   from plane p2 (this warp's level 1 one iteration earlier; the x-neighbours by
//                  warp shuffle, the two tile-edge columns from the halo lanes);
//   +z             from plane p2 - 1 (two iterations earlier);
//   -z             from plane p2 + 1 = p1 (this iteration);
// so they stay in registers.  Only +y (from row y - 1) and -y (from row y + 1) cross warps,
// through a 3-slot shared-memory ring of plane slices: slot k % 3 is written by level 1 of
// iteration k, read by level 2 of iteration k + 1, and rewritten by level 1 of iteration k + 3,
// after the barrier of iteration k + 2 -- one barrier per iteration orders it all.  Results equal
// two single steps bit for bit.  DRAM traffic: one read of S(t) (plus the two halo rows of each
// tile, mostly served from L2 by the neighbouring tiles) and one write of S(t+2) per two steps.
// The level-1 loads of the next plane are issued one iteration ahead into registers, and the
// plane after that is requested into L2, so the load latency overlaps the barrier and level 2.
//
// Measured on GB300 (D3Q7 384^3, GLUPS; one-step kernel: 126 in FP32, 250 in FP16): without any
// prefetch 55-113 (tile heights 6, 8, 14; the loads of each plane exposed), L2 prefetch only 67,
// register prefetch only 195, both 207 in FP32; FP16 with both 183 (instruction bound by the
// conversions and roundings, where the one-step kernel moves half the bytes at the copy peak).
// Resources at TY = 8: 10 warps, 156-161 registers, 30 KB of shared memory, one block per SM;
// 384^3 makes 3 x 48 tiles of 128 x 8 (144 blocks on 152 SMs), each marching all 384 planes.
#pragma once

#include "bfp.cuh"

namespace lee {

constexpr int kT3W = 128;  // tile columns
constexpr int kT3V = 4;    // cells per lane

template <class S>
__host__ __device__ constexpr bool axis_only() {
    for (int i = 0; i < S::Q; ++i) {
        int n = 0;
        for (int a = 0; a < 3; ++a) n += S::c(i, a) * S::c(i, a);
        if (n > 1) return false;
    }
    return S::D == 3 && S::Q == 7;
}

template <class S>
__host__ __device__ constexpr int vel_index(int cx, int cy, int cz) {
    for (int i = 0; i < S::Q; ++i)
        if (S::c(i, 0) == cx && S::c(i, 1) == cy && S::c(i, 2) == cz) return i;
    return -1;
}

template <int TY>
constexpr int t3_smem_bytes() {
    return 3 * (TY + 2) * 2 * kT3W * (int)sizeof(float);
}

// A value rounded to the storage type and widened back: what a stored state holds.
template <class T>
__device__ __forceinline__ float t3_round(float v) {
    if constexpr (std::is_same<T, float>::value) {
        return v;
    } else {
        return Store<T>::load(Store<T>::make(v));
    }
}

constexpr int kT3Rows = 8;  // TY: rows per tile

template <class S, class T, int TY>
__global__ void __launch_bounds__((TY + 2) * 32, 1) k_stream_collide_3d2(const T *__restrict__ src, T *__restrict__ dst,
                                                                       int nx, int ny, int nz, long long pitch, int HZ,
                                                                       CollideCoef<float> cf) {
    static_assert(axis_only<S>(), "the 3D two-step tile needs the seven axis velocities");
    constexpr int Q = S::Q;
    constexpr int W = TY + 2;
    constexpr int iR = vel_index<S>(0, 0, 0), iPX = vel_index<S>(1, 0, 0), iMX = vel_index<S>(-1, 0, 0);
    constexpr int iPY = vel_index<S>(0, 1, 0), iMY = vel_index<S>(0, -1, 0);
    constexpr int iPZ = vel_index<S>(0, 0, 1), iMZ = vel_index<S>(0, 0, -1);
    static_assert(iR >= 0 && iPX >= 0 && iMX >= 0 && iPY >= 0 && iMY >= 0 && iPZ >= 0 && iMZ >= 0, "axis set");
    // ring[slot][row][0: +y, 1: -y][column]
    extern __shared__ __align__(16) float t3_ring[];
    auto ring = [&](int slot, int row, int v) { return t3_ring + ((slot * W + row) * 2 + v) * kT3W; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * kT3W, y0 = blockIdx.y * TY, z0 = blockIdx.z * HZ;
    auto wrap = [](int v, int n) {
        v %= n;
        return v < 0 ? v + n : v;
    };
    const int y = y0 - 1 + warp;  // this warp's row (may lie past ny in the last tile row)
    const int rows[3] = {wrap(y - 1, ny), wrap(y, ny), wrap(y + 1, ny)};  // y-1, y, y+1
    const int xa = wrap(x0 + kT3V * lane, nx);
    const int xedge = wrap(lane == 0 ? x0 - 1 : x0 + kT3W, nx);
    // halo cell: column x0 - 1 for even lanes (lane 0 is the one used), x0 + 128 for odd (lane 1);
    // it pulls velocity i from column xh - c_x = xhp[1 - c_x]
    const int xh = (lane & 1) ? x0 + kT3W : x0 - 1;
    const int xhp[3] = {wrap(xh - 1, nx), wrap(xh, nx), wrap(xh + 1, nx)};
    const long long plane = (long long)nx * ny;

    // level-1 state carried between iterations (FP32 values of the stored type)
    float r1[kT3V], px1[kT3V], mx1[kT3V];  // plane p1 - 1: rest, +x, -x
    float hpx1 = 0.f, hmx1 = 0.f;          // plane p1 - 1: +x of the halo cell (lane 0), -x (lane 1)
    float pz1[kT3V], pz2[kT3V];            // +z of planes p1 - 1 and p1 - 2
#pragma unroll
    for (int e = 0; e < kT3V; ++e) r1[e] = px1[e] = mx1[e] = pz1[e] = pz2[e] = 0.f;

    const int iters = HZ + 2;
    // Level-1 inputs of plane p: the lane's vectors, the tile-edge element (lanes 0 and 31) and
    // the halo cell's pulls; loaded one iteration ahead.  BFP16 keeps them as loaded (mantissas
    // and exponent bytes) and decodes them when the next iteration uses them, so that the loads
    // stay in flight across the barrier.
    constexpr bool kBfp = std::is_same<T, Bfp16>::value;
    struct In {
        float v[Q][kT3V];
        float edge[Q];
        float h[Q];
    };
    struct InBfp {
        uint2 m[Q];
        unsigned e[Q], eu[Q], ee[Q], hu[Q], he[Q];
    };
    using Raw = std::conditional_t<kBfp, InBfp, In>;
    auto load_in = [&](int p, Raw &in) {
        const int pl[3] = {wrap(p - 1, nz), wrap(p, nz), wrap(p + 1, nz)};
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = S::c(i, 0), cy = S::c(i, 1), cz = S::c(i, 2);
            const long long ri = (long long)i * pitch + pl[1 - cz] * plane + (long long)rows[1 - cy] * nx;
            if constexpr (kBfp) {
                const uint8_t *ex = bfp_exps<Q>(src, pitch);
                in.m[i] = __ldg(reinterpret_cast<const uint2 *>(src + ri + xa));
                in.e[i] = __ldg(ex + ((ri + xa) >> 3));
                if constexpr (cx != 0) {
                    if (lane == (cx == 1 ? 0 : 31)) {
                        in.eu[i] = __ldg(reinterpret_cast<const unsigned short *>(src + ri + xedge));
                        in.ee[i] = __ldg(ex + ((ri + xedge) >> 3));
                    }
                }
                if (lane < 2) {  // the halo cell is used by lanes 0 and 1 only
                    in.hu[i] = __ldg(reinterpret_cast<const unsigned short *>(src + ri + xhp[1 - cx]));
                    in.he[i] = __ldg(ex + ((ri + xhp[1 - cx]) >> 3));
                }
            } else {
                const T *rowp = src + ri;
                load_vec<T, kT3V>(rowp + xa, in.v[i]);
                if constexpr (cx != 0) {
                    if (lane == (cx == 1 ? 0 : 31)) in.edge[i] = Store<T>::load(rowp[xedge]);
                }
                in.h[i] = Store<T>::load(rowp[xhp[1 - cx]]);
            }
        });
    };
    auto widen = [&](const Raw &r, In &o) {
        if constexpr (kBfp) {
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = S::c(i, 0);
                const BfpDec k = bfp_dec(r.e[i]);
                const float2 a = bfp_pair(r.m[i].x, k), b = bfp_pair(r.m[i].y, k);
                o.v[i][0] = a.x;
                o.v[i][1] = a.y;
                o.v[i][2] = b.x;
                o.v[i][3] = b.y;
                if constexpr (cx != 0) {
                    if (lane == (cx == 1 ? 0 : 31)) o.edge[i] = bfp_val(r.eu[i], bfp_dec(r.ee[i]));
                }
                o.h[i] = lane < 2 ? bfp_val(r.hu[i], bfp_dec(r.he[i])) : 0.f;
            });
        } else {
            o = r;
        }
    };
    auto prefetch_plane = [&](int p) {
        if ((lane & 7) == 0) {
            const int pl[3] = {wrap(p - 1, nz), wrap(p, nz), wrap(p + 1, nz)};
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cy = S::c(i, 1), cz = S::c(i, 2);
                prefetch_l2(src + (long long)i * pitch + pl[1 - cz] * plane + (long long)rows[1 - cy] * nx + xa);
            });
        }
    };
    Raw nxt;
    load_in(z0 - 1, nxt);
    for (int k = 0; k < iters; ++k) {
        const int p1 = z0 - 1 + k;
        // ---- level 1: plane p1, row y
        In cur;
        widen(nxt, cur);
        if (k + 1 < iters) load_in(p1 + 1, nxt);
        if (k + 2 < iters) prefetch_plane(p1 + 2);
        float pa[Q][kT3V], hin[Q][1];
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = S::c(i, 0);
            const float *v = cur.v[i];
            if constexpr (cx == 0) {
#pragma unroll
                for (int e = 0; e < kT3V; ++e) pa[i][e] = v[e];
            } else if constexpr (cx == 1) {
                float left = __shfl_up_sync(kFull, v[kT3V - 1], 1);
                if (lane == 0) left = cur.edge[i];
                pa[i][0] = left;
#pragma unroll
                for (int e = 1; e < kT3V; ++e) pa[i][e] = v[e - 1];
            } else {
                float right = __shfl_down_sync(kFull, v[0], 1);
                if (lane == 31) right = cur.edge[i];
#pragma unroll
                for (int e = 0; e + 1 < kT3V; ++e) pa[i][e] = v[e + 1];
                pa[i][kT3V - 1] = right;
            }
            hin[i][0] = cur.h[i];
        });
        float post[Q][kT3V], hout[Q][1];
        collide_chunk<S, true>(pa, post, cf);
        collide_chunk<S, true>(hin, hout, cf);
        if constexpr (!kBfp) {  // a stored state (BFP16 keeps level 1 in FP32: one rounding per launch)
#pragma unroll
            for (int i = 0; i < Q; ++i) {
#pragma unroll
                for (int e = 0; e < kT3V; ++e) post[i][e] = t3_round<T>(post[i][e]);
                hout[i][0] = t3_round<T>(hout[i][0]);
            }
        }
        *reinterpret_cast<float4 *>(ring(k % 3, warp, 0) + kT3V * lane) =
            make_float4(post[iPY][0], post[iPY][1], post[iPY][2], post[iPY][3]);
        *reinterpret_cast<float4 *>(ring(k % 3, warp, 1) + kT3V * lane) =
            make_float4(post[iMY][0], post[iMY][1], post[iMY][2], post[iMY][3]);
        __syncthreads();  // level 1 of plane p1 visible; level 2 of plane p1 - 2 done with its slot

        // ---- level 2: plane p2 = p1 - 1, rows y0 .. y0+TY-1 (warp-uniform condition)
        const int p2 = p1 - 1;
        if (k >= 2 && warp >= 1 && warp <= TY) {
            float pb[Q][kT3V];
            const int sp = (k - 1) % 3;
            const float4 a = *reinterpret_cast<const float4 *>(ring(sp, warp - 1, 0) + kT3V * lane);
            const float4 b = *reinterpret_cast<const float4 *>(ring(sp, warp + 1, 1) + kT3V * lane);
            const float left = __shfl_up_sync(kFull, px1[kT3V - 1], 1);
            const float right = __shfl_down_sync(kFull, mx1[0], 1);
            const float hright = __shfl_sync(kFull, hmx1, 1);
#pragma unroll
            for (int e = 0; e < kT3V; ++e) {
                pb[iR][e] = r1[e];
                pb[iPZ][e] = pz2[e];
                pb[iMZ][e] = post[iMZ][e];
            }
            pb[iPX][0] = lane == 0 ? hpx1 : left;
#pragma unroll
            for (int e = 1; e < kT3V; ++e) pb[iPX][e] = px1[e - 1];
#pragma unroll
            for (int e = 0; e + 1 < kT3V; ++e) pb[iMX][e] = mx1[e + 1];
            pb[iMX][kT3V - 1] = lane == 31 ? hright : right;
            pb[iPY][0] = a.x; pb[iPY][1] = a.y; pb[iPY][2] = a.z; pb[iPY][3] = a.w;
            pb[iMY][0] = b.x; pb[iMY][1] = b.y; pb[iMY][2] = b.z; pb[iMY][3] = b.w;
            float out[Q][kT3V];
            collide_chunk<S, true>(pb, out, cf);
            const bool st = y < ny && p2 < nz && x0 + kT3V * lane < nx;
            const long long oi = (long long)p2 * plane + (long long)y * nx + x0 + kT3V * lane;
            if constexpr (kBfp) {  // every lane takes part in the block exponents of its pair
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    const long long e = (long long)i * pitch + oi;
                    bfp_store_vec<kT3V>(dst + e, bfp_exps<Q>(dst, pitch) + (e >> 3), out[i], st);
                });
            } else if (st) {
                T *outp = dst + oi;
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    store_vec<T, kT3V>(outp + (long long)i * pitch, out[i]);
                });
            }
        }
        // ---- carry level 1 of plane p1 to the next iteration
#pragma unroll
        for (int e = 0; e < kT3V; ++e) {
            r1[e] = post[iR][e];
            px1[e] = post[iPX][e];
            mx1[e] = post[iMX][e];
            pz2[e] = pz1[e];
            pz1[e] = post[iPZ][e];
        }
        hpx1 = hout[iPX][0];
        hmx1 = hout[iMX][0];
    }
}

// ---- host side: resident capacity (set outside any stream capture) and the launch
template <class S, class T, int TY>
int *t3_capacity() {
    static int cap[64] = {0};
    return cap;
}
template <class S, class T, int TY>
cudaError_t t3_prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (t3_capacity<S, T, TY>()[dev]) return cudaSuccess;
    constexpr int smem = t3_smem_bytes<TY>();
    e = cudaFuncSetAttribute(k_stream_collide_3d2<S, T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_3d2<S, T, TY>, (TY + 2) * 32, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    t3_capacity<S, T, TY>()[dev] = per_sm * sms > 0 ? per_sm * sms : 1;
    return cudaSuccess;
}
// Tiles of 128 x TY cells cut into z segments so that all blocks are resident in one wave.
template <class S, class T, int TY>
cudaError_t t3_launch(const StepLaunch &L) {
    if (L.open || L.nx % kT3V != 0) return cudaErrorInvalidValue;
    if (std::is_same<T, Bfp16>::value && L.nx % kBfpBlock != 0) return cudaErrorInvalidValue;  // lane pairs = blocks
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || t3_capacity<S, T, TY>()[dev] == 0) return cudaErrorNotReady;  // prepare first
    const int strips = (L.nx + kT3W - 1) / kT3W, ytiles = (L.ny + TY - 1) / TY;
    int zsegs = t3_capacity<S, T, TY>()[dev] / (strips * ytiles);
    if (zsegs < 1) zsegs = 1;
    if (zsegs > L.nz) zsegs = L.nz;
    const int HZ = (L.nz + zsegs - 1) / zsegs;
    const dim3 grid(strips, ytiles, (L.nz + HZ - 1) / HZ);
    const CollideCoef<float> cf = make_coef<float>(L.omega, L.coefM, L.coefN);
    k_stream_collide_3d2<S, T, TY><<<grid, (TY + 2) * 32, t3_smem_bytes<TY>(), L.stream>>>(
        static_cast<const T *>(L.src), static_cast<T *>(L.dst), L.nx, L.ny, L.nz, L.pitch, HZ, cf);
    return cudaGetLastError();
}

}  // namespace lee

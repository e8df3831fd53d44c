// tb3d_tma.cuh -- the 3D two-step tile of tb3d.cuh (D3Q7 and diatomic D3Q7, periodic), fed by
// the Tensor Memory Accelerator instead of per-thread loads.
//
// Same arithmetic and the same on-chip data flow as k_stream_collide_3d2 (tb3d.cuh): a block owns
// 128 columns x TY rows and marches through its z segment; warp w computes level 1 (S(t+1)) on
// row y0 - 1 + w of plane p1 and, for w = 1 .. TY, level 2 (S(t+2)) on the same row of plane
// p1 - 1.  Rest, +-x, +-z stay in the lane's registers between iterations, +-y cross warps
// through a 3-slot shared-memory ring.  What differs is where S(t) comes from:
//   - level-1 inputs: one TMA box per velocity and plane (128 columns x TY + 2 source rows,
//     and for BFP16 the matching box of exponent bytes) lands in an NS-stage shared-memory ring;
//     one elected thread issues the boxes of iteration k + NS as soon as the barrier of
//     iteration k has released its stage, and the row warps wait for a stage on its mbarrier
//     (transaction count).  So several planes are in flight without holding them in registers,
//     and the warps that compute issue no global loads for the bulk of the data;
//   - rows that wrap around y (first and last tile row) come in single-row boxes into two extra
//     row slots per velocity (a box reads zeros beyond the grid, it does not wrap); z wraps in
//     the box coordinate (one plane per box); x never leaves the tile (nx % 128 == 0);
//   - the halo columns x0 - 1 and x0 + 128 of level 1 belong to a dedicated halo warp (one lane
//     per cell, 2 (TY + 2) cells, loads issued one iteration ahead), which passes level 2 the
//     +x / -x values through shared memory; the row warps' lanes 0 and 31 load the one element
//     of S(t) their 4-cell vectors lack (one iteration ahead).
// Results equal those of k_stream_collide_3d2 bit for bit (same operations on the same values):
// two single steps for FP32; decode, two FP32 steps, encode for BFP16.
//
// Preconditions (else the solver keeps the register-fed tile): nx % 128 == 0, ny % TY == 0,
// ny >= 2 TY, pitch % 128 == 0 (so that the BFP16 exponent rows, nx / 8 bytes apart and pitch / 8
// bytes between velocities, are multiples of 16 bytes as tensor-map strides).
//
// Warps: TY + 2 row warps, the halo warp, and a producer warp whose lane 0 issues the boxes.  The
// consumers (row and halo warps) meet at named barrier 1 once per iteration; after it one thread
// releases the stage (mbarrier `empty`) and the producer refills it with the boxes of iteration
// k + NS (mbarrier `full`, transaction count), so the producer stays NS stages ahead on its own.
//
// Failure handling: every wait on an mbarrier is bounded (wait_ns of %globaltimer).  When a
// consumer's wait runs out, the block records it in *wait_flag (mapped host memory the handle
// reads after its next synchronisation) and the consumers leave; the producer, whose own wait for
// a released stage then runs out too, waits (bounded) for its copies still in flight and leaves
// last.  `inject` != 0 announces 16 bytes more than the first stage receives, so that its wait runs
// out: the test of that path, without any fault.
//
// Measured on GB300 (D3Q7 384^3, GLUPS): FP32 166 (three stages) against 217 for the register-fed
// tile, BFP16 105 (four stages) against 125 (register-fed) and 197 (one step per launch); two
// blocks per SM at 88 registers spilled and ran slower (BFP16 84-88).  The stages are not what
// holds it back: the same boxes streamed through the same rings without any arithmetic arrive at
// 8-9 TB/s with one block per SM.  The ten computing warps of the one block per SM that the
// registers allow wait on each other once per plane and on the shared-memory loads right after
// each stage wait (ncu: 40 % issue slots busy, stalls on fixed-latency dependencies, barrier and
// scoreboards), where the register-fed tile has its inputs in registers already.  So the solver
// keeps the register-fed tile and takes this one only when LEE_T3_TMA=1 asks for it.
#pragma once

#include "tb3d.cuh"
#include "tma.cuh"

namespace lee {

// ---- storage policies: the staged row format and the global-memory accesses
// FP32 state: 512-byte rows of 128 floats.
struct T3tIoF32 {
    using Elem = float;
    static constexpr bool kExp = false;
    static constexpr int kValRow = kT3W * 4;
    static constexpr CUtensorMapDataType kType = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    static constexpr bool kRound = false;
    using Raw = float;
    __device__ static __forceinline__ void ld4(const unsigned char *v, const unsigned char *, int lane, float (&o)[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(v + 16 * lane);
        o[0] = t.x;
        o[1] = t.y;
        o[2] = t.z;
        o[3] = t.w;
    }
    __device__ static __forceinline__ Raw ldg1(const float *__restrict__ g, long long, long long idx) {
        return __ldg(g + idx);
    }
    __device__ static __forceinline__ float cvt1(const Raw &r) { return r; }
    __device__ static __forceinline__ float round(float v) { return v; }
    __device__ static __forceinline__ void st4(float *__restrict__ g, long long, long long idx, const float (&v)[4],
                                               bool st) {
        if (st) tb_st(g + idx, v);
    }
};

// BFP16 state: 256-byte rows of 128 mantissas and 16-byte rows of their exponent bytes; level 1
// stays in FP32 (one rounding per launch).
template <int Q>
struct T3tIoBfp {
    using Elem = Bfp16;
    static constexpr bool kExp = true;
    static constexpr int kValRow = kT3W * 2;
    static constexpr CUtensorMapDataType kType = CU_TENSOR_MAP_DATA_TYPE_UINT16;
    static constexpr bool kRound = false;
    struct Raw {
        unsigned u, e;
    };
    __device__ static __forceinline__ void ld4(const unsigned char *v, const unsigned char *ex, int lane,
                                               float (&o)[4]) {
        const uint2 m = *reinterpret_cast<const uint2 *>(v + 8 * lane);
        const BfpDec k = bfp_dec(ex[lane >> 1]);  // cells 4L .. 4L+3 lie in block L / 2
        const float2 a = bfp_pair(m.x, k), b = bfp_pair(m.y, k);
        o[0] = a.x;
        o[1] = a.y;
        o[2] = b.x;
        o[3] = b.y;
    }
    __device__ static __forceinline__ Raw ldg1(const Bfp16 *__restrict__ g, long long pitch, long long idx) {
        return Raw{(unsigned)__ldg(reinterpret_cast<const unsigned short *>(g + idx)),
                   (unsigned)__ldg(bfp_exps<Q>(g, pitch) + (idx >> 3))};
    }
    __device__ static __forceinline__ float cvt1(const Raw &r) { return bfp_val(r.u, bfp_dec(r.e)); }
    __device__ static __forceinline__ float round(float v) { return v; }
    __device__ static __forceinline__ void st4(Bfp16 *__restrict__ g, long long pitch, long long idx, const float (&v)[4],
                                               bool st) {
        bfp_store_vec<kT3V>(g + idx, bfp_exps<Q>(g, pitch) + (idx >> 3), v, st);
    }
};

// ---- shared-memory layout (offsets from a 128-byte aligned base)
// stage s, velocity i: [values: TY + 2 box rows | 2 wrap rows][exponents: box rows | 2 wrap slots]
template <int Q, class IO, int TY, int NS>
struct T3tLayout {
    static constexpr int kRows = TY + 2;
    static constexpr int kValBox = kRows * IO::kValRow;
    static constexpr int kValBytes = (kValBox + 2 * IO::kValRow + 127) / 128 * 128;
    static constexpr int kExpBox = IO::kExp ? (kRows * 16 + 127) / 128 * 128 : 0;
    static constexpr int kExpBytes = IO::kExp ? kExpBox + 2 * 128 : 0;
    static constexpr int kVelBytes = kValBytes + kExpBytes;
    static constexpr int kStageBytes = Q * kVelBytes;
    static constexpr int kRingOff = NS * kStageBytes;
    static constexpr int kRingBytes = 3 * kRows * 2 * kT3W * 4;
    static constexpr int kHaloOff = kRingOff + kRingBytes;
    static constexpr int kHaloBytes = (3 * kRows * 2 * 4 + 15) / 16 * 16;
    static constexpr int kBarOff = kHaloOff + kHaloBytes;
    static constexpr int kBytes = kBarOff + 2 * NS * 8 + 16 + 128;  // full, empty, abort; + base alignment
    // transaction bytes: one velocity's boxes, one wrapped row
    static constexpr unsigned kBoxTx = kRows * (IO::kValRow + (IO::kExp ? 16 : 0));
    static constexpr unsigned kRowTx = IO::kValRow + (IO::kExp ? 16 : 0);
};

// MINB blocks per SM: the register budget per thread, a multiple of 8 (the allocation unit)
template <int TY, int MINB>
constexpr int t3t_threads() {
    return (TY + 4) * 32;  // TY + 2 row warps, the halo warp, the producer warp
}
template <int TY, int MINB>
constexpr int t3t_max_regs() {
    return (65536 / (t3t_threads<TY, MINB>() * MINB)) / 8 * 8 > 255 ? 255
                                                                    : (65536 / (t3t_threads<TY, MINB>() * MINB)) / 8 * 8;
}

template <class S, class IO, int TY, int NS, int MINB>
__global__ void __launch_bounds__(t3t_threads<TY, MINB>()) __maxnreg__((t3t_max_regs<TY, MINB>()))
    k_stream_collide_3d2t(const __grid_constant__ CUtensorMap vbox, const __grid_constant__ CUtensorMap vrow,
                          const __grid_constant__ CUtensorMap ebox, const __grid_constant__ CUtensorMap erow,
                          const typename IO::Elem *__restrict__ src, typename IO::Elem *__restrict__ dst, int nx,
                          int ny, int nz, long long pitch, int HZ, CollideCoef<float> cf, unsigned *wait_flag,
                          long long wait_ns, int inject) {
    static_assert(axis_only<S>(), "the 3D two-step tile needs the seven axis velocities");
    static_assert(2 * (TY + 2) <= 32, "one halo-warp lane per halo cell");
    constexpr int Q = S::Q;
    constexpr int R = TY + 2;
    constexpr int kConsumers = (R + 1) * 32;  // row warps and the halo warp: named barrier 1
    using L = T3tLayout<Q, IO, TY, NS>;
    constexpr int iR = vel_index<S>(0, 0, 0), iPX = vel_index<S>(1, 0, 0), iMX = vel_index<S>(-1, 0, 0);
    constexpr int iPY = vel_index<S>(0, 1, 0), iMY = vel_index<S>(0, -1, 0);
    constexpr int iPZ = vel_index<S>(0, 0, 1), iMZ = vel_index<S>(0, 0, -1);

    extern __shared__ __align__(128) unsigned char t3t_raw[];
    unsigned char *sm = t3t_raw + ((128u - (smem_addr(t3t_raw) & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + L::kBarOff);  // stage landed
    uint64_t *empty = full + NS;                                      // stage read by the consumers
    volatile unsigned *abort_flag = reinterpret_cast<volatile unsigned *>(empty + NS);
    float *ringp = reinterpret_cast<float *>(sm + L::kRingOff);
    float *hxs = reinterpret_cast<float *>(sm + L::kHaloOff);  // [slot][row][0: +x of x0-1, 1: -x of x0+128]
    auto ring = [&](int slot, int row, int v) { return ringp + ((slot * R + row) * 2 + v) * kT3W; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * kT3W, y0 = blockIdx.y * TY, z0 = blockIdx.z * HZ;
    auto wrap = [](int v, int n) {
        v %= n;
        return v < 0 ? v + n : v;
    };
    const long long plane = (long long)nx * ny;
    const int iters = HZ + 2;
    const int xl = wrap(x0 - 1, nx), xr = wrap(x0 + kT3W, nx);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        *abort_flag = 0u;
        fence_barrier_init();
    }
    __syncthreads();  // the only block-wide barrier; from here on the producer runs on its own

    // ---- producer warp (lane 0): the level-1 inputs of iteration k (plane p1 = z0 - 1 + k) into
    // stage k % NS, as soon as the consumers released that stage (iteration k - NS done).
    // Velocity i needs source rows y0 - 1 - c_y .. y0 + TY - c_y of plane p1 - c_z; only the first
    // two and the last two of them can wrap (y0 is a multiple of TY, ny of TY, ny >= 2 TY).
    if (warp == R + 1) {
        if (lane != 0) return;
        tma_prefetch_desc(&vbox);
        tma_prefetch_desc(&vrow);
        if constexpr (IO::kExp) {
            tma_prefetch_desc(&ebox);
            tma_prefetch_desc(&erow);
        }
        unsigned tx = 0;
        static_for<Q>([&](auto I) {
            constexpr int cy = S::c(decltype(I)::value, 1);
            const int yb = y0 - 1 - cy;
            tx += L::kBoxTx;
            const int cand[4] = {0, 1, R - 2, R - 1};
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (yb + cand[c] < 0 || yb + cand[c] >= ny) tx += L::kRowTx;
        });
        int issued = 0;
        bool ok = true;
        for (int k = 0; k < iters; ++k) {
            const int s = k % NS;
            if (k >= NS && !mbar_wait_bounded(&empty[s], (unsigned)(k / NS - 1) & 1u, wait_ns)) {
                ok = false;
                break;
            }
            if (*abort_flag) break;
            const int p1 = z0 - 1 + k;
            unsigned char *st = sm + s * L::kStageBytes;
            mbar_arrive_expect_tx(&full[s], tx + ((inject && k == 0) ? 16u : 0u));
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cy = S::c(i, 1), cz = S::c(i, 2);
                const int yb = y0 - 1 - cy;
                const int zz = wrap(p1 - cz, nz);
                unsigned char *vb = st + i * L::kVelBytes;
                tma_load_4d(vb, &vbox, x0, yb, zz, i, &full[s]);
                if constexpr (IO::kExp) tma_load_4d(vb + L::kValBytes, &ebox, x0 / 8, yb, zz, i, &full[s]);
                const int cand[4] = {0, 1, R - 2, R - 1};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int ys = yb + cand[c];
                    if (ys >= 0 && ys < ny) continue;
                    const int sl = ys < 0 ? ys + 2 : ys - ny;
                    tma_load_4d(vb + L::kValBox + sl * IO::kValRow, &vrow, x0, wrap(ys, ny), zz, i, &full[s]);
                    if constexpr (IO::kExp)
                        tma_load_4d(vb + L::kValBytes + L::kExpBox + sl * 128, &erow, x0 / 8, wrap(ys, ny), zz, i,
                                    &full[s]);
                }
            });
            ++issued;
        }
        if (!ok || *abort_flag) {  // the consumers gave up: let the copies in flight land, then leave
            for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
                mbar_wait_bounded(&full[j % NS], (unsigned)(j / NS) & 1u, 2000000);
            spin_ns(200000);
        }
        return;
    }

    // ---- row warps: where their source row of each c_y sits in a stage (j = 1 - c_y)
    int voff[3], eoff[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int ys = y0 - 1 + warp - (1 - j);
        if (ys >= 0 && ys < ny) {
            voff[j] = warp * IO::kValRow;
            eoff[j] = L::kValBytes + warp * 16;
        } else {
            const int sl = ys < 0 ? ys + 2 : ys - ny;
            voff[j] = L::kValBox + sl * IO::kValRow;
            eoff[j] = L::kValBytes + L::kExpBox + sl * 128;
        }
    }
    const int yw = wrap(y0 - 1 + warp, ny);  // this row warp's row (wrapped)
    // lanes 0 and 31: the element of S(t) that the 4-cell vectors of +x (column x0 - 1) and -x
    // (column x0 + 128) lack, from this warp's row of plane p
    auto load_edge = [&](int p, typename IO::Raw &r) {
        const long long rowi = (long long)wrap(p, nz) * plane + (long long)yw * nx;
        if (lane == 0) {
            r = IO::ldg1(src, pitch, (long long)iPX * pitch + rowi + xl);
        } else if (lane == 31) {
            r = IO::ldg1(src, pitch, (long long)iMX * pitch + rowi + xr);
        }
    };
    // ---- halo warp: lane c < 2 R computes level 1 at column (c odd ? x0 + 128 : x0 - 1) of row
    // y0 - 1 + c / 2; it pulls velocity i from column hxc[1 - c_x], row hy[1 - c_y]
    const int hrow = lane >> 1;
    const int yh = wrap(y0 - 1 + hrow, ny);
    const int xc = (lane & 1) ? xr : xl;
    const int hy[3] = {wrap(yh - 1, ny), yh, wrap(yh + 1, ny)};
    const int hxc[3] = {wrap(xc - 1, nx), xc, wrap(xc + 1, nx)};
    auto load_halo = [&](int p, typename IO::Raw(&r)[Q]) {
        if (lane < 2 * R) {
            const int pl[3] = {wrap(p - 1, nz), wrap(p, nz), wrap(p + 1, nz)};
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = S::c(i, 0), cy = S::c(i, 1), cz = S::c(i, 2);
                r[i] = IO::ldg1(src, pitch,
                                (long long)i * pitch + pl[1 - cz] * plane + (long long)hy[1 - cy] * nx + hxc[1 - cx]);
            });
        }
    };

    // After the barrier of iteration k: release stage k % NS to the producer, or, if any row warp's
    // wait timed out, record it and leave (the producer drains the copies in flight).
    auto end_of_level1 = [&](int k, bool timed_out) -> bool {
        if (timed_out) {
            if (threadIdx.x == 0) {
                *abort_flag = 1u;
                if (wait_flag) {
                    *reinterpret_cast<volatile unsigned *>(wait_flag) = 1u;
                    __threadfence_system();
                }
            }
            return false;
        }
        if (threadIdx.x == 0) mbar_arrive(&empty[k % NS]);
        return true;
    };

    // The halo warp and the row warps run separate loops with the same barrier sequence (named
    // barrier 1, once per iteration), so that neither keeps the other's registers alive.
    if (warp == R) {
        typename IO::Raw hr_n[Q];
        load_halo(z0 - 1, hr_n);
        for (int k = 0; k < iters; ++k) {
            typename IO::Raw hr[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) hr[i] = hr_n[i];
            if (k + 1 < iters) load_halo(z0 + k, hr_n);
            if (lane < 2 * R) {
                float hin[Q][1], hout[Q][1];
#pragma unroll
                for (int i = 0; i < Q; ++i) hin[i][0] = IO::cvt1(hr[i]);
                collide_chunk<S, true>(hin, hout, cf);
                hxs[((k % 3) * R + hrow) * 2 + (lane & 1)] = IO::round((lane & 1) ? hout[iMX][0] : hout[iPX][0]);
            }
            if (!end_of_level1(k, bar_or(1, kConsumers, false))) return;
        }
        return;
    }

    typename IO::Raw er{}, er_n{};
    load_edge(z0 - 1, er_n);
    float r1[kT3V], px1[kT3V], mx1[kT3V], pz1[kT3V], pz2[kT3V];
#pragma unroll
    for (int e = 0; e < kT3V; ++e) r1[e] = px1[e] = mx1[e] = pz1[e] = pz2[e] = 0.f;

    for (int k = 0; k < iters; ++k) {
        const int p1 = z0 - 1 + k;
        // ---- level 1: plane p1, row y0 - 1 + warp
        er = er_n;
        if (k + 1 < iters) load_edge(p1 + 1, er_n);
        const bool ok = mbar_wait_bounded(&full[k % NS], (unsigned)(k / NS) & 1u, wait_ns);
        const unsigned char *st = sm + (k % NS) * L::kStageBytes;
        float post[Q][kT3V];
        {
            float pa[Q][kT3V];
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = S::c(i, 0), cy = S::c(i, 1);
                const unsigned char *vb = st + i * L::kVelBytes;
                float v[kT3V];
                IO::ld4(vb + voff[1 - cy], vb + eoff[1 - cy], lane, v);
                if constexpr (cx == 0) {
#pragma unroll
                    for (int e = 0; e < kT3V; ++e) pa[i][e] = v[e];
                } else if constexpr (cx == 1) {
                    float left = __shfl_up_sync(kFull, v[kT3V - 1], 1);
                    if (lane == 0) left = IO::cvt1(er);
                    pa[i][0] = left;
#pragma unroll
                    for (int e = 1; e < kT3V; ++e) pa[i][e] = v[e - 1];
                } else {
                    float right = __shfl_down_sync(kFull, v[0], 1);
                    if (lane == 31) right = IO::cvt1(er);
#pragma unroll
                    for (int e = 0; e + 1 < kT3V; ++e) pa[i][e] = v[e + 1];
                    pa[i][kT3V - 1] = right;
                }
            });
            collide_chunk<S, true>(pa, post, cf);
        }
        if constexpr (IO::kRound) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
#pragma unroll
                for (int e = 0; e < kT3V; ++e) post[i][e] = IO::round(post[i][e]);
        }
        *reinterpret_cast<float4 *>(ring(k % 3, warp, 0) + kT3V * lane) =
            make_float4(post[iPY][0], post[iPY][1], post[iPY][2], post[iPY][3]);
        *reinterpret_cast<float4 *>(ring(k % 3, warp, 1) + kT3V * lane) =
            make_float4(post[iMY][0], post[iMY][1], post[iMY][2], post[iMY][3]);
        // level 1 of plane p1 visible; level 2 of plane p1 - 2 done with its slots; stage k % NS read
        if (!end_of_level1(k, bar_or(1, kConsumers, !ok))) return;

        // ---- level 2: plane p2 = p1 - 1, rows y0 .. y0+TY-1 (warp-uniform condition).  Its pulls
        // are gathered first, so that the carried level-1 values can move on before the collision.
        const int p2 = p1 - 1;
        const bool l2 = k >= 2 && warp >= 1 && warp <= TY;
        float pb[Q][kT3V];
        if (l2) {
            const int sp = (k - 1) % 3;
            const float4 a = *reinterpret_cast<const float4 *>(ring(sp, warp - 1, 0) + kT3V * lane);
            const float4 b = *reinterpret_cast<const float4 *>(ring(sp, warp + 1, 1) + kT3V * lane);
            const float left = __shfl_up_sync(kFull, px1[kT3V - 1], 1);
            const float right = __shfl_down_sync(kFull, mx1[0], 1);
            const float hl = hxs[(sp * R + warp) * 2 + 0], hrt = hxs[(sp * R + warp) * 2 + 1];
#pragma unroll
            for (int e = 0; e < kT3V; ++e) {
                pb[iR][e] = r1[e];
                pb[iPZ][e] = pz2[e];
                pb[iMZ][e] = post[iMZ][e];
            }
            pb[iPX][0] = lane == 0 ? hl : left;
#pragma unroll
            for (int e = 1; e < kT3V; ++e) pb[iPX][e] = px1[e - 1];
#pragma unroll
            for (int e = 0; e + 1 < kT3V; ++e) pb[iMX][e] = mx1[e + 1];
            pb[iMX][kT3V - 1] = lane == 31 ? hrt : right;
            pb[iPY][0] = a.x; pb[iPY][1] = a.y; pb[iPY][2] = a.z; pb[iPY][3] = a.w;
            pb[iMY][0] = b.x; pb[iMY][1] = b.y; pb[iMY][2] = b.z; pb[iMY][3] = b.w;
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
        if (l2) {
            float out[Q][kT3V];
            collide_chunk<S, true>(pb, out, cf);
            const int y = y0 - 1 + warp;
            const bool stv = y < ny && p2 < nz;
            const long long oi = (long long)p2 * plane + (long long)y * nx + x0 + kT3V * lane;
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                IO::st4(dst, pitch, (long long)i * pitch + oi, out[i], stv);
            });
        }
    }
}

// ---- host side (kT3tRows and t3t_eligible: ops.cuh)

template <class S, class IO, int TY, int NS, int MINB>
int *t3t_capacity() {
    static int cap[64] = {0};
    return cap;
}
template <class S, class IO, int TY, int NS, int MINB>
cudaError_t t3t_prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (t3t_capacity<S, IO, TY, NS, MINB>()[dev]) return cudaSuccess;
    if (!encode_tiled_fn()) return cudaErrorNotSupported;
    constexpr int smem = T3tLayout<S::Q, IO, TY, NS>::kBytes;
    auto kern = k_stream_collide_3d2t<S, IO, TY, NS, MINB>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, t3t_threads<TY, MINB>(), smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    t3t_capacity<S, IO, TY, NS, MINB>()[dev] = per_sm * sms > 0 ? per_sm * sms : 1;
    return cudaSuccess;
}

// Tensor maps over state copy `g` and the launch (tiles of 128 x TY cells, z segments so that all
// blocks are resident in one wave).
template <class S, class IO, int TY, int NS, int MINB>
cudaError_t t3t_launch(const StepLaunch &Lc) {
    using L = T3tLayout<S::Q, IO, TY, NS>;
    if (Lc.open || Lc.slab || Lc.nx % kT3W != 0 || Lc.ny % TY != 0 || Lc.ny < 2 * TY || Lc.pitch % 128 != 0)
        return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || t3t_capacity<S, IO, TY, NS, MINB>()[dev] == 0) return cudaErrorNotReady;
    const unsigned long long nx = Lc.nx, ny = Lc.ny, nz = Lc.nz, P = Lc.pitch;
    constexpr unsigned long long E = IO::kValRow / kT3W;  // bytes per stored value
    CUtensorMap vbox, vrow, ebox, erow;
    {
        const unsigned long long dims[4] = {nx, ny, nz, (unsigned long long)S::Q};
        const unsigned long long str[3] = {nx * E, nx * ny * E, P * E};
        e = encode_map4(&vbox, IO::kType, Lc.src, dims, str, kT3W, L::kRows);
        if (e == cudaSuccess) e = encode_map4(&vrow, IO::kType, Lc.src, dims, str, kT3W, 1);
    }
    if (e == cudaSuccess) {
        if constexpr (IO::kExp) {
            const void *ex = static_cast<const unsigned char *>(Lc.src) + 2ull * S::Q * P;
            const unsigned long long dims[4] = {nx / 8, ny, nz, (unsigned long long)S::Q};
            const unsigned long long str[3] = {nx / 8, nx * ny / 8, P / 8};
            e = encode_map4(&ebox, CU_TENSOR_MAP_DATA_TYPE_UINT8, ex, dims, str, 16, L::kRows);
            if (e == cudaSuccess) e = encode_map4(&erow, CU_TENSOR_MAP_DATA_TYPE_UINT8, ex, dims, str, 16, 1);
        } else {
            ebox = vbox;
            erow = vrow;
        }
    }
    if (e != cudaSuccess) return e;
    const int strips = Lc.nx / kT3W, ytiles = Lc.ny / TY;
    int zsegs = t3t_capacity<S, IO, TY, NS, MINB>()[dev] / (strips * ytiles);
    if (zsegs < 1) zsegs = 1;
    if (zsegs > Lc.nz) zsegs = Lc.nz;
    const int HZ = (Lc.nz + zsegs - 1) / zsegs;
    const dim3 grid(strips, ytiles, (Lc.nz + HZ - 1) / HZ);
    const CollideCoef<float> cf = make_coef<float>(Lc.omega, Lc.coefM, Lc.coefN);
    k_stream_collide_3d2t<S, IO, TY, NS, MINB><<<grid, t3t_threads<TY, MINB>(), L::kBytes, Lc.stream>>>(
        vbox, vrow, ebox, erow, static_cast<const typename IO::Elem *>(Lc.src), static_cast<typename IO::Elem *>(Lc.dst),
        Lc.nx, Lc.ny, Lc.nz, Lc.pitch, HZ, cf, Lc.wait_flag, Lc.wait_ns > 0 ? Lc.wait_ns : 1000000000LL,
        Lc.t3_inject);
    return cudaGetLastError();
}

}  // namespace lee

// step_launch.cuh -- launch configuration of the fused stream-collide kernels for one velocity set:
// the one-step kernel (cells per thread, grid) and the two-step and K-step 2D kernels (tile height
// from the resident capacity).  Together with kernels.cuh and velsets.cuh this fixes what the
// profiled hot-path launches execute.
#pragma once

#include "ops.cuh"

namespace lee {

template <class S, class T, int V, bool OPEN, bool CUT = false>
cudaError_t launch_step_v(const StepLaunch &L) {
    using C = typename Store<T>::C;
    GridDesc gd;
    gd.nx = L.nx;
    gd.ny = L.ny;
    gd.nz = L.nz;
    gd.nxc = L.nx / V;
    gd.nchunks = (long long)gd.nxc * L.ny * L.nz;
    gd.pitch = L.pitch;
    const CollideCoef<C> cf = make_coef<C>(L.omega, L.coefM, L.coefN);
    OpenEdge<C> ob;
    ob.sponge_w = L.sponge_w;
    ob.sponge_smax = (C)L.sponge_smax;
    ob.ghost = static_cast<const C *>(L.ghost);
    ob.ghost_L = L.ghost_L;
    ob.skip_border = L.skip_border;
    const long long blocks = (gd.nchunks + 255) / 256;
    k_stream_collide<S, T, V, OPEN, CUT><<<(unsigned)blocks, 256, 0, L.stream>>>(static_cast<const T *>(L.src),
                                                                                   static_cast<T *>(L.dst), gd, cf, ob);
    return cudaGetLastError();
}

// Vector width: one 16-byte access per velocity and thread (8 bytes for the 19-velocity set, to
// bound register use); one cell per thread when nx is not a multiple of the width.
template <class S, class T>
constexpr int vec_width() {
    constexpr int bytes = (S::Q > 13) ? 8 : 16;
    constexpr int v = bytes / (int)sizeof(T);
    return v < 1 ? 1 : v;
}

// BFP16 storage (bfp.cuh): 8 cells per lane (4 for the 13- and 19-velocity sets, which would
// need 128 registers at 8; LEE_BFP_CELLS=4 or 8 at create time picks either, for comparisons)
// when nx is a multiple of the 8-cell block, one cell per lane otherwise.
template <class S, int V, bool OPEN>
cudaError_t launch_step_bfp_v(const StepLaunch &L) {
    GridDesc gd;
    gd.nx = L.nx;
    gd.ny = L.ny;
    gd.nz = L.nz;
    gd.nxc = L.nx / V;
    gd.nchunks = (long long)gd.nxc * L.ny * L.nz;
    gd.pitch = L.pitch;
    const CollideCoef<float> cf = make_coef<float>(L.omega, L.coefM, L.coefN);
    const OpenEdge<float> ob{L.sponge_w, (float)L.sponge_smax, nullptr, 0};
    const long long blocks = (gd.nchunks + 255) / 256;
    k_stream_collide_bfp<S, V, OPEN><<<(unsigned)blocks, 256, 0, L.stream>>>(static_cast<const Bfp16 *>(L.src),
                                                                               static_cast<Bfp16 *>(L.dst), gd, cf, ob);
    return cudaGetLastError();
}
template <class S>
cudaError_t launch_step_bfp(const StepLaunch &L) {
    if (L.ghost) return cudaErrorInvalidValue;  // no learned edge on BFP16 storage
    if (!L.force_scalar && L.nx % kBfpBlock == 0) {
        const int V = L.bfp_cells ? L.bfp_cells : (S::Q > 9 ? 4 : 8);
        if (V == 4) return L.open ? launch_step_bfp_v<S, 4, true>(L) : launch_step_bfp_v<S, 4, false>(L);
        return L.open ? launch_step_bfp_v<S, 8, true>(L) : launch_step_bfp_v<S, 8, false>(L);
    }
    return L.open ? launch_step_bfp_v<S, 1, true>(L) : launch_step_bfp_v<S, 1, false>(L);
}

template <class S, class T>
cudaError_t launch_step_t(const StepLaunch &L) {
    if constexpr (std::is_same<T, Bfp16>::value) {
        return launch_step_bfp<S>(L);
    } else {
        constexpr int V = vec_width<S, T>();
        if constexpr (S::D >= 2) {
            if (L.slab) {  // periodic except along the cut, which reads the halo planes
                if constexpr (V > 1) {
                    if (!L.force_scalar && L.nx % V == 0) return launch_step_v<S, T, V, false, true>(L);
                }
                return launch_step_v<S, T, 1, false, true>(L);
            }
        }
        if constexpr (V > 1) {
            if (!L.force_scalar && L.nx % V == 0)
                return L.open ? launch_step_v<S, T, V, true>(L) : launch_step_v<S, T, V, false>(L);
        }
        return L.open ? launch_step_v<S, T, 1, true>(L) : launch_step_v<S, T, 1, false>(L);
    }
}

template <class Fn>
cudaError_t with_storage(int storage, Fn &&fn) {
    switch (storage) {
    case LEE_STORE_F64: return fn((double *)nullptr);
    case LEE_STORE_F32: return fn((float *)nullptr);
    case LEE_STORE_F16: return fn((__half *)nullptr);
    case LEE_STORE_BF16: return fn((__nv_bfloat16 *)nullptr);
    case LEE_STORE_BFP16: return fn((Bfp16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

// Resident capacity of the two-step kernel (blocks per SM x SMs) per device, set by
// two_step_prepare outside any stream capture.
template <class S>
int *two_step_capacity() {
    static int cap[64] = {0};
    return cap;
}
template <class S>
cudaError_t two_step_prepare() {
    if constexpr (S::D != 2) {
        return cudaErrorInvalidValue;
    } else {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (two_step_capacity<S>()[dev]) return cudaSuccess;
        constexpr int smem = tb_smem_bytes<S>();
        e = cudaFuncSetAttribute(k_stream_collide_2step<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stream_collide_2step<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, per_sm_pf = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_2step<S, false>, 128, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_pf, k_stream_collide_2step<S, true>, 128, smem);
        if (per_sm_pf < per_sm) per_sm = per_sm_pf;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        two_step_capacity<S>()[dev] = per_sm * sms > 0 ? per_sm * sms : 1;
        return cudaSuccess;
    }
}
template <class S>
cudaError_t two_step_launch(const StepLaunch &L) {
    if constexpr (S::D != 2) {
        return cudaErrorInvalidValue;
    } else {
        if (L.storage != LEE_STORE_F32 || L.open || L.nx % 4 != 0 || L.ny < 3) return cudaErrorInvalidValue;
        const CollideCoef<float> cf = make_coef<float>(L.omega, L.coefM, L.coefN);
        constexpr int smem = tb_smem_bytes<S>();
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64 || two_step_capacity<S>()[dev] == 0) return cudaErrorNotReady;  // prepare first
        // tile height: the smallest multiple of 4 (>= 16) that puts every tile in one resident wave
        const int strips = (L.nx + kTbW - 1) / kTbW;
        int segs = two_step_capacity<S>()[dev] / strips;
        if (segs < 1) segs = 1;
        int H = (L.ny + segs - 1) / segs;
        H = (H + 3) / 4 * 4;
        if (H < 16) H = 16;
        const dim3 grid(strips, (L.ny + H - 1) / H);
        const long long bytes = 2LL * S::Q * (long long)sizeof(float) * L.nx * L.ny;
        auto kern = bytes <= kTbL2PrefetchMaxBytes ? k_stream_collide_2step<S, true> : k_stream_collide_2step<S, false>;
        kern<<<grid, 128, smem, L.stream>>>(static_cast<const float *>(L.src), static_cast<float *>(L.dst), L.nx, L.ny,
                                            L.pitch, H, cf);
        return cudaGetLastError();
    }
}


// The same for K steps per launch (K = 3, 4): resident capacity per device, then the launch.
// IO: the storage policy of the tile (TileIoF32, or TileIoBfp for BFP16 storage).
template <class S, int K, class IO>
int *kstep_capacity() {
    static int cap[64] = {0};
    return cap;
}
template <class S, int K, class IO = TileIoF32>
cudaError_t kstep_prepare() {
    if constexpr (S::D != 2) {
        return cudaErrorInvalidValue;
    } else {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (kstep_capacity<S, K, IO>()[dev]) return cudaSuccess;
        constexpr int smem = tbk_smem_bytes<S, K>();
        e = cudaFuncSetAttribute(k_stream_collide_kstep<S, K, IO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_kstep<S, K, IO>, kTbkThreads, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        kstep_capacity<S, K, IO>()[dev] = per_sm * sms > 0 ? per_sm * sms : 1;
        return cudaSuccess;
    }
}
template <class S, int K, class IO = TileIoF32>
cudaError_t kstep_launch(const StepLaunch &L) {
    if constexpr (S::D != 2) {
        return cudaErrorInvalidValue;
    } else {
        using E = typename IO::Elem;
        constexpr bool bfp = std::is_same<E, Bfp16>::value;
        constexpr int storage = bfp ? LEE_STORE_BFP16
                                    : std::is_same<E, float>::value ? LEE_STORE_F32
                                    : std::is_same<E, __half>::value ? LEE_STORE_F16 : LEE_STORE_BF16;
        if (L.storage != storage || L.open || L.nx % (bfp ? kBfpBlock : 4) != 0 || L.ny < 3)
            return cudaErrorInvalidValue;
        const CollideCoef<float> cf = make_coef<float>(L.omega, L.coefM, L.coefN);
        constexpr int smem = tbk_smem_bytes<S, K>();
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64 || kstep_capacity<S, K, IO>()[dev] == 0) return cudaErrorNotReady;  // prepare first
        // tile height: the smallest multiple of 4 (>= 16) that puts every tile in one resident wave
        const int strips = (L.nx + kTbW - 1) / kTbW;
        int segs = kstep_capacity<S, K, IO>()[dev] / strips;
        if (segs < 1) segs = 1;
        int H = (L.ny + segs - 1) / segs;
        H = (H + 3) / 4 * 4;
        if (H < 16) H = 16;
        const dim3 grid(strips, (L.ny + H - 1) / H);
        // No L2 prefetch: it helps the byte-bound two-step kernel on small grids, but this kernel
        // is bound by instruction issue, and the prefetch instructions cost more than they save
        // (measured on GB300, D2Q5 2048^2: 402 GLUPS without, 388 with).
        k_stream_collide_kstep<S, K, IO><<<grid, kTbkThreads, smem, L.stream>>>(static_cast<const E *>(L.src),
                                                                         static_cast<E *>(L.dst), L.nx, L.ny, L.pitch,
                                                                         H, cf);
        return cudaGetLastError();
    }
}

}  // namespace lee

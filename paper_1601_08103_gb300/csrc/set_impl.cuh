// set_impl.cuh -- host launchers for one velocity set, instantiated by the set_*.cu units.
#pragma once

#include "ops.cuh"

namespace lee {

template <class S, class T, int V, bool OPEN>
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
    const long long blocks = (gd.nchunks + 255) / 256;
    k_stream_collide<S, T, V, OPEN><<<(unsigned)blocks, 256, 0, L.stream>>>(static_cast<const T *>(L.src),
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

template <class S, class T>
cudaError_t launch_step_t(const StepLaunch &L) {
    constexpr int V = vec_width<S, T>();
    if constexpr (V > 1) {
        if (!L.force_scalar && L.nx % V == 0)
            return L.open ? launch_step_v<S, T, V, true>(L) : launch_step_v<S, T, V, false>(L);
    }
    return L.open ? launch_step_v<S, T, 1, true>(L) : launch_step_v<S, T, 1, false>(L);
}

template <class Fn>
cudaError_t with_storage(int storage, Fn &&fn) {
    switch (storage) {
    case LEE_STORE_F64: return fn((double *)nullptr);
    case LEE_STORE_F32: return fn((float *)nullptr);
    case LEE_STORE_F16: return fn((__half *)nullptr);
    case LEE_STORE_BF16: return fn((__nv_bfloat16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

template <class S>
struct SetImpl {
    static cudaError_t step(const StepLaunch &L) {
        return with_storage(L.storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            return launch_step_t<S, T>(L);
        });
    }
    static cudaError_t init(int storage, const double *rho, const double *u, const double *theta, void *g, long long cells,
                            long long pitch, const SetConsts &k, cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_init_equilibrium<S, T><<<aux_blocks(cells), 256, 0, st>>>(rho, u, theta, static_cast<T *>(g), cells, pitch, k);
            return cudaGetLastError();
        });
    }
    static cudaError_t init_maxabs(const double *rho, const double *u, const double *theta, long long cells,
                                   const SetConsts &k, unsigned int *maxbits, cudaStream_t st) {
        k_init_maxabs<S><<<aux_blocks(cells), 256, 0, st>>>(rho, u, theta, cells, k, maxbits);
        return cudaGetLastError();
    }
    static cudaError_t moments(int storage, const void *g, long long cells, long long pitch, const SetConsts &k, double *rho,
                               double *u, double *theta, cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_moments<S, T><<<aux_blocks(cells), 256, 0, st>>>(static_cast<const T *>(g), cells, pitch, k, rho, u, theta);
            return cudaGetLastError();
        });
    }
    static cudaError_t reduce_partial(int storage, const void *g, long long cells, long long pitch, const SetConsts &k,
                                      double *partial, int nblocks, cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_reduce_partial<S, T><<<nblocks, kReduceThreads, 0, st>>>(static_cast<const T *>(g), cells, pitch, k, partial);
            return cudaGetLastError();
        });
    }
    static cudaError_t export_f64(int storage, const void *g, long long cells, long long pitch, const SetConsts &k,
                                  double *out, cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_export<S, T><<<aux_blocks(cells), 256, 0, st>>>(static_cast<const T *>(g), cells, pitch, k, out);
            return cudaGetLastError();
        });
    }
    static cudaError_t import_f64(int storage, const double *in, long long cells, long long pitch, const SetConsts &k,
                                  void *g, cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_import<S, T><<<aux_blocks(cells), 256, 0, st>>>(in, cells, pitch, k, static_cast<T *>(g));
            return cudaGetLastError();
        });
    }
    static cudaError_t sponge_damp(int storage, void *g, int nx, int ny, int nz, long long pitch, int w, double smax,
                                   cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            using C = typename Store<T>::C;
            GridDesc gd{nx, ny, nz, nx, (long long)nx * ny * nz, pitch};
            k_sponge_damp<S, T><<<aux_blocks(gd.nchunks), 256, 0, st>>>(static_cast<T *>(g), gd, w, (C)smax);
            return cudaGetLastError();
        });
    }
    static cudaError_t onchip_1d(const StepLaunch &L, void *g, long long nsteps) {
        if constexpr (S::D != 1) {
            return cudaErrorInvalidValue;
        } else {
            return with_storage(L.storage, [&](auto *tp) {
                using T = std::remove_pointer_t<decltype(tp)>;
                using C = typename Store<T>::C;
                const size_t smem = 2 * sizeof(T) * (size_t)S::Q * (size_t)L.nx;
                if (smem > (size_t)kMaxOnchipSmem) return cudaErrorInvalidValue;
                cudaError_t e = cudaFuncSetAttribute(k_onchip_1d<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
                if (e != cudaSuccess) return e;
                const CollideCoef<C> cf = make_coef<C>(L.omega, L.coefM, L.coefN);
                OpenEdge<C> ob{L.sponge_w, (C)L.sponge_smax, nullptr, 0};
                const int threads = L.nx < 1024 ? ((L.nx + 31) / 32) * 32 : 1024;
                k_onchip_1d<S, T><<<1, threads, smem, L.stream>>>(static_cast<T *>(g), L.nx, L.pitch, cf, ob, L.open,
                                                                  nsteps);
                return cudaGetLastError();
            });
        }
    }
    // Resident capacity of the two-step kernel (blocks per SM x SMs) per device, set by
    // step2_prepare outside any stream capture.
    static int *step2_capacity() {
        static int cap[64] = {0};
        return cap;
    }
    static cudaError_t step2_prepare() {
        if constexpr (S::D != 2) {
            return cudaErrorInvalidValue;
        } else {
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return e;
            if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
            if (step2_capacity()[dev]) return cudaSuccess;
            constexpr int smem = tb_smem_bytes<S>();
            e = cudaFuncSetAttribute(k_stream_collide_2step<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_2step<S>, 128, smem);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            step2_capacity()[dev] = per_sm * sms > 0 ? per_sm * sms : 1;
            return cudaSuccess;
        }
    }
    static cudaError_t step2(const StepLaunch &L) {
        if constexpr (S::D != 2) {
            return cudaErrorInvalidValue;
        } else {
            if (L.storage != LEE_STORE_F32 || L.open || L.nx % 4 != 0 || L.ny < 3) return cudaErrorInvalidValue;
            const CollideCoef<float> cf = make_coef<float>(L.omega, L.coefM, L.coefN);
            constexpr int smem = tb_smem_bytes<S>();
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return e;
            if (dev < 0 || dev >= 64 || step2_capacity()[dev] == 0) return cudaErrorNotReady;  // prepare first
            // tile height: the smallest multiple of 4 (>= 16) that puts every tile in one resident wave
            const int strips = (L.nx + kTbW - 1) / kTbW;
            int segs = step2_capacity()[dev] / strips;
            if (segs < 1) segs = 1;
            int H = (L.ny + segs - 1) / segs;
            H = (H + 3) / 4 * 4;
            if (H < 16) H = 16;
            const dim3 grid(strips, (L.ny + H - 1) / H);
            k_stream_collide_2step<S><<<grid, 128, smem, L.stream>>>(static_cast<const float *>(L.src),
                                                                     static_cast<float *>(L.dst), L.nx, L.ny, L.pitch, H,
                                                                     cf);
            return cudaGetLastError();
        }
    }
    static SetOps make() {
        SetOps o{};
        o.D = S::D;
        o.Q = S::Q;
        o.step = &step;
        o.init = &init;
        o.init_maxabs = &init_maxabs;
        o.moments = &moments;
        o.reduce_partial = &reduce_partial;
        o.export_f64 = &export_f64;
        o.import_f64 = &import_f64;
        o.sponge_damp = &sponge_damp;
        o.onchip_1d = S::D == 1 ? &onchip_1d : nullptr;
        o.step2 = S::D == 2 ? &step2 : nullptr;
        o.step2_prepare = S::D == 2 ? &step2_prepare : nullptr;
        for (int i = 0; i < S::Q; ++i) {
            for (int a = 0; a < 3; ++a) o.c[i][a] = S::c(i, a);
            o.shell[i] = S::shell(i);
        }
        return o;
    }
};

}  // namespace lee

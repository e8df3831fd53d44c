// set_impl.cuh -- host launchers for one velocity set, instantiated by the set_*.cu units.
#pragma once

#include "onchip_cluster.cuh"
#include "split.cuh"
#include "step_launch.cuh"
#include "tb3d.cuh"
#include "tb3d_tma.cuh"

namespace lee {

// Split storage (split.cuh): pointers into one state copy and the FP32 coefficients.
template <class S>
struct SplitView {
    static float *m(void *base) { return static_cast<float *>(base); }
    static const float *m(const void *base) { return static_cast<const float *>(base); }
    static __half *n(void *base, long long pitch) {
        return reinterpret_cast<__half *>(static_cast<float *>(base) + (long long)(S::D + 2) * pitch);
    }
    static const __half *n(const void *base, long long pitch) {
        return reinterpret_cast<const __half *>(static_cast<const float *>(base) + (long long)(S::D + 2) * pitch);
    }
};

template <class S>
SplitCoef split_coef(double omega, double scale) {
    const SetConsts k = host_consts<S>(scale);
    SplitCoef c{};
    for (int t = 0; t < 4; ++t) {
        const double fa = k.a1 + 0.5 * t * k.c1, fb = k.a2 + 0.5 * t * k.c2;
        c.alpha[t] = (float)(k.f[t] * (fa - k.kR * fb));
        c.beta[t] = (float)(k.f[t] * k.kE * fb);
        c.gamma[t] = (float)(k.f[t] * k.b * k.inv_rho0);
        c.ew[t] = (float)k.ew[t];
        c.dec[t] = (float)k.dec[t];
        c.enc[t] = (float)k.enc[t];
    }
    c.one_minus_omega = 1.0f - (float)omega;
    return c;
}

template <class S>
cudaError_t launch_split_step(const StepLaunch &L) {
    if (L.open) return cudaErrorInvalidValue;  // periodic grids only
    constexpr int VV = S::Q > 13 ? 2 : 4;  // bound the registers of the q-heavy sets
    const int V = (L.force_scalar || L.nx % VV != 0) ? 1 : VV;
    GridDesc gd;
    gd.nx = L.nx;
    gd.ny = L.ny;
    gd.nz = L.nz;
    gd.nxc = L.nx / V;
    gd.nchunks = (long long)gd.nxc * L.ny * L.nz;
    gd.pitch = L.pitch;
    const SplitCoef cf = split_coef<S>(L.omega, L.store_scale);
    const float *ms = SplitView<S>::m(L.src);
    const __half *ns = SplitView<S>::n(L.src, L.pitch);
    float *md = SplitView<S>::m(L.dst);
    __half *nd = SplitView<S>::n(L.dst, L.pitch);
    if (V == VV && gd.nxc % 32 == 0) {
        const long long tiles = (long long)(gd.nxc / 32) * ((L.ny + 3) / 4) * L.nz;
        k_split_step<S, VV, true><<<(unsigned)tiles, 128, 0, L.stream>>>(ms, ns, md, nd, gd, cf);
        return cudaGetLastError();
    }
    const unsigned blocks = (unsigned)((gd.nchunks + 127) / 128);
    if (V == VV) k_split_step<S, VV, false><<<blocks, 128, 0, L.stream>>>(ms, ns, md, nd, gd, cf);
    else k_split_step<S, 1, false><<<blocks, 128, 0, L.stream>>>(ms, ns, md, nd, gd, cf);
    return cudaGetLastError();
}

template <class S>
struct SetImpl {
    static cudaError_t step(const StepLaunch &L) {
        if (L.storage == LEE_STORE_SPLIT16) return launch_split_step<S>(L);
        return with_storage(L.storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            return launch_step_t<S, T>(L);
        });
    }
    static cudaError_t init(int storage, const double *rho, const double *u, const double *theta, void *g, long long cells,
                            long long pitch, const SetConsts &k, cudaStream_t st) {
        if (storage == LEE_STORE_SPLIT16) {
            k_split_init<S><<<aux_blocks(cells), 256, 0, st>>>(rho, u, theta, SplitView<S>::m(g),
                                                               SplitView<S>::n(g, pitch), cells, pitch, k);
            return cudaGetLastError();
        }
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            if constexpr (std::is_same<T, Bfp16>::value)
                k_init_equilibrium_bfp<S><<<aux_blocks(cells), 256, 0, st>>>(rho, u, theta, static_cast<T *>(g), cells,
                                                                              pitch, k);
            else
                k_init_equilibrium<S, T><<<aux_blocks(cells), 256, 0, st>>>(rho, u, theta, static_cast<T *>(g), cells,
                                                                            pitch, k);
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
        if (storage == LEE_STORE_SPLIT16) {
            k_split_moments<S><<<aux_blocks(cells), 256, 0, st>>>(SplitView<S>::m(g), cells, pitch, k, rho, u, theta);
            return cudaGetLastError();
        }
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_moments<S, T><<<aux_blocks(cells), 256, 0, st>>>(static_cast<const T *>(g), cells, pitch, k, rho, u, theta);
            return cudaGetLastError();
        });
    }
    static cudaError_t reduce_partial(int storage, const void *g, long long cells, long long pitch, const SetConsts &k,
                                      double *partial, int nblocks, cudaStream_t st) {
        if (storage == LEE_STORE_SPLIT16) {
            k_split_reduce_partial<S><<<nblocks, kReduceThreads, 0, st>>>(SplitView<S>::m(g), SplitView<S>::n(g, pitch),
                                                                          cells, pitch, k, partial);
            return cudaGetLastError();
        }
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_reduce_partial<S, T><<<nblocks, kReduceThreads, 0, st>>>(static_cast<const T *>(g), cells, pitch, partial);
            return cudaGetLastError();
        });
    }
    static cudaError_t export_f64(int storage, const void *g, long long cells, long long pitch, const SetConsts &k,
                                  double *out, cudaStream_t st) {
        if (storage == LEE_STORE_SPLIT16) {
            k_split_export<S><<<aux_blocks(cells), 256, 0, st>>>(SplitView<S>::m(g), SplitView<S>::n(g, pitch), cells,
                                                                 pitch, k, out);
            return cudaGetLastError();
        }
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            k_export<S, T><<<aux_blocks(cells), 256, 0, st>>>(static_cast<const T *>(g), cells, pitch, k, out);
            return cudaGetLastError();
        });
    }
    static cudaError_t import_f64(int storage, const double *in, long long cells, long long pitch, const SetConsts &k,
                                  void *g, cudaStream_t st) {
        if (storage == LEE_STORE_SPLIT16) {
            k_split_import<S><<<aux_blocks(cells), 256, 0, st>>>(in, cells, pitch, k, SplitView<S>::m(g),
                                                                 SplitView<S>::n(g, pitch));
            return cudaGetLastError();
        }
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            if constexpr (std::is_same<T, Bfp16>::value)
                k_import_bfp<S><<<aux_blocks(cells), 256, 0, st>>>(in, cells, pitch, static_cast<T *>(g));
            else
                k_import<S, T><<<aux_blocks(cells), 256, 0, st>>>(in, cells, pitch, k, static_cast<T *>(g));
            return cudaGetLastError();
        });
    }
    static cudaError_t slab_pack(int storage, const void *g, long long pitch, long long plane, int nl, void *lo,
                                 void *hi, cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) -> cudaError_t {
            using T = std::remove_pointer_t<decltype(tp)>;
            if constexpr (std::is_same<T, Bfp16>::value || S::D < 2) {
                return cudaErrorInvalidValue;
            } else {
                k_slab_pack<S, T><<<aux_blocks(plane), 256, 0, st>>>(static_cast<const T *>(g), pitch, plane, nl,
                                                                     static_cast<T *>(lo), static_cast<T *>(hi));
                return cudaGetLastError();
            }
        });
    }
    static cudaError_t slab_unpack(int storage, void *g, long long pitch, long long plane, int nl, const void *lo,
                                   const void *hi, cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) -> cudaError_t {
            using T = std::remove_pointer_t<decltype(tp)>;
            if constexpr (std::is_same<T, Bfp16>::value || S::D < 2) {
                return cudaErrorInvalidValue;
            } else {
                k_slab_unpack<S, T><<<aux_blocks(plane), 256, 0, st>>>(static_cast<T *>(g), pitch, plane, nl,
                                                                       static_cast<const T *>(lo),
                                                                       static_cast<const T *>(hi));
                return cudaGetLastError();
            }
        });
    }
    static cudaError_t sponge_damp(int storage, void *g, int nx, int ny, int nz, long long pitch, int w, double smax,
                                   cudaStream_t st) {
        return with_storage(storage, [&](auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            using C = typename Store<T>::C;
            GridDesc gd{nx, ny, nz, nx, (long long)nx * ny * nz, pitch};
            if constexpr (std::is_same<T, Bfp16>::value)
                k_sponge_damp_bfp<S><<<aux_blocks(gd.nchunks), 256, 0, st>>>(static_cast<T *>(g), gd, w, (C)smax);
            else
                k_sponge_damp<S, T><<<aux_blocks(gd.nchunks), 256, 0, st>>>(static_cast<T *>(g), gd, w, (C)smax);
            return cudaGetLastError();
        });
    }
    static cudaError_t onchip_1d(const StepLaunch &L, void *g, long long nsteps) {
        if constexpr (S::D != 1) {
            return cudaErrorInvalidValue;
        } else {
            return with_storage(L.storage, [&](auto *tp) -> cudaError_t {
                using T = std::remove_pointer_t<decltype(tp)>;
                using C = typename Store<T>::C;
                if constexpr (std::is_same<T, Bfp16>::value) {
                    return cudaErrorInvalidValue;  // BFP16 runs one launch per step
                } else {
                const size_t smem = 2 * sizeof(T) * (size_t)S::Q * (size_t)L.nx;
                if (smem > (size_t)kMaxOnchipSmem) return cudaErrorInvalidValue;
                cudaError_t e = cudaFuncSetAttribute(k_onchip_1d<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
                if (e != cudaSuccess) return e;
                const CollideCoef<C> cf = make_coef<C>(L.omega, L.coefM, L.coefN);
                OpenEdge<C> ob{L.sponge_w, (C)L.sponge_smax, nullptr, 0};
                if (L.nx >= 64 * kOnchipCluster) {
                    // a cluster of kOnchipCluster CTAs, one segment each (onchip_cluster.cuh)
                    const int seg = (L.nx + kOnchipCluster - 1) / kOnchipCluster;
                    const size_t csmem = 2 * sizeof(T) * (size_t)S::Q * (size_t)seg;
                    e = cudaFuncSetAttribute(k_onchip_1d_cluster<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)csmem);
                    if (e == cudaSuccess && kOnchipCluster > 8)  // clusters above 8 CTAs are opt-in
                        e = cudaFuncSetAttribute(k_onchip_1d_cluster<S, T>,
                                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                    if (e != cudaSuccess) return e;
                    cudaLaunchConfig_t lc = {};
                    lc.gridDim = dim3(kOnchipCluster);
                    lc.blockDim = dim3(seg < 1024 ? ((seg + 31) / 32) * 32 : 1024);
                    lc.dynamicSmemBytes = csmem;
                    lc.stream = L.stream;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeClusterDimension;
                    attr[0].val.clusterDim.x = kOnchipCluster;
                    attr[0].val.clusterDim.y = 1;
                    attr[0].val.clusterDim.z = 1;
                    lc.attrs = attr;
                    lc.numAttrs = 1;
                    e = cudaLaunchKernelEx(&lc, k_onchip_1d_cluster<S, T>, static_cast<T *>(g), L.nx, L.pitch, cf, ob,
                                           L.open, nsteps);
                    if (e != cudaSuccess) return e;
                    return cudaGetLastError();
                }
                const int threads = L.nx < 1024 ? ((L.nx + 31) / 32) * 32 : 1024;
                k_onchip_1d<S, T><<<1, threads, smem, L.stream>>>(static_cast<T *>(g), L.nx, L.pitch, cf, ob, L.open,
                                                                  nsteps);
                return cudaGetLastError();
                }
            });
        }
    }
    static cudaError_t step2_prepare() { return two_step_prepare<S>(); }
    static cudaError_t step2(const StepLaunch &L) { return two_step_launch<S>(L); }
    // K = 3 or 4 steps per launch: FP32 storage (bit-identical to single steps), or BFP16, FP16 and
    // BF16 storage (FP32 levels in between, one rounding to the storage per launch)
    template <class IO>
    static cudaError_t stepk_prepare_io(int k) {
        return k == 3 ? kstep_prepare<S, 3, IO>() : k == 4 ? kstep_prepare<S, 4, IO>() : cudaErrorInvalidValue;
    }
    template <class IO>
    static cudaError_t stepk_io(const StepLaunch &L, int k) {
        return k == 3 ? kstep_launch<S, 3, IO>(L) : k == 4 ? kstep_launch<S, 4, IO>(L) : cudaErrorInvalidValue;
    }
    static cudaError_t stepk_prepare(int k, int storage) {
        switch (storage) {
        case LEE_STORE_BFP16: return stepk_prepare_io<TileIoBfp<S::Q>>(k);
        case LEE_STORE_F16: return stepk_prepare_io<TileIo16<__half>>(k);
        case LEE_STORE_BF16: return stepk_prepare_io<TileIo16<__nv_bfloat16>>(k);
        case LEE_STORE_F32: return stepk_prepare_io<TileIoF32>(k);
        default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t stepk(const StepLaunch &L, int k) {
        switch (L.storage) {
        case LEE_STORE_BFP16: return stepk_io<TileIoBfp<S::Q>>(L, k);
        case LEE_STORE_F16: return stepk_io<TileIo16<__half>>(L, k);
        case LEE_STORE_BF16: return stepk_io<TileIo16<__nv_bfloat16>>(L, k);
        case LEE_STORE_F32: return stepk_io<TileIoF32>(L, k);
        default: return cudaErrorInvalidValue;
        }
    }
    // two steps per launch in 3D (axis-velocity sets; FP32 storage, or BFP16 with level 1 in FP32)
    // TMA-fed tile instantiations (one block per SM: the BFP16 tile needs 131 registers per thread
    // without spilling, and 88 per thread, for two blocks, spilled and ran slower): BFP16 with four
    // stages, FP32 with three
    using TmaBfp = T3tIoBfp<S::Q>;
    static cudaError_t step3d2_prepare(int storage, int tma) {
        if constexpr (!axis_only<S>()) {
            return cudaErrorInvalidValue;
        } else {
            if (tma) {
                if (storage == LEE_STORE_BFP16) return t3t_prepare<S, TmaBfp, kT3tRows, 4, 1>();
                return storage == LEE_STORE_F32 ? t3t_prepare<S, T3tIoF32, kT3tRows, 3, 1>() : cudaErrorInvalidValue;
            }
            if (storage == LEE_STORE_BFP16) return t3_prepare<S, Bfp16, kT3Rows>();
            return storage == LEE_STORE_F32 ? t3_prepare<S, float, kT3Rows>() : cudaErrorInvalidValue;
        }
    }
    static cudaError_t step3d2(const StepLaunch &L) {
        if constexpr (!axis_only<S>()) {
            return cudaErrorInvalidValue;
        } else {
            if (L.t3_tma) {
                if (L.storage == LEE_STORE_BFP16) return t3t_launch<S, TmaBfp, kT3tRows, 4, 1>(L);
                return L.storage == LEE_STORE_F32 ? t3t_launch<S, T3tIoF32, kT3tRows, 3, 1>(L) : cudaErrorInvalidValue;
            }
            if (L.storage == LEE_STORE_BFP16) return t3_launch<S, Bfp16, kT3Rows>(L);
            return L.storage == LEE_STORE_F32 ? t3_launch<S, float, kT3Rows>(L) : cudaErrorInvalidValue;
        }
    }
    static cudaError_t edge_fixup(const StepLaunch &L) {
        if constexpr (S::D != 2) {
            return cudaErrorInvalidValue;
        } else {
            return with_storage(L.storage, [&](auto *tp) -> cudaError_t {
                using T = std::remove_pointer_t<decltype(tp)>;
                using C = typename Store<T>::C;
                if constexpr (std::is_same<T, Bfp16>::value) {
                    return cudaErrorInvalidValue;  // no learned edge on BFP16 storage
                } else {
                    const GridDesc gd{L.nx, L.ny, 1, L.nx, (long long)L.nx * L.ny, L.pitch};
                    const CollideCoef<C> cf = make_coef<C>(L.omega, L.coefM, L.coefN);
                    const int nb = 2 * L.ny + 2 * (L.nx - 2);
                    k_edge_fixup<S, T><<<(nb + 127) / 128, 128, 0, L.stream>>>(
                        static_cast<const T *>(L.src), static_cast<T *>(L.dst), gd, cf, static_cast<const C *>(L.ghost),
                        L.ghost_L);
                    return cudaGetLastError();
                }
            });
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
        o.slab_pack = S::D >= 2 ? &slab_pack : nullptr;
        o.slab_unpack = S::D >= 2 ? &slab_unpack : nullptr;
        o.slab_crossing = slab_crossing<S>();
        o.onchip_1d = S::D == 1 ? &onchip_1d : nullptr;
        o.step2 = S::D == 2 ? &step2 : nullptr;
        o.step2_prepare = S::D == 2 ? &step2_prepare : nullptr;
        o.stepk = S::D == 2 ? &stepk : nullptr;
        o.stepk_prepare = S::D == 2 ? &stepk_prepare : nullptr;
        o.step3d2 = axis_only<S>() ? &step3d2 : nullptr;
        o.step3d2_prepare = axis_only<S>() ? &step3d2_prepare : nullptr;
        o.edge_fixup = S::D == 2 ? &edge_fixup : nullptr;
        for (int i = 0; i < S::Q; ++i) {
            for (int a = 0; a < 3; ++a) o.c[i][a] = S::c(i, a);
            o.shell[i] = S::shell(i);
        }
        return o;
    }
};

}  // namespace lee

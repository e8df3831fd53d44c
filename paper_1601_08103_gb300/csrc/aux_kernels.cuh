// aux_kernels.cuh -- auxiliary kernels of the solver (sm_103a): equilibrium initialisation,
// per-cell moments, FP64 reductions, sponge damping of an initial state, FP64 import/export.
// They run once per job, not per time step.
#pragma once

#include "kernels.cuh"

namespace lee {

// ---------------------------------------------------------------------------------------------
// auxiliary kernels: equilibrium initialisation, moments, reductions, FP64 import/export
// ---------------------------------------------------------------------------------------------

// Per-set FP64 constants for the auxiliary kernels (general form of Sec. 5).
struct SetConsts {
    double rho0, theta0, gamma, a1, a2, b, c1, c2;
    double f[4];     // f* per shell
    double beta[4];  // beta per shell
    double scale;    // 16-bit storage scale S (1 otherwise)
};

template <class S>
__device__ __forceinline__ double decode(double stored, int i, const SetConsts &k, bool scaled) {
    return scaled ? stored * (k.f[S::shell(i)] / k.scale) : stored;
}

// g_i = g_i^eq(rho', u', theta') (Sec. 7 initial condition), encoded into storage type T.
template <class S, class T>
__global__ void k_init_equilibrium(const double *__restrict__ rho, const double *__restrict__ u,
                                   const double *__restrict__ theta, T *__restrict__ g, long long cells, long long pitch,
                                   SetConsts k) {
    constexpr bool scaled = Store<T>::scaled;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        const double r = rho[x], th = theta[x];
        double uu[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < S::D; ++a) uu[a] = u[(long long)a * cells + x];
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int s = S::shell(i);
            double cu = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) cu += S::c(i, a) * uu[a];
            const double bracket = k.a1 * r + k.a2 * th + k.b * cu + 0.5 * (double)s * (k.c1 * r + k.c2 * th);
            const double v = scaled ? bracket * k.scale : bracket * k.f[s];
            g[(long long)i * pitch + x] = Store<T>::make((typename Store<T>::C)v);
        });
    }
}

// Largest |g_i^eq / f*_i| of the initial fields, as float bits for atomicMax (non-negative floats
// order like their bit patterns).
template <class S>
__global__ void k_init_maxabs(const double *__restrict__ rho, const double *__restrict__ u,
                              const double *__restrict__ theta, long long cells, SetConsts k,
                              unsigned int *__restrict__ maxbits) {
    float m = 0.f;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        const double r = rho[x], th = theta[x];
        double uu[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < S::D; ++a) uu[a] = u[(long long)a * cells + x];
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int s = S::shell(i);
            double cu = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) cu += S::c(i, a) * uu[a];
            const double bracket = k.a1 * r + k.a2 * th + k.b * cu + 0.5 * (double)s * (k.c1 * r + k.c2 * th);
            m = fmaxf(m, (float)fabs(bracket));
        });
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(m));
}

// Sponge damping of a stored post-collision state: g* <- (1 - sigma(d)) g* in the frame cells.
// Applied once after init_fields so that the initial state is a post-collision state like every
// later one (the equilibrium is its own collision; the frame damping is not).
template <class S, class T>
__global__ void k_sponge_damp(T *__restrict__ g, GridDesc gd, int w, typename Store<T>::C smax) {
    using C = typename Store<T>::C;
    const long long cells = (long long)gd.nx * gd.ny * gd.nz;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(x % gd.nx);
        const long long r = x / gd.nx;
        const int cy = (int)(r % gd.ny), cz = (int)(r / gd.ny);
        const C damp = sponge_factor<C>(cx, cy, cz, gd, S::D, w, smax);
        if (damp == C(1)) continue;
#pragma unroll
        for (int i = 0; i < S::Q; ++i) {
            T *p = g + (long long)i * gd.pitch + x;
            *p = Store<T>::make(Store<T>::load(*p) * damp);
        }
    }
}

// Per-cell moments (Sec. 4 discrete moments, Sec. 5 temperature) in FP64.
template <class S, class T>
__global__ void k_moments(const T *__restrict__ g, long long cells, long long pitch, SetConsts k, double *__restrict__ rho,
                          double *__restrict__ u, double *__restrict__ theta) {
    constexpr bool scaled = Store<T>::scaled;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        double r = 0.0, e = 0.0, j[3] = {0.0, 0.0, 0.0};
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int s = S::shell(i);
            const double v = decode<S>((double)Store<T>::load(g[(long long)i * pitch + x]), i, k, scaled);
            r += v;
#pragma unroll
            for (int a = 0; a < 3; ++a) j[a] += S::c(i, a) * v;
            e += 0.5 * ((double)s + k.beta[s]) * v;
        });
        if (rho) rho[x] = r;
        if (u) {
#pragma unroll
            for (int a = 0; a < S::D; ++a) u[(long long)a * cells + x] = j[a] / k.rho0;
        }
        if (theta) theta[x] = ((k.gamma - 1.0) * e - k.theta0 * r) / k.rho0;
    }
}

constexpr int kReduceThreads = 256;
constexpr int kReduceMax = 8;  // D + 4 <= 7 values, padded

// Block partial sums of the D + 4 diagnostics (see lee_lbm_reduce), fixed order per block.
template <class S, class T>
__global__ void __launch_bounds__(kReduceThreads) k_reduce_partial(const T *__restrict__ g, long long cells, long long pitch,
                                                                   SetConsts k, double *__restrict__ partial) {
    constexpr bool scaled = Store<T>::scaled;
    constexpr int NV = S::D + 4;
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int s = S::shell(i);
            const double v = decode<S>((double)Store<T>::load(g[(long long)i * pitch + x]), i, k, scaled);
            if (!isfinite(v)) {
                acc[NV - 1] += 1.0;
            } else {
                acc[0] += v;
#pragma unroll
                for (int a = 0; a < S::D; ++a) acc[1 + a] += S::c(i, a) * v;
                acc[S::D + 1] += 0.5 * ((double)s + k.beta[s]) * v;
                acc[S::D + 2] += v * v / k.f[s];
            }
        });
    }
    __shared__ double sh[kReduceThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double a = acc[v];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(kFull, a, off);
        if (lane == 0) sh[warp][v] = a;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double a = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) a += sh[w][threadIdx.x];
        partial[(long long)blockIdx.x * kReduceMax + threadIdx.x] = a;
    }
}

// Ordered sum of the block partials (one warp per output value).
__global__ void k_reduce_final(const double *__restrict__ partial, int nblocks, int nv, double *__restrict__ out);

// FP64 [q][cells] <-> storage (checkpoint export / import).
template <class S, class T>
__global__ void k_export(const T *__restrict__ g, long long cells, long long pitch, SetConsts k, double *__restrict__ out) {
    constexpr bool scaled = Store<T>::scaled;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            out[(long long)i * cells + x] = decode<S>((double)Store<T>::load(g[(long long)i * pitch + x]), i, k, scaled);
        });
    }
}

template <class S, class T>
__global__ void k_import(const double *__restrict__ in, long long cells, long long pitch, SetConsts k, T *__restrict__ g) {
    constexpr bool scaled = Store<T>::scaled;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int s = S::shell(i);
            const double v = in[(long long)i * cells + x];
            const double st = scaled ? v * (k.scale / k.f[s]) : v;
            g[(long long)i * pitch + x] = Store<T>::make((typename Store<T>::C)st);
        });
    }
}

}  // namespace lee

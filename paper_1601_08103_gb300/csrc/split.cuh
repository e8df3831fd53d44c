// split.cuh -- split storage (LEE_STORE_SPLIT16) for periodic grids: per cell the conserved
// moments m = (rho', j_1 .. j_D, E) in FP32 and the post-collision non-equilibrium parts
//     n*_i = (1 - w) (g_i - g_i^eq(m)),   w = 1 / tau,
// in FP16, stored as S n*_i / f*_i (S the power-of-two storage scale).  The post-collision state
// is g*_i = g_i^eq(m) + n*_i: BGK keeps m and scales the non-equilibrium part by 1 - w (Sec. 6),
// and H(tau) = (1 - w) I + w E with E the projection onto the equilibria (Sec. 8, the projection
// structure of H(1)).  Only the small n* is rounded to 16 bits.
//
// Per cell and copy this takes 4 (D + 2) + 2 q bytes: 58 B for D3Q19 against 76 B in FP32 and
// 38 B in FP16.  A pull step reconstructs every incoming population from the moments and the
// non-equilibrium part of the cell it comes from, so the moment arrays are read once per
// neighbour row (from cache) and once from DRAM.
//
// Layout of one state copy: moments [D + 2][pitch] FP32 (E last), then n [q][pitch] FP16.
#pragma once

#include "aux_kernels.cuh"

namespace lee {

// Coefficients in the arithmetic type (FP32).  With theta' = kE E - kR rho' and u' = j / rho0,
// the general equilibrium of Sec. 5 is linear in (rho', E, j):
//     g_i^eq = alpha_t rho' + beta_t E + gamma_t (c_i . j),   t = shell(i),
//     alpha_t = f*_t ((a1 + t c1 / 2) - kR (a2 + t c2 / 2)),  beta_t = f*_t kE (a2 + t c2 / 2),
//     gamma_t = f*_t b / rho0;
// E = sum_t ew_t P_t with P_t the shell sums; stored n <-> g units: g = dec_t x stored.
struct SplitCoef {
    float alpha[4], beta[4], gamma[4], ew[4], dec[4], enc[4];
    float one_minus_omega;
};

inline int split_bytes_per_cell(int D, int Q) { return 4 * (D + 2) + 2 * Q; }

// Row rowp at columns x0 - 1 .. x0 + V (periodic) as ext[0 .. V+1]: the thread's aligned vector,
// and one element on each side from the neighbouring lanes (or a scalar load at a row or warp
// edge).  Element e of the pull for c_x is ext[1 + e - c_x].
template <int V, class T>
__device__ __forceinline__ void split_row(const T *__restrict__ rowp, int x0, int nx, bool has_left, bool has_right,
                                          float (&ext)[V + 2]) {
    float v[V];
    load_vec<T, V>(rowp + x0, v);
    const float prev = __shfl_up_sync(kFull, v[V - 1], 1);
    const float next = __shfl_down_sync(kFull, v[0], 1);
    ext[0] = has_left ? prev : Store<T>::load(rowp[x0 == 0 ? nx - 1 : x0 - 1]);
#pragma unroll
    for (int e = 0; e < V; ++e) ext[1 + e] = v[e];
    ext[V + 1] = has_right ? next : Store<T>::load(rowp[x0 + V == nx ? 0 : x0 + V]);
}

// First velocity with the same source row offset (c_y, c_z) as velocity i.
template <class S>
__host__ __device__ constexpr int first_of_row(int i) {
    for (int j = 0; j < S::Q; ++j)
        if (S::c(j, 1) == S::c(i, 1) && S::c(j, 2) == S::c(i, 2)) return j;
    return -1;
}

// One step: every thread V consecutive cells of an x-row; all lanes of a warp take part in the
// shuffles (lanes past the end work on a clamped chunk and store nothing).  The moments of each
// source row (c_y, c_z) are loaded once and serve every velocity that pulls from that row.
// TILED (nx a multiple of 32 V): the 4 warps of a block take the same 32 V columns of 4
// consecutive y-rows of one z-plane, so the moment rows y-1 .. y+4 they pull from are shared in
// L1; otherwise threads take consecutive chunks of the grid in x, y, z order.
template <class S, int V, bool TILED>
__global__ void __launch_bounds__(128, 5) k_split_step(const float *__restrict__ msrc, const __half *__restrict__ nsrc,
                                                       float *__restrict__ mdst, __half *__restrict__ ndst, GridDesc gd,
                                                       SplitCoef cf) {
    constexpr int Q = S::Q, D = S::D, NM = D + 2;
    const int lane = threadIdx.x & 31;
    bool active;
    int xc, y, z;
    if constexpr (TILED) {
        const int nbx = gd.nxc / 32, nby = (gd.ny + 3) / 4;
        const long long b = blockIdx.x;
        xc = (int)(b % nbx) * 32 + lane;
        const long long t = b / nbx;
        y = (int)(t % nby) * 4 + (threadIdx.x >> 5);
        z = (int)(t / nby);
        if (y >= gd.ny) return;  // the whole warp: no shuffle partner is left behind
        active = true;
    } else {
        const long long raw = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        active = raw < gd.nchunks;
        const long long chunk = active ? raw : gd.nchunks - 1;
        chunk_coords(chunk, gd, xc, y, z);
    }
    const int x0 = xc * V;
    const bool has_left = lane > 0 && xc > 0, has_right = lane < 31 && xc < gd.nxc - 1;

    float g[Q][V];
    static_for<Q>([&](auto R) {
        constexpr int r = decltype(R)::value;
        if constexpr (first_of_row<S>(r) == r) {
            constexpr int cy = S::c(r, 1), cz = S::c(r, 2);
            int ys = y - cy, zs = z - cz;
            if (ys < 0) ys += gd.ny;
            if (ys >= gd.ny) ys -= gd.ny;
            if (zs < 0) zs += gd.nz;
            if (zs >= gd.nz) zs -= gd.nz;
            const long long rowoff = ((long long)zs * gd.ny + ys) * gd.nx;
            float m[NM][V + 2];
#pragma unroll
            for (int k = 0; k < NM; ++k)
                split_row<V>(msrc + (long long)k * gd.pitch + rowoff, x0, gd.nx, has_left, has_right, m[k]);
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                if constexpr (first_of_row<S>(i) == r) {
                    constexpr int cx = S::c(i, 0), t = S::shell(i);
                    float nn[V];
                    if constexpr (cx == 0) {
                        load_vec<__half, V>(nsrc + (long long)i * gd.pitch + rowoff + x0, nn);
                    } else {
                        float ext[V + 2];
                        split_row<V>(nsrc + (long long)i * gd.pitch + rowoff, x0, gd.nx, has_left, has_right, ext);
#pragma unroll
                        for (int e = 0; e < V; ++e) nn[e] = ext[1 + e - cx];
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const int o = 1 + e - cx;
                        float cj = 0.f;
                        static_for<D>([&](auto A) {
                            constexpr int a = decltype(A)::value;
                            if constexpr (S::c(i, a) == 1) cj += m[1 + a][o];
                            if constexpr (S::c(i, a) == -1) cj -= m[1 + a][o];
                        });
                        const float eq = fmaf(cf.alpha[t], m[0][o], fmaf(cf.beta[t], m[NM - 1][o], cf.gamma[t] * cj));
                        g[i][e] = fmaf(cf.dec[t], nn[e], eq);
                    }
                }
            });
        }
    });
    if (!active) return;  // no more shuffles below
    const long long cell0 = ((long long)z * gd.ny + y) * gd.nx + x0;
    float mo[NM][V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        float P[4] = {0.f, 0.f, 0.f, 0.f}, j[3] = {0.f, 0.f, 0.f};
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            P[S::shell(i)] += g[i][e];
            static_for<D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                if constexpr (S::c(i, a) == 1) j[a] += g[i][e];
                if constexpr (S::c(i, a) == -1) j[a] -= g[i][e];
            });
        });
        float rho = 0.f, E = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            rho += P[s];
            E = fmaf(cf.ew[s], P[s], E);
        }
        mo[0][e] = rho;
#pragma unroll
        for (int a = 0; a < D; ++a) mo[1 + a][e] = j[a];
        mo[NM - 1][e] = E;
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int t = S::shell(i);
            float cj = 0.f;
            static_for<D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                if constexpr (S::c(i, a) == 1) cj += j[a];
                if constexpr (S::c(i, a) == -1) cj -= j[a];
            });
            const float eq = fmaf(cf.alpha[t], rho, fmaf(cf.beta[t], E, cf.gamma[t] * cj));
            g[i][e] = cf.enc[t] * (cf.one_minus_omega * (g[i][e] - eq));  // stored n*
        });
    }
#pragma unroll
    for (int k = 0; k < NM; ++k) store_vec<float, V>(mdst + (long long)k * gd.pitch + cell0, mo[k]);
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        store_vec<__half, V>(ndst + (long long)i * gd.pitch + cell0, g[i]);
    });
}

// Initial state from FP64 fields: m = (rho', rho0 u', E) with E = (rho0 theta' + theta0 rho') /
// (gamma - 1) (the energy moment of g^eq, Secs. 4-5), and n* = 0 (g(0) = g^eq is its own
// collision).
template <class S>
__global__ void k_split_init(const double *__restrict__ rho, const double *__restrict__ u,
                             const double *__restrict__ theta, float *__restrict__ m, __half *__restrict__ n,
                             long long cells, long long pitch, SetConsts k) {
    constexpr int D = S::D, NM = D + 2;
    const double cT = k.rho0 / (k.gamma - 1.0), cR = k.theta0 / (k.gamma - 1.0);
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        const double r = rho[x];
        m[x] = (float)r;
#pragma unroll
        for (int a = 0; a < D; ++a) m[(long long)(1 + a) * pitch + x] = (float)(k.rho0 * u[(long long)a * cells + x]);
        m[(long long)(NM - 1) * pitch + x] = (float)fma(cT, theta[x], cR * r);
#pragma unroll
        for (int i = 0; i < S::Q; ++i) n[(long long)i * pitch + x] = __float2half_rn(0.f);
    }
}

// Post-collision populations of one cell in FP64, g*_i = g^eq_i(m) + dec_t n_i.
template <class S, class F>
__device__ __forceinline__ void split_cell(const float *__restrict__ m, const __half *__restrict__ n, long long pitch,
                                           long long x, const SetConsts &k, F &&put) {
    constexpr int D = S::D, NM = D + 2;
    const double r = (double)m[x], E = (double)m[(long long)(NM - 1) * pitch + x];
    double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < D; ++a) j[a] = (double)m[(long long)(1 + a) * pitch + x];
    // g^eq from (rho', u' = j / rho0, theta' = kE E - kR rho') with the init/moments coefficients
    const double th = fma(k.kE, E, -k.kR * r);
    double uu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) uu[a] = j[a] * k.inv_rho0;
    equilibrium_cell<S, 0>(r, th, uu, k, [&](int i, double eq) {
        const double st = (double)__half2float(n[(long long)i * pitch + x]);
        put(i, eq + k.dec[S::shell(i)] * st);
    });
}

template <class S>
__global__ void k_split_moments(const float *__restrict__ m, long long cells, long long pitch, SetConsts k,
                                double *__restrict__ rho, double *__restrict__ u, double *__restrict__ theta) {
    constexpr int D = S::D, NM = D + 2;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        const double r = (double)m[x];
        if (rho) rho[x] = r;
        if (u) {
#pragma unroll
            for (int a = 0; a < D; ++a) u[(long long)a * cells + x] = (double)m[(long long)(1 + a) * pitch + x] * k.inv_rho0;
        }
        if (theta) theta[x] = fma(k.kE, (double)m[(long long)(NM - 1) * pitch + x], -k.kR * r);
    }
}

template <class S>
__global__ void k_split_export(const float *__restrict__ m, const __half *__restrict__ n, long long cells,
                               long long pitch, SetConsts k, double *__restrict__ out) {
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x)
        split_cell<S>(m, n, pitch, x, k, [&](int i, double v) { out[(long long)i * cells + x] = v; });
}

// FP64 populations -> split state: m = their moments (rounded to FP32), n = S (g - g^eq(m)) / f*
// with g^eq taken at the rounded moments.
template <class S>
__global__ void k_split_import(const double *__restrict__ in, long long cells, long long pitch, SetConsts k,
                               float *__restrict__ m, __half *__restrict__ n) {
    constexpr int D = S::D, NM = D + 2;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        double P[4] = {0.0, 0.0, 0.0, 0.0}, j[3] = {0.0, 0.0, 0.0};
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const double v = in[(long long)i * cells + x];
            P[S::shell(i)] += v;
            static_for<D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                if constexpr (S::c(i, a) == 1) j[a] += v;
                if constexpr (S::c(i, a) == -1) j[a] -= v;
            });
        });
        double r = 0.0, E = 0.0;
        for (int s = 0; s < 4; ++s) {
            r += P[s];
            E = fma(k.ew[s], P[s], E);
        }
        m[x] = (float)r;
        for (int a = 0; a < D; ++a) m[(long long)(1 + a) * pitch + x] = (float)j[a];
        m[(long long)(NM - 1) * pitch + x] = (float)E;
        const double rf = (double)(float)r, Ef = (double)(float)E;
        double uu[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < D; ++a) uu[a] = (double)(float)j[a] * k.inv_rho0;
        equilibrium_cell<S, 0>(rf, fma(k.kE, Ef, -k.kR * rf), uu, k, [&](int i, double eq) {
            const double v = in[(long long)i * cells + x];
            n[(long long)i * pitch + x] = __float2half_rn((float)((v - eq) * k.enc[S::shell(i)]));
        });
    }
}

// Raw block sums of the reduction (see k_reduce_partial) over the reconstructed populations.
template <class S>
__global__ void __launch_bounds__(kReduceThreads) k_split_reduce_partial(const float *__restrict__ m,
                                                                         const __half *__restrict__ n, long long cells,
                                                                         long long pitch, SetConsts k,
                                                                         double *__restrict__ partial) {
    constexpr int NS = n_shells<S>(), D = S::D, NR = reduce_nraw<S>();
    double acc[NR];
#pragma unroll
    for (int v = 0; v < NR; ++v) acc[v] = 0.0;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        split_cell<S>(m, n, pitch, x, k, [&](int i, double v) {
            if (!isfinite(v)) {
                acc[NR - 1] += 1.0;
                return;
            }
            const int kk = shell_slot<S>(S::shell(i));
            acc[kk] += v;
            acc[NS + kk] = fma(v, v, acc[NS + kk]);
            for (int a = 0; a < D; ++a) acc[2 * NS + kk * D + a] += (double)S::c(i, a) * v;
        });
    }
    __shared__ double sh[kReduceThreads / 32][NR];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NR; ++v) {
        double a = acc[v];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(kFull, a, off);
        if (lane == 0) sh[warp][v] = a;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        double a = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) a += sh[w][threadIdx.x];
        partial[(long long)blockIdx.x * kReduceMax + threadIdx.x] = a;
    }
}

}  // namespace lee

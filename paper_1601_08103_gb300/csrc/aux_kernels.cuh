// aux_kernels.cuh -- auxiliary kernels of the solver (sm_103a): equilibrium initialisation,
// per-cell moments, FP64 reductions, sponge damping of an initial state, FP64 import/export.
// They run once per job, not per time step.
#pragma once

#include "bfp.cuh"

namespace lee {

// ---------------------------------------------------------------------------------------------
// auxiliary kernels: equilibrium initialisation, moments, reductions, FP64 import/export
// ---------------------------------------------------------------------------------------------

// Per-set FP64 constants for the auxiliary kernels (general form of Sec. 5).  The kernels work
// on per-shell sums (every weight and coefficient depends on the shell |c_i|^2 only), so the
// shell factors are folded on the host and each population costs one or two FP64 additions:
//   g_i^eq = eqA[.][s] rho' + eqB[.][s] theta' + eqC[.][s] (c_i . u')   (i in shell s;
//            [0] the population itself, [1] the scaled 16-bit value S g_i / f*_s, per unit S),
//   with eqA = F (a1 + s c1 / 2), eqB = F (a2 + s c2 / 2), eqC = F b, F = f*_s resp. 1;
//   a stored 16-bit value decodes as g = dec[s] x stored, dec = f*_s / S (enc = 1 / dec);
//   the energy moment weight of shell s is ew[s] = (s + beta_s) / 2;
//   u' = j / rho0 and theta' = kE e - kR rho' with kE = (gamma - 1) / rho0, kR = theta0 / rho0.
// (|c|^2 = s for every velocity of shell s.)
struct SetConsts {
    double rho0, theta0, gamma, a1, a2, b, c1, c2;
    double f[4];     // f* per shell
    double beta[4];  // beta per shell
    double scale;    // 16-bit storage scale S (1 otherwise)
    double eqA[2][4], eqB[2][4], eqC[2][4];
    double dec[4], enc[4], ew[4];
    double inv_rho0, kE, kR;
};

// Shells present in set S, in increasing order, and the compact slot of shell s.
template <class S>
__host__ __device__ constexpr int n_shells() {
    int n = 0;
    for (int s = 0; s < 4; ++s) n += shell_present<S>(s) ? 1 : 0;
    return n;
}
template <class S>
__host__ __device__ constexpr int shell_slot(int s) {
    int n = 0;
    for (int t = 0; t < s; ++t) n += shell_present<S>(t) ? 1 : 0;
    return n;
}

template <class S>
__device__ __forceinline__ double decode(double stored, int i, const SetConsts &k, bool scaled) {
    return scaled ? stored * k.dec[S::shell(i)] : stored;
}

// g_i^eq of one cell for every velocity: per shell two products, per velocity the signed sum of
// the velocity components it moves along and one fused multiply-add.
template <class S, int SC, class F>
__device__ __forceinline__ void equilibrium_cell(double r, double th, const double (&uu)[3], const SetConsts &k, F &&put) {
    double base[4];
    static_for<4>([&](auto Sx) {
        constexpr int s = decltype(Sx)::value;
        if constexpr (shell_present<S>(s)) base[s] = fma(k.eqB[SC][s], th, k.eqA[SC][s] * r);
    });
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int s = S::shell(i);
        constexpr bool moving = S::c(i, 0) != 0 || S::c(i, 1) != 0 || S::c(i, 2) != 0;
        if constexpr (!moving) {
            put(i, base[s]);
        } else {
            double cu = 0.0;
            bool first = true;
            static_for<3>([&](auto A) {
                constexpr int a = decltype(A)::value;
                constexpr int c = S::c(i, a);
                if constexpr (c != 0) {
                    const double t = c == 1 ? uu[a] : -uu[a];
                    cu = first ? t : cu + t;
                    first = false;
                }
            });
            put(i, fma(k.eqC[SC][s], cu, base[s]));
        }
    });
}

// g_i = g_i^eq(rho', u', theta') (Sec. 7 initial condition), encoded into storage type T.
template <class S, class T>
__global__ void k_init_equilibrium(const double *__restrict__ rho, const double *__restrict__ u,
                                   const double *__restrict__ theta, T *__restrict__ g, long long cells, long long pitch,
                                   SetConsts k) {
    constexpr int SC = Store<T>::scaled ? 1 : 0;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        double uu[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < S::D; ++a) uu[a] = u[(long long)a * cells + x];
        equilibrium_cell<S, SC>(rho[x], theta[x], uu, k, [&](int i, double v) {
            if (SC) v *= k.scale;
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
        double uu[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < S::D; ++a) uu[a] = u[(long long)a * cells + x];
        equilibrium_cell<S, 1>(rho[x], theta[x], uu, k, [&](int, double v) { m = fmaxf(m, (float)fabs(v)); });
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(m));
}

// One border cell (x, y) of an open 2D grid, pulled with the entering populations of the learned
// edge and collided: ghost(e, k) gives the population entering through edge e (0: x = 0, 1:
// x = nx - 1, 2: y = 0, 3: y = ny - 1) at position k along it.  The pulls follow the fused step's
// open-edge rules and the collision is collide_cell, so the cell gets what one step run with the
// ghosts throughout gives it (a corner takes one population from each of its two edges).
// `pulled(i, xs, ys)` gives the stored value of velocity i at source cell (xs, ys) inside the grid
// (edge_fixup_cell reads it from src).
template <class S, class T, class Ghost, class Pulled>
__device__ __forceinline__ void edge_fixup_cell_from(T *__restrict__ dst, const GridDesc &gd,
                                                     const CollideCoef<typename Store<T>::C> &cf, Ghost ghost,
                                                     Pulled pulled, int x, int y) {
    static_assert(S::D == 2, "border cells of 2D grids");
    using C = typename Store<T>::C;
    const int nx = gd.nx, ny = gd.ny;
    C pull[S::Q][1], post[S::Q][1];
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = S::c(i, 0), cy = S::c(i, 1);
        const int xs = x - cx, ys = y - cy;
        C v = C(0);
        if (ys < 0 || ys >= ny) {  // enters through the bottom (c_y = +1) or top edge
            if (cx == 0) v = ghost(cy == 1 ? 2 : 3, x);
        } else if (xs < 0) {  // through the left edge
            if (cy == 0) v = ghost(0, y);
        } else if (xs >= nx) {  // through the right edge
            if (cy == 0) v = ghost(1, y);
        } else {
            v = pulled(i, xs, ys);
        }
        pull[i][0] = v;
    });
    collide_cell<S, 0>(pull, post, cf);
#pragma unroll
    for (int i = 0; i < S::Q; ++i) dst[(long long)i * gd.pitch + (long long)y * nx + x] = Store<T>::make(post[i][0]);
}
template <class S, class T, class Ghost>
__device__ __forceinline__ void edge_fixup_cell(const T *__restrict__ src, T *__restrict__ dst, const GridDesc &gd,
                                                const CollideCoef<typename Store<T>::C> &cf, Ghost ghost, int x,
                                                int y) {
    edge_fixup_cell_from<S, T>(dst, gd, cf, ghost, [&](int i, int xs, int ys) {
        return Store<T>::load(src[(long long)i * gd.pitch + (long long)ys * gd.nx + xs]);
    }, x, y);
}

// The border cells of an open 2D grid for one step of the learned edge, from the step's source
// state and the network's entering populations (ghost[4][L]): one thread per border cell (corners
// belong to the x-edges).  The interior cells come from the step kernel, which leaves these cells
// unwritten (OpenEdge::skip_border), so the two can run at the same time.
template <class S, class T>
__global__ void k_edge_fixup(const T *__restrict__ src, T *__restrict__ dst, GridDesc gd,
                             CollideCoef<typename Store<T>::C> cf, const typename Store<T>::C *__restrict__ ghost,
                             int L) {
    using C = typename Store<T>::C;
    const int nx = gd.nx, ny = gd.ny;
    const int nb = 2 * ny + 2 * (nx - 2);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nb; r += gridDim.x * blockDim.x) {
        int x, y;
        if (r < ny) {
            x = 0;
            y = r;
        } else if (r < 2 * ny) {
            x = nx - 1;
            y = r - ny;
        } else if (r < 2 * ny + (nx - 2)) {
            x = 1 + (r - 2 * ny);
            y = 0;
        } else {
            x = 1 + (r - 2 * ny - (nx - 2));
            y = ny - 1;
        }
        edge_fixup_cell<S, T>(src, dst, gd, cf, [&](int e, int k) -> C { return ghost[e * L + k]; }, x, y);
    }
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

// Per-shell sums of one cell's stored populations: P[slot] = sum g, J[slot][a] = sum c_a g (in
// stored units), and whether every value is finite.
template <class S, class T>
__device__ __forceinline__ bool shell_sums(const T *__restrict__ g, long long pitch, long long x,
                                           double (&P)[n_shells<S>()], double (&J)[n_shells<S>()][3],
                                           double (&Sq)[n_shells<S>()]) {
    bool finite = true;
    static_for<n_shells<S>()>([&](auto K) {
        constexpr int k = decltype(K)::value;
        P[k] = 0.0;
        Sq[k] = 0.0;
        J[k][0] = J[k][1] = J[k][2] = 0.0;
    });
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int k = shell_slot<S>(S::shell(i));
        const double v = (double)load_elem<S, T>(g, pitch, (long long)i * pitch + x);
        finite = finite && isfinite(v);
        P[k] += v;
        Sq[k] = fma(v, v, Sq[k]);
        static_for<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr (S::c(i, a) == 1) J[k][a] += v;
            if constexpr (S::c(i, a) == -1) J[k][a] -= v;
        });
    });
    return finite;
}

// Per-cell moments (Sec. 4 discrete moments, Sec. 5 temperature) in FP64.
template <class S, class T>
__global__ void k_moments(const T *__restrict__ g, long long cells, long long pitch, SetConsts k, double *__restrict__ rho,
                          double *__restrict__ u, double *__restrict__ theta) {
    constexpr bool scaled = Store<T>::scaled;
    constexpr int NS = n_shells<S>();
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        double P[NS], J[NS][3], Sq[NS];
        shell_sums<S, T>(g, pitch, x, P, J, Sq);
        double r = 0.0, e = 0.0, j[3] = {0.0, 0.0, 0.0};
        static_for<4>([&](auto Sx) {
            constexpr int s = decltype(Sx)::value;
            if constexpr (shell_present<S>(s)) {
                constexpr int kk = shell_slot<S>(s);
                const double p = scaled ? P[kk] * k.dec[s] : P[kk];
                r += p;
                e = fma(k.ew[s], p, e);
#pragma unroll
                for (int a = 0; a < S::D; ++a) j[a] += scaled ? J[kk][a] * k.dec[s] : J[kk][a];
            }
        });
        if (rho) rho[x] = r;
        if (u) {
#pragma unroll
            for (int a = 0; a < S::D; ++a) u[(long long)a * cells + x] = j[a] * k.inv_rho0;
        }
        if (theta) theta[x] = fma(k.kE, e, -k.kR * r);
    }
}

constexpr int kReduceThreads = 256;
constexpr int kReduceMax = 16;  // raw accumulators per block (<= 16, see reduce_nraw)

// Raw accumulators of a reduction, per block: for every present shell (compact slot k)
//   [k] = sum g,  [NS + k] = sum g^2,  [2 NS + k D + a] = sum c_a g   (stored units),
// and [NR - 1] = number of non-finite values.  The weights come in when the block sums are
// combined (k_reduce_final): the paper's diagnostics are linear in these shell sums.
template <class S>
__host__ __device__ constexpr int reduce_nraw() {
    return 2 * n_shells<S>() + n_shells<S>() * S::D + 1;
}

template <class S, class T>
__global__ void __launch_bounds__(kReduceThreads) k_reduce_partial(const T *__restrict__ g, long long cells, long long pitch,
                                                                   double *__restrict__ partial) {
    constexpr int NS = n_shells<S>(), D = S::D, NR = reduce_nraw<S>();
    static_assert(NR <= kReduceMax, "raw accumulators do not fit");
    double acc[NR];
#pragma unroll
    for (int v = 0; v < NR; ++v) acc[v] = 0.0;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        double P[NS], J[NS][3], Sq[NS];
        if (!shell_sums<S, T>(g, pitch, x, P, J, Sq)) {
            // count the non-finite values of this cell; its finite ones still add up
            static_for<S::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const double v = (double)load_elem<S, T>(g, pitch, (long long)i * pitch + x);
                if (!isfinite(v)) acc[NR - 1] += 1.0;
            });
            static_for<S::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int k = shell_slot<S>(S::shell(i));
                const double v = (double)load_elem<S, T>(g, pitch, (long long)i * pitch + x);
                if (isfinite(v)) {
                    acc[k] += v;
                    acc[NS + k] = fma(v, v, acc[NS + k]);
                    static_for<D>([&](auto A) {
                        constexpr int a = decltype(A)::value;
                        if constexpr (S::c(i, a) == 1) acc[2 * NS + k * D + a] += v;
                        if constexpr (S::c(i, a) == -1) acc[2 * NS + k * D + a] -= v;
                    });
                }
            });
            continue;
        }
        static_for<NS>([&](auto K) {
            constexpr int k = decltype(K)::value;
            acc[k] += P[k];
            acc[NS + k] += Sq[k];
#pragma unroll
            for (int a = 0; a < D; ++a) acc[2 * NS + k * D + a] += J[k][a];
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

// How the raw block sums combine into the D + 4 diagnostics of lee_lbm_reduce:
//   sum rho' = sum_k dec_k P_k, sum j_a = sum_k dec_k J_ka, energy moment = sum_k ew_k dec_k P_k,
//   weighted energy = sum_k dec_k^2 Sq_k / f*_k, non-finite count (dec_k = 1 unless the storage
//   is scaled).
struct ReduceCombine {
    int D, ns, nraw;
    double dec[4], ew[4], f[4];  // per compact slot
};

// Ordered sum of the block partials (one warp per raw value) and the combination above; one
// block of 32 * nraw threads.
__global__ void k_reduce_final(const double *__restrict__ partial, int nblocks, ReduceCombine c, double *__restrict__ out);

// FP64 [q][cells] <-> storage (checkpoint export / import).
template <class S, class T>
__global__ void k_export(const T *__restrict__ g, long long cells, long long pitch, SetConsts k, double *__restrict__ out) {
    constexpr bool scaled = Store<T>::scaled;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (long long)gridDim.x * blockDim.x) {
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            out[(long long)i * cells + x] = decode<S>((double)load_elem<S, T>(g, pitch, (long long)i * pitch + x), i, k, scaled);
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
            const double st = scaled ? v * k.enc[s] : v;
            g[(long long)i * pitch + x] = Store<T>::make((typename Store<T>::C)st);
        });
    }
}

// ---------------------------------------------------------------------------------------------
// slab halos: a grid that is one slab of a periodic domain cut along its last axis
// ---------------------------------------------------------------------------------------------
// A population crosses the cut if its velocity moves along the last axis a = D - 1.  Messages hold
// one plane per crossing velocity, in the library's velocity order.
template <class S>
__host__ __device__ constexpr int slab_crossing() {
    int n = 0;
    for (int i = 0; i < S::Q; ++i) n += S::c(i, S::D - 1) == 1 ? 1 : 0;
    return n;
}
// Position of velocity i among the crossing velocities with c_a = sign.
template <class S>
__host__ __device__ constexpr int slab_slot(int i, int sign) {
    int n = 0;
    for (int j = 0; j < i; ++j) n += S::c(j, S::D - 1) == sign ? 1 : 0;
    return n;
}

// g points at the first owned cell of a state copy (velocity arrays `pitch` apart, each with one
// halo plane before the owned planes and one after).  Pack: the populations leaving downward
// (c_a = -1) from the first owned plane into send_lo, those leaving upward (c_a = +1) from the last
// owned plane into send_hi.
template <class S, class T>
__global__ void k_slab_pack(const T *__restrict__ g, long long pitch, long long plane, int nl, T *__restrict__ send_lo,
                            T *__restrict__ send_hi) {
    constexpr int a = S::D - 1;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < plane; x += (long long)gridDim.x * blockDim.x) {
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if constexpr (S::c(i, a) == -1)
                send_lo[(long long)slab_slot<S>(i, -1) * plane + x] = g[(long long)i * pitch + x];
            if constexpr (S::c(i, a) == 1)
                send_hi[(long long)slab_slot<S>(i, 1) * plane + x] = g[(long long)i * pitch + (long long)(nl - 1) * plane + x];
        });
    }
}
// Unpack: the populations entering from below (c_a = +1, the lower neighbour's send_hi) into the
// halo plane before the owned planes, those entering from above (c_a = -1) into the one after.
template <class S, class T>
__global__ void k_slab_unpack(T *__restrict__ g, long long pitch, long long plane, int nl, const T *__restrict__ recv_lo,
                              const T *__restrict__ recv_hi) {
    constexpr int a = S::D - 1;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < plane; x += (long long)gridDim.x * blockDim.x) {
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if constexpr (S::c(i, a) == 1)
                g[(long long)i * pitch - plane + x] = recv_lo[(long long)slab_slot<S>(i, 1) * plane + x];
            if constexpr (S::c(i, a) == -1)
                g[(long long)i * pitch + (long long)nl * plane + x] = recv_hi[(long long)slab_slot<S>(i, -1) * plane + x];
        });
    }
}

// ---------------------------------------------------------------------------------------------
// writers of BFP16 state (bfp.cuh): every block of 8 cells is encoded together
// ---------------------------------------------------------------------------------------------
// One thread per cell with whole warps in every iteration (the loop bound is warp-uniform), so the
// 8 lanes of a block share its exponent by shuffles; cells past the grid take part as zeros and
// store nothing.  `value(i, x)` gives the FP32 value of velocity i at cell x.
template <class S, class F>
__device__ __forceinline__ void bfp_write_cells(Bfp16 *__restrict__ g, long long cells, long long pitch, F &&value) {
    uint8_t *__restrict__ ex = bfp_exps<S::Q>(g, pitch);
    const long long n = (cells + kBfpBlock - 1) / kBfpBlock * kBfpBlock;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < n; w0 += stride) {
        const long long x = w0 + (threadIdx.x & 31);
        const bool valid = x < cells;
        float v[S::Q];
        value(valid ? x : -1, v);
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const long long e = (long long)i * pitch + x;
            const float one[1] = {v[i]};
            bfp_store_vec<1>(g + e, ex + (e >> 3), one, valid);
        });
    }
}

// g_i = g_i^eq(rho', u', theta') (Sec. 7 initial condition), rounded to FP32 and encoded.
template <class S>
__global__ void k_init_equilibrium_bfp(const double *__restrict__ rho, const double *__restrict__ u,
                                       const double *__restrict__ theta, Bfp16 *__restrict__ g, long long cells,
                                       long long pitch, SetConsts k) {
    bfp_write_cells<S>(g, cells, pitch, [&](long long x, float (&v)[S::Q]) {
        if (x < 0) {
#pragma unroll
            for (int i = 0; i < S::Q; ++i) v[i] = 0.f;
            return;
        }
        double uu[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < S::D; ++a) uu[a] = u[(long long)a * cells + x];
        equilibrium_cell<S, 0>(rho[x], theta[x], uu, k, [&](int i, double val) { v[i] = (float)val; });
    });
}

// FP64 [q][cells] -> BFP16 (resume): each value rounded to FP32, then encoded.
template <class S>
__global__ void k_import_bfp(const double *__restrict__ in, long long cells, long long pitch, Bfp16 *__restrict__ g) {
    bfp_write_cells<S>(g, cells, pitch, [&](long long x, float (&v)[S::Q]) {
#pragma unroll
        for (int i = 0; i < S::Q; ++i) v[i] = x < 0 ? 0.f : (float)in[(long long)i * cells + x];
    });
}

// Sponge damping of a stored BFP16 state (after init_fields): decoded, damped as in the FP32
// kernel, re-encoded (in place: each warp reads its blocks before it writes them).
template <class S>
__global__ void k_sponge_damp_bfp(Bfp16 *__restrict__ g, GridDesc gd, int w, float smax) {
    const long long cells = (long long)gd.nx * gd.ny * gd.nz;
    const uint8_t *ex = bfp_exps<S::Q>(g, gd.pitch);
    bfp_write_cells<S>(g, cells, gd.pitch, [&](long long x, float (&v)[S::Q]) {
        if (x < 0) {
#pragma unroll
            for (int i = 0; i < S::Q; ++i) v[i] = 0.f;
            return;
        }
        const int cx = (int)(x % gd.nx);
        const long long r = x / gd.nx;
        const int cy = (int)(r % gd.ny), cz = (int)(r / gd.ny);
        const float damp = sponge_factor<float>(cx, cy, cz, gd, S::D, w, smax);
#pragma unroll
        for (int i = 0; i < S::Q; ++i) v[i] = bfp_load1(g, ex, (long long)i * gd.pitch + x) * damp;
    });
}

}  // namespace lee

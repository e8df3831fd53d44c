// kernels.cuh -- device code of the lattice Boltzmann solver (sm_103a).
//
// Hot path: one fused pull-stream + BGK-collide kernel per time step (Sec. 6, eq. "LBE update
// scheme").  Populations live in structure-of-arrays layout, one array per velocity, x fastest,
// in a ping-pong pair of buffers.  With SoA and a pull step every stored population is read
// exactly once and written exactly once per step, so DRAM traffic equals the algorithmic
// 2 * q * sizeof(storage) bytes per cell without any shared-memory staging:
//   - each thread owns V consecutive cells of one x-row (one 16-byte vector per velocity);
//   - a velocity with c_x = 0 is a plain aligned vector load from row (y - c_y, z - c_z);
//   - c_x = +1 / -1 shifts the vector by one element: the missing element comes from the
//     neighbouring lane by warp shuffle, or by a scalar load at a row start or warp edge.
// The collision works on per-shell sums (all weights, additional energies and coefficients of
// the velocity sets depend on |c_i|^2 only), with the whole moment -> equilibrium -> relaxation
// chain folded on the host into two small matrices (see CollideCoef).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "velsets.cuh"

namespace lee {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------------------------
// compile-time loops
// ---------------------------------------------------------------------------------------------
template <class F, int... Is>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <class S>
__host__ __device__ constexpr bool shell_present(int s) {
    for (int i = 0; i < S::Q; ++i)
        if (S::shell(i) == s) return true;
    return false;
}

// ---------------------------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------------------------
template <class T>
struct Store;
template <>
struct Store<double> {
    using C = double;  // collision arithmetic type
    static constexpr bool scaled = false;
    __device__ static double load(double v) { return v; }
    __device__ static double make(double v) { return v; }
};
template <>
struct Store<float> {
    using C = float;
    static constexpr bool scaled = false;
    __device__ static float load(float v) { return v; }
    __device__ static float make(float v) { return v; }
};
template <>
struct Store<__half> {
    using C = float;
    static constexpr bool scaled = true;  // stores S * g / f*
    __device__ static float load(__half v) { return __half2float(v); }
    __device__ static __half make(float v) { return __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
    using C = float;
    static constexpr bool scaled = true;
    __device__ static float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 make(float v) { return __float2bfloat16_rn(v); }
};

template <int BYTES>
struct Raw;
template <>
struct Raw<16> { using type = uint4; };
template <>
struct Raw<8> { using type = uint2; };
template <>
struct Raw<4> { using type = unsigned int; };
template <>
struct Raw<2> { using type = unsigned short; };

// V consecutive elements starting at p (p aligned to V * sizeof(T)), read-only path.
template <class T, int V>
__device__ __forceinline__ void load_vec(const T *__restrict__ p, typename Store<T>::C (&out)[V]) {
    if constexpr (V * sizeof(T) == 8 && sizeof(T) == 8) {
        out[0] = Store<T>::load(__ldg(p));
    } else {
        using R = typename Raw<V * sizeof(T)>::type;
        union {
            R r;
            T e[V];
        } u;
        u.r = __ldg(reinterpret_cast<const R *>(p));
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = Store<T>::load(u.e[k]);
    }
}

template <class T, int V>
__device__ __forceinline__ void store_vec(T *__restrict__ p, const typename Store<T>::C (&in)[V]) {
    if constexpr (V * sizeof(T) == 8 && sizeof(T) == 8) {
        *p = Store<T>::make(in[0]);
    } else {
        using R = typename Raw<V * sizeof(T)>::type;
        union {
            R r;
            T e[V];
        } u;
#pragma unroll
        for (int k = 0; k < V; ++k) u.e[k] = Store<T>::make(in[k]);
        *reinterpret_cast<R *>(p) = u.r;
    }
}

// ---------------------------------------------------------------------------------------------
// kernel parameters
// ---------------------------------------------------------------------------------------------
struct GridDesc {
    int nx, ny, nz;
    int nxc;            // chunks per row = nx / V
    long long nchunks;  // nxc * ny * nz
    long long pitch;    // elements between consecutive velocity arrays
};

// (xc, y, z) of chunk c = xc + nxc (y + ny z): two 32-bit unsigned divisions while the grid has
// fewer than 2^32 chunks (a warp-uniform test), 64-bit divisions beyond.
__device__ __forceinline__ void chunk_coords(long long c, const GridDesc &gd, int &xc, int &y, int &z) {
    if (gd.nchunks <= 0xFFFFFFFFLL) {
        const unsigned u = (unsigned)c, nxc = (unsigned)gd.nxc, ny = (unsigned)gd.ny;
        const unsigned row = u / nxc;
        xc = (int)(u - row * nxc);
        const unsigned zz = row / ny;
        y = (int)(row - zz * ny);
        z = (int)zz;
    } else {
        const long long row = c / gd.nxc;
        xc = (int)(c - row * gd.nxc);
        const long long zz = row / gd.ny;
        y = (int)(row - zz * gd.ny);
        z = (int)zz;
    }
}

// Collision folded into shell space.  With P_s = sum_{i in shell s} g_i and
// J_s = sum_{i in shell s} c_i g_i, the post-collision population of velocity i in shell t is
//     g*_i = (1 - w) g_i + sum_s M[t][s] P_s + c_i . (sum_s N[t][s] J_s),     w = 1/tau,
// where M and N contain w, f*, the coefficients a1, a2, b, c1, c2, gamma, theta0, rho0 and the
// energies (|c|^2 + beta)/2 (built by the host; exact algebra of Secs. 4-6).
// Conservation of rho', j and the energy moment is an exact identity between these coefficients.
// To keep it exact in FP32 arithmetic, every coefficient is derived from the already rounded w,
// 1 - w is formed in the arithmetic type (exact for 1/2 <= w <= 2), and M is carried as a pair
// M + Mlo (Mlo = the rounding residual of M, zero when M is representable); N is w times a
// power of two for every set and needs no residual.  Rounding of the coefficients then adds no
// systematic drift; only the (unbiased) rounding of the arithmetic remains.
template <class C>
struct CollideCoef {
    C one_minus_omega;
    C M[4][4];
    C Mlo[4][4];
    C N[4][4];
};

// Open-edge treatment for non-periodic grids.
template <class C>
struct OpenEdge {
    int sponge_w;        // 0 = no sponge
    C sponge_smax;
    const C *ghost;      // nullptr = zero-incoming; else [4][L] entering populations (2D)
    int ghost_L;
    int skip_border;     // 2D: leave the border cells unwritten (the learned edge's kernels own them)
};

// ---------------------------------------------------------------------------------------------
// collision of one cell (index K of the per-thread vector)
// ---------------------------------------------------------------------------------------------
template <class S>
__host__ __device__ constexpr int first_in_shell(int s) {
    for (int i = 0; i < S::Q; ++i)
        if (S::shell(i) == s) return i;
    return -1;
}
template <class S>
__host__ __device__ constexpr int first_on_axis(int s, int a) {
    for (int i = 0; i < S::Q; ++i)
        if (S::shell(i) == s && S::c(i, a) != 0) return i;
    return -1;
}
template <class S>
__host__ __device__ constexpr int first_present_shell(int from) {
    for (int s = from; s < 4; ++s)
        if (shell_present<S>(s)) return s;
    return -1;
}

template <class S>
__host__ __device__ constexpr int moving_shells() {
    int n = 0;
    for (int s = 1; s < 4; ++s) n += shell_present<S>(s) ? 1 : 0;
    return n;
}

// Every rounding is spelled out so that no result depends on the compiler's contraction of a
// multiply and an add: with one moving shell the momentum term of velocity i is one fused
// multiply-add per axis, eq = fma(+-N[t][s1], J[s1][a], eq); with several moving shells the sums
// KJ[t][a] = sum_s N[t][s] J[s][a] (a chain of fused multiply-adds) are added to eq.
template <class S, int K, class C, int V>
__device__ __forceinline__ void collide_cell(const C (&g)[S::Q][V], C (&out)[S::Q][V], const CollideCoef<C> &cf) {
    // Accumulators start at -0.0 so that the first addition folds away exactly.
    C P[4] = {C(-0.0), C(-0.0), C(-0.0), C(-0.0)};
    C J[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s) J[s][0] = J[s][1] = J[s][2] = C(-0.0);
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int s = S::shell(i);
        const C v = g[i][K];
        P[s] += v;
        static_for<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr (S::c(i, a) == 1) J[s][a] += v;
            if constexpr (S::c(i, a) == -1) J[s][a] -= v;
        });
    });
    C B[4], KJ[4][3];
    static_for<4>([&](auto T) {
        constexpr int t = decltype(T)::value;
        if constexpr (shell_present<S>(t)) {
            C acc = C(-0.0);
            if constexpr (std::is_same<C, float>::value) {
                static_for<4>([&](auto Sx) {
                    constexpr int s = decltype(Sx)::value;
                    if constexpr (shell_present<S>(s)) acc = fma(cf.Mlo[t][s], P[s], acc);
                });
            }
            static_for<4>([&](auto Sx) {
                constexpr int s = decltype(Sx)::value;
                if constexpr (shell_present<S>(s)) acc = fma(cf.M[t][s], P[s], acc);
            });
            B[t] = acc;
            if constexpr (t > 0 && moving_shells<S>() > 1) {
                static_for<S::D>([&](auto A) {
                    constexpr int a = decltype(A)::value;
                    C kj = C(-0.0);
                    static_for<4>([&](auto Sx) {
                        constexpr int s = decltype(Sx)::value;
                        if constexpr (s > 0 && shell_present<S>(s)) kj = fma(cf.N[t][s], J[s][a], kj);
                    });
                    KJ[t][a] = kj;
                });
            }
        }
    });
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int t = S::shell(i);
        C eq = B[t];
        static_for<S::D>([&](auto A) {
            constexpr int a = decltype(A)::value;
            constexpr int c = S::c(i, a);
            if constexpr (c != 0 && moving_shells<S>() == 1) {
                constexpr int s1 = first_present_shell<S>(1);
                eq = fma(c == 1 ? cf.N[t][s1] : -cf.N[t][s1], J[s1][a], eq);
            } else if constexpr (c == 1) {
                eq += KJ[t][a];
            } else if constexpr (c == -1) {
                eq -= KJ[t][a];
            }
        });
        out[i][K] = fma(cf.one_minus_omega, g[i][K], eq);
    });
}

// FP32 collision of two cells (K, K+1) at once with the packed f32x2 add, mul and fma of sm_100
// and later.  Every packed operation rounds each half exactly like the scalar operation it
// replaces in collide_cell (a - b is a + (-b); a first accumulation into -0.0 is the value itself,
// or a plain product for the fma chains), so the result is the same bit for bit with half the FP
// instructions.
__device__ __forceinline__ float2 splat2(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

template <class S, int K, int V>
__device__ __forceinline__ void collide_pair(const float (&g)[S::Q][V], float (&out)[S::Q][V],
                                             const CollideCoef<float> &cf) {
    static_assert(K + 1 < V, "a pair needs two cells");
    float2 P[4], J[4][3];
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int s = S::shell(i);
        const float2 v = make_float2(g[i][K], g[i][K + 1]);
        if constexpr (i == first_in_shell<S>(s)) P[s] = v;
        else P[s] = __fadd2_rn(P[s], v);
        static_for<3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            constexpr int c = S::c(i, a);
            if constexpr (c != 0) {
                const float2 sv = c == 1 ? v : neg2(v);
                if constexpr (i == first_on_axis<S>(s, a)) J[s][a] = sv;
                else J[s][a] = __fadd2_rn(J[s][a], sv);
            }
        });
    });
    float2 B[4], KJ[4][3];
    static_for<4>([&](auto T) {
        constexpr int t = decltype(T)::value;
        if constexpr (shell_present<S>(t)) {
            constexpr int s0 = first_present_shell<S>(0);
            float2 acc;
            static_for<4>([&](auto Sx) {
                constexpr int s = decltype(Sx)::value;
                if constexpr (shell_present<S>(s)) {
                    if constexpr (s == s0) acc = __fmul2_rn(splat2(cf.Mlo[t][s]), P[s]);
                    else acc = __ffma2_rn(splat2(cf.Mlo[t][s]), P[s], acc);
                }
            });
            static_for<4>([&](auto Sx) {
                constexpr int s = decltype(Sx)::value;
                if constexpr (shell_present<S>(s)) acc = __ffma2_rn(splat2(cf.M[t][s]), P[s], acc);
            });
            B[t] = acc;
            if constexpr (t > 0 && moving_shells<S>() > 1) {
                constexpr int s1 = first_present_shell<S>(1);
                static_for<S::D>([&](auto A) {
                    constexpr int a = decltype(A)::value;
                    float2 kj;
                    static_for<4>([&](auto Sx) {
                        constexpr int s = decltype(Sx)::value;
                        if constexpr (s > 0 && shell_present<S>(s)) {
                            if constexpr (s == s1) kj = __fmul2_rn(splat2(cf.N[t][s]), J[s][a]);
                            else kj = __ffma2_rn(splat2(cf.N[t][s]), J[s][a], kj);
                        }
                    });
                    KJ[t][a] = kj;
                });
            }
        }
    });
    const float2 omm = splat2(cf.one_minus_omega);
    static_for<S::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int t = S::shell(i);
        float2 eq = B[t];
        static_for<S::D>([&](auto A) {
            constexpr int a = decltype(A)::value;
            constexpr int c = S::c(i, a);
            if constexpr (c != 0 && moving_shells<S>() == 1) {
                constexpr int s1 = first_present_shell<S>(1);
                eq = __ffma2_rn(splat2(c == 1 ? cf.N[t][s1] : -cf.N[t][s1]), J[s1][a], eq);
            } else if constexpr (c == 1) {
                eq = __fadd2_rn(eq, KJ[t][a]);
            } else if constexpr (c == -1) {
                eq = __fadd2_rn(eq, neg2(KJ[t][a]));
            }
        });
        const float2 r = __ffma2_rn(omm, make_float2(g[i][K], g[i][K + 1]), eq);
        out[i][K] = r.x;
        out[i][K + 1] = r.y;
    });
}

// All V cells of a chunk: FP32 pairs on the packed path, anything else one cell at a time (both
// give the same bits).
template <class S, bool PACK = true, class C, int V>
__device__ __forceinline__ void collide_chunk(const C (&g)[S::Q][V], C (&out)[S::Q][V], const CollideCoef<C> &cf) {
    if constexpr (PACK && std::is_same<C, float>::value && V % 2 == 0) {
        static_for<V / 2>([&](auto Kx) { collide_pair<S, 2 * decltype(Kx)::value>(g, out, cf); });
    } else {
        static_for<V>([&](auto Kx) { collide_cell<S, decltype(Kx)::value>(g, out, cf); });
    }
}

template <class C>
__device__ __forceinline__ C sponge_factor(int x, int y, int z, const GridDesc &gd, int D, int w, C smax) {
    int d = 0;
    const int p[3] = {x, y, z};
    const int n[3] = {gd.nx, gd.ny, gd.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            d = max(d, w - p[a]);
            d = max(d, p[a] - (n[a] - 1 - w));
        }
    }
    if (d <= 0) return C(1);
    const C r = C(d) / C(w);
    return fma(-(smax * r), r, C(1));  // 1 - smax r^2, one rounding of the product (smax r) r
}

// ---------------------------------------------------------------------------------------------
// fused pull-stream + collide, one time step
// ---------------------------------------------------------------------------------------------
// One thread's share of a step: V cells starting at chunk `raw` of the grid gd.  All 32 lanes of
// the warp must call this together (warp shuffles); lanes with raw >= nchunks compute on a clamped
// chunk and store nothing.  CUT (a slab of a larger periodic domain, cut along its last axis: y in
// 2D, z in 3D): along that axis nothing wraps -- the rows just before and after the grid are read
// where they lie in memory, in the halo planes the caller keeps there -- and every other axis is
// periodic.
template <class S, class T, int V, bool OPEN, bool CUT = false>
__device__ __forceinline__ void stream_collide_chunk(const T *__restrict__ src, T *__restrict__ dst, const GridDesc &gd,
                                                     const CollideCoef<typename Store<T>::C> &cf,
                                                     const OpenEdge<typename Store<T>::C> &ob, long long raw) {
    static_assert(!(CUT && OPEN), "a slab is periodic across its cut faces' neighbours");
    using C = typename Store<T>::C;
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
        if constexpr (cy != 0 && !(CUT && S::D == 2)) {
            if (ys < 0) { if constexpr (OPEN) row_out = true; else ys += gd.ny; }
            if (ys >= gd.ny) { if constexpr (OPEN) row_out = true; else ys -= gd.ny; }
        }
        if constexpr (cz != 0 && !(CUT && S::D == 3)) {
            if (zs < 0) { if constexpr (OPEN) row_out = true; else zs += gd.nz; }
            if (zs >= gd.nz) { if constexpr (OPEN) row_out = true; else zs -= gd.nz; }
        }
        const T *rowp = src + (long long)i * gd.pitch + ((long long)zs * gd.ny + ys) * gd.nx;
        C v[V];
        if (!row_out) {
            load_vec<T, V>(rowp + x0, v);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = C(0);
            if constexpr (OPEN && S::D == 2 && cx == 0) {
                if (ob.ghost != nullptr) {  // entering through the bottom (c_y = +1) or top edge
                    const C *gp = ob.ghost + (cy == 1 ? 2 : 3) * ob.ghost_L + x0;
#pragma unroll
                    for (int k = 0; k < V; ++k) v[k] = gp[k];
                }
            }
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
                left = out ? C(0) : Store<T>::load(rowp[xs]);
                if constexpr (OPEN && S::D == 2 && cy == 0) {
                    if (xs < 0 && ob.ghost != nullptr) left = ob.ghost[0 * ob.ghost_L + y];
                }
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
                right = out ? C(0) : Store<T>::load(rowp[xs]);
                if constexpr (OPEN && S::D == 2 && cy == 0) {
                    if (x0 + V >= gd.nx && ob.ghost != nullptr) right = ob.ghost[1 * ob.ghost_L + y];
                }
            }
#pragma unroll
            for (int k = 0; k < V - 1; ++k) pull[i][k] = v[k + 1];
            pull[i][V - 1] = right;
        }
    });

    C post[S::Q][V];
    // one cell at a time: this kernel streams at the memory bound, and the packed f32x2 pairs
    // (same bits) cost it 9 to 12 registers and occupancy
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

    if (active) {
        T *outp = dst + ((long long)z * gd.ny + y) * gd.nx + x0;
        if constexpr (OPEN && S::D == 2) {
            if (ob.skip_border) {
                if (y == 0 || y == gd.ny - 1) return;
                if (x0 == 0 || x0 + V >= gd.nx) {  // a chunk that holds x = 0 or x = nx - 1
                    static_for<S::Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
#pragma unroll
                        for (int k = 0; k < V; ++k) {
                            if (x0 + k >= 1 && x0 + k <= gd.nx - 2)
                                outp[(long long)i * gd.pitch + k] = Store<T>::make(post[i][k]);
                        }
                    });
                    return;
                }
            }
        }
        static_for<S::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            store_vec<T, V>(outp + (long long)i * gd.pitch, post[i]);
        });
    }
}

// All n steps of a small 1D grid in one launch: one block keeps both population copies in
// shared memory (in the storage type, so every step rounds exactly like the global-memory path)
// and synchronises between steps.  Same per-cell arithmetic as k_stream_collide, so the result
// equals n launches of it bit for bit.  The final state is written back to g (in place).
template <class S, class T>
__global__ void __launch_bounds__(1024) k_onchip_1d(T *__restrict__ g, int nx, long long pitch,
                                                    CollideCoef<typename Store<T>::C> cf,
                                                    OpenEdge<typename Store<T>::C> ob, bool open, long long nsteps) {
    using C = typename Store<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *bufA = reinterpret_cast<T *>(smem_raw);
    T *bufB = bufA + (size_t)S::Q * nx;
    for (int k = threadIdx.x; k < S::Q * nx; k += blockDim.x) bufA[k] = g[(long long)(k / nx) * pitch + k % nx];
    __syncthreads();
    const GridDesc gd{nx, 1, 1, nx, nx, nx};
    for (long long step = 0; step < nsteps; ++step) {
        const T *src = (step & 1) ? bufB : bufA;
        T *dst = (step & 1) ? bufA : bufB;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            C pull[S::Q][1], post[S::Q][1];
            static_for<S::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                int xs = x - S::c(i, 0);
                bool out = false;
                if (xs < 0) { if (open) out = true; else xs += nx; }
                if (xs >= nx) { if (open) out = true; else xs -= nx; }
                pull[i][0] = out ? C(0) : Store<T>::load(src[i * nx + xs]);
            });
            collide_cell<S, 0>(pull, post, cf);
            if (open && ob.sponge_w > 0) {
                const C damp = sponge_factor<C>(x, 0, 0, gd, 1, ob.sponge_w, ob.sponge_smax);
#pragma unroll
                for (int i = 0; i < S::Q; ++i) post[i][0] *= damp;
            }
#pragma unroll
            for (int i = 0; i < S::Q; ++i) dst[i * nx + x] = Store<T>::make(post[i][0]);
        }
        __syncthreads();
    }
    const T *fin = (nsteps & 1) ? bufB : bufA;
    for (int k = threadIdx.x; k < S::Q * nx; k += blockDim.x) g[(long long)(k / nx) * pitch + k % nx] = fin[k];
}

// One fused time step on one grid: one thread per V-cell chunk.
template <class S, class T, int V, bool OPEN, bool CUT = false>
__global__ void __launch_bounds__(256) k_stream_collide(const T *__restrict__ src, T *__restrict__ dst, GridDesc gd,
                                                        CollideCoef<typename Store<T>::C> cf,
                                                        OpenEdge<typename Store<T>::C> ob) {
    stream_collide_chunk<S, T, V, OPEN, CUT>(src, dst, gd, cf, ob, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------------------------
// two time steps per launch (temporal blocking) for periodic 2D FP32 grids with nx % 4 == 0
// ---------------------------------------------------------------------------------------------
// A block (4 warps) owns an output tile of kTbW = 128 columns x H rows (H a multiple of 4, chosen
// by the host so that all tiles are resident at once) and marches down it four rows per
// iteration, one row per warp, four cells (one float4) per lane.  Output row b at t+2 needs
// S(t+1) on rows b-1..b+1 and columns x0-1..x0+128, which needs S(t) on rows b-2..b+2 and
// columns x0-2..x0+129.  Per iteration k (rows relative to the tile):
//   A_k: S(t+1) rows 4k-1 .. 4k+2 (one per warp) are pulled from S(t) in global memory exactly as
//        in the one-step kernel (aligned float4 loads of rows y - c_y, x-neighbours by warp
//        shuffle, the two edge columns by scalar loads), collided, and written to slot k of a
//        3-slot shared-memory ring of 4-row blocks, together with the halo columns x0-1 and
//        x0+128 (one f32x2 pair in lane 0);
//   barrier;
//   B_k: S(t+2) rows 4k-4 .. 4k-1 are pulled from ring slots k-1 and k, collided and stored.
// A_{k+1} writes slot k+1, which no B_k reads, so one barrier per iteration separates every
// producer from its consumers, and the tile needs H/4 + 1 iterations.  S(t+1) is kept in the
// storage type, so every value is rounded exactly as in two single steps: the result equals them
// bit for bit.  DRAM sees one read and one write of every population per two steps, plus two
// halo rows above and below each tile that the neighbouring tiles (running at the same time)
// mostly serve from L2.  The ring is the only shared memory: 3 x 4 x q x (128 + 8) floats,
// 32.6 KB for D2Q5; with the registers of the load prefetch (below) five blocks (20 warps) fit on
// an SM.
constexpr int kTbW = 128;
constexpr int kTbV = kTbW / 32;            // cells per lane
constexpr int kTbRow = kTbW + 8;           // ring row: columns x0-4 .. x0+131 (x0-1 .. x0+128 used)
constexpr int kTbR1 = 3;                   // ring depth in 4-row blocks
constexpr int kTbMinBlocks = 5;            // blocks per SM the register budget is sized for
constexpr bool kTbPacked = true;           // collide a lane's cells as f32x2 pairs
// Grids whose two population copies take at most this many bytes also ask L2 for the rows of
// the iteration after next (prefetch.global.L2): measured on GB300 it gains 4 % on 2048^2 D2Q5
// FP32 (168 MB, about the L2's 129 MB) and loses 6 % on 4096^2 and 4 % on 8192^2.
constexpr long long kTbL2PrefetchMaxBytes = 256LL << 20;

template <class S>
constexpr int tb_smem_bytes() {
    return kTbR1 * 4 * S::Q * kTbRow * (int)sizeof(float);
}

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }

__device__ __forceinline__ void tb_st(float *p, const float (&v)[kTbV]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Pulls the four cells of one lane for velocity i from a ring row (offsets relative to x0-4):
// the lane's own cells sit at 4*lane+4; c_x = +1 takes one element from the left neighbour lane
// (or offset 3 for lane 0), c_x = -1 one from the right neighbour (or offset kTbW+4 for lane 31).
template <int cx>
__device__ __forceinline__ void tb_pull(const float *row, int lane, float (&out)[kTbV]) {
    const float4 t = *reinterpret_cast<const float4 *>(row + kTbV * lane + 4);
    const float v[4] = {t.x, t.y, t.z, t.w};
    if constexpr (cx == 0) {
#pragma unroll
        for (int e = 0; e < kTbV; ++e) out[e] = v[e];
    } else if constexpr (cx == 1) {
        float left = __shfl_up_sync(kFull, v[kTbV - 1], 1);
        if (lane == 0) left = row[3];
        out[0] = left;
#pragma unroll
        for (int e = 1; e < kTbV; ++e) out[e] = v[e - 1];
    } else {
        float right = __shfl_down_sync(kFull, v[0], 1);
        if (lane == 31) right = row[kTbW + 4];
#pragma unroll
        for (int e = 0; e + 1 < kTbV; ++e) out[e] = v[e + 1];
        out[kTbV - 1] = right;
    }
}

// One tile (columns x0 .. x0+kTbW-1, rows y0 .. y0+H-1) of two fused steps; the whole block calls
// it.  PF: also prefetch into L2 the rows of the iteration after next.
template <class S, bool PF>
__device__ __forceinline__ void tb_tile(const float *__restrict__ src, float *__restrict__ dst, int nx, int ny,
                                        long long pitch, int H, const CollideCoef<float> &cf, int x0, int y0,
                                        float *tb_smem) {
    static_assert(S::D == 2, "two-step tiles are 2D");
    constexpr int Q = S::Q;
    auto r1 = [&](int blk, int w, int i) { return tb_smem + (((blk % kTbR1) * 4 + w) * Q + i) * kTbRow; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int iters = H / 4 + 1;

    // Periodic columns, fixed for the tile: the lane's float4 (nx is a multiple of 4, so a chunk
    // never straddles the wrap; columns of the last strip past nx hold the periodic continuation
    // of the row) and the scalar columns x0-2 .. x0 and x0+127 .. x0+129 of the edges.
    auto wrap_x = [&](int x) {
        x %= nx;
        return x < 0 ? x + nx : x;
    };
    const int xa = wrap_x(x0 + kTbV * lane);
    int xe[6];  // columns x0-2, x0-1, x0, x0+127, x0+128, x0+129
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        xe[e] = wrap_x(x0 - 2 + e);
        xe[3 + e] = wrap_x(x0 + kTbW - 1 + e);
    }
    // Loads of pass A are issued one iteration ahead into registers, so their latency overlaps
    // the barrier and pass B of the iteration before.  Row a = y0 - 1 + 4k + warp of S(t+1) needs
    // S(t) rows a-1, a, a+1; rn is row a of the next iteration to load, reduced modulo ny.
    struct Pre {
        float4 t[Q];      // the lane's four cells of velocity i from row a - c_y
        float edge[Q];    // lane 0: column x0-1 (c_x = +1); lane 31: column x0+128 (c_x = -1)
        float halo[Q][2]; // lane 0: the pulls of the halo columns x0-1 and x0+128
    };
    Pre pre;
    int rn = (y0 - 1 + warp) % ny;
    if (rn < 0) rn += ny;
    auto load_a = [&](int k) {  // called once for each k = 0, 1, 2, ... in this order
        const int a = y0 - 1 + 4 * k + warp;
        if (a <= y0 + H) {
            const int rows[3] = {rn == 0 ? ny - 1 : rn - 1, rn, rn + 1 == ny ? 0 : rn + 1};  // a-1, a, a+1
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = S::c(i, 0), cy = S::c(i, 1);
                const float *rowp = src + (long long)i * pitch + (long long)rows[1 - cy] * nx;
                pre.t[i] = __ldg(reinterpret_cast<const float4 *>(rowp + xa));
                if constexpr (cx == 1) {
                    if (lane == 0) pre.edge[i] = __ldg(rowp + xe[1]);
                } else if constexpr (cx == -1) {
                    if (lane == 31) pre.edge[i] = __ldg(rowp + xe[4]);
                }
                if (lane == 0) {  // cell x pulls velocity i from column x - c_x
                    pre.halo[i][0] = __ldg(rowp + xe[1 - cx]);
                    pre.halo[i][1] = __ldg(rowp + xe[4 - cx]);
                }
            });
        }
        rn += 4;
        while (rn >= ny) rn -= ny;  // at most two passes: ny >= 3
        if constexpr (PF) {
            // one lane per 128-byte line of the warp's 512 bytes, only for rows the tile needs
            if ((lane & 7) == 0 && a + 4 <= y0 + H) {
                const int rows2[3] = {rn == 0 ? ny - 1 : rn - 1, rn, rn + 1 == ny ? 0 : rn + 1};
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int cy = S::c(i, 1);
                    prefetch_l2(src + (long long)i * pitch + (long long)rows2[1 - cy] * nx + xa);
                });
            }
        }
    };
    load_a(0);

    // B_k: S(t+2) row b from S(t+1) rows b-1 .. b+1 of the ring, collided and stored.
    auto pass_b = [&](int b) {
        float pb[Q][kTbV];
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = S::c(i, 0), cy = S::c(i, 1);
            const int rr = b - cy - (y0 - 1);  // row within the S(t+1) blocks
            tb_pull<cx>(r1(rr >> 2, rr & 3, i), lane, pb[i]);
        });
        float post[Q][kTbV];
        collide_chunk<S, kTbPacked>(pb, post, cf);
        if (b < ny && x0 + kTbV * lane < nx) {
            float *outp = dst + (long long)b * nx + x0 + kTbV * lane;
#pragma unroll
            for (int i = 0; i < Q; ++i) tb_st(outp + (long long)i * pitch, post[i]);
        }
    };

    for (int k = 0; k < iters; ++k) {
        const int a = y0 - 1 + 4 * k + warp;
        if (a <= y0 + H) {  // warp-uniform; rows past y0 + H are not needed
            float pa[Q][kTbV];
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = S::c(i, 0);
                const float4 t = pre.t[i];
                if constexpr (cx == 0) {
                    pa[i][0] = t.x; pa[i][1] = t.y; pa[i][2] = t.z; pa[i][3] = t.w;
                } else if constexpr (cx == 1) {
                    float left = __shfl_up_sync(kFull, t.w, 1);
                    if (lane == 0) left = pre.edge[i];
                    pa[i][0] = left; pa[i][1] = t.x; pa[i][2] = t.y; pa[i][3] = t.z;
                } else {
                    float right = __shfl_down_sync(kFull, t.x, 1);
                    if (lane == 31) right = pre.edge[i];
                    pa[i][0] = t.y; pa[i][1] = t.z; pa[i][2] = t.w; pa[i][3] = right;
                }
            });
            float post[Q][kTbV];
            collide_chunk<S, kTbPacked>(pa, post, cf);
#pragma unroll
            for (int i = 0; i < Q; ++i) tb_st(r1(k, warp, i) + kTbV * lane + 4, post[i]);
            // the two halo columns of S(t+1), x0 - 1 (offset 3) and x0 + 128 (offset kTbW + 4), as
            // one pair in lane 0
            if (lane == 0) {
                float q1[Q][2];
                collide_chunk<S, kTbPacked>(pre.halo, q1, cf);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    r1(k, warp, i)[3] = q1[i][0];
                    r1(k, warp, i)[kTbW + 4] = q1[i][1];
                }
            }
        }
        if (k + 1 < iters) load_a(k + 1);
        __syncthreads();  // A_k complete and visible; every B_{k-1} done (slot k+1 is free)
        // B_k: rows y0 + 4k - 4 .. y0 + 4k - 1 from slots k-1, k
        if (k >= 1) pass_b(y0 + 4 * k - 4 + warp);
    }
}

template <class S, bool PF>
__global__ void __launch_bounds__(128, kTbMinBlocks) k_stream_collide_2step(const float *__restrict__ src,
                                                                            float *__restrict__ dst, int nx, int ny,
                                                                            long long pitch, int H,
                                                                            CollideCoef<float> cf) {
    extern __shared__ __align__(16) float tb_smem[];
    tb_tile<S, PF>(src, dst, nx, ny, pitch, H, cf, blockIdx.x * kTbW, blockIdx.y * H, tb_smem);
}

// Two fused steps over many periodic domains.  Block b works on tile tiles[b] = (domain,
// x0, y0) of height doms[domain].H; the host orders the tiles largest first so that the block
// scheduler balances uneven domains.
struct TbDomain {
    int nx, ny, H;
    long long pitch, offset;
    CollideCoef<float> cf;
};

template <class S>
__global__ void __launch_bounds__(128, kTbMinBlocks) k_stream_collide_2step_batched(const float *__restrict__ src,
                                                                      float *__restrict__ dst,
                                                                      const TbDomain *__restrict__ doms,
                                                                      const int3 *__restrict__ tiles) {
    extern __shared__ __align__(16) float tb_smem[];
    const int3 tl = tiles[blockIdx.x];
    const TbDomain &D = doms[tl.x];
    tb_tile<S, false>(src + D.offset, dst + D.offset, D.nx, D.ny, D.pitch, D.H, D.cf, tl.y, tl.z, tb_smem);
}

// ---------------------------------------------------------------------------------------------
// K time steps per launch (deeper temporal blocking), periodic 2D FP32 grids with nx % 4 == 0
// ---------------------------------------------------------------------------------------------
// The two-step tile generalised to K levels (K = 4 by default, 3 on request), without the L2
// prefetch (this kernel is issue bound; the prefetch cost 3.5 % on 2048^2).  Level l
// (1 <= l < K) is S(t+l) on rows y0-(K-l) .. y0+H-1+(K-l) and columns x0-(K-l) .. x0+127+(K-l)
// of the tile; it lives in its own 2-slot ring of 4-row blocks (block j of level l holds rows
// y0-(K-l)+4j .. y0-(K-l)+4j+3, one per row warp).  Level K is the output tile, stored to global
// memory.  Iteration k runs
//   level 1, block k: pulled from S(t) in global memory (loads issued one iteration ahead);
//   barrier;
//   level l = 2 .. K-1, block k-(l-1): pulled from blocks k-(l-1) and k-l+2 of level l-1; barrier;
//   level K, block k-(K-1): likewise, and stored.
// Level l, block j reads blocks j+1 (written in the interval just before) and j (one iteration
// earlier) of level l-1, and overwrites the slot of its own block j-2, which level l+1 last read
// one iteration earlier; so two slots per ring suffice with one barrier per level: K-1 barriers
// per iteration and H/4 + K - 1 iterations per tile.  A block has four row warps (128 columns of
// one row each) and a fifth warp for the K-l halo columns on each side of every level l < K, for
// all four rows at once.  Every level is rounded to FP32 exactly like a stored state, so the
// result equals K single steps bit for bit.  Shared memory: K-1 rings of 2 x 4 x q x (128+8)
// floats, 65.3 KB for four levels of D2Q5 (three blocks = 15 warps per SM).
//
// Measured on GB300 (D2Q5, GLUPS on 2048^2 / 4096^2 / 8192^2): two steps per launch 284 / 298 /
// 290; three levels with 3-slot rings and one barrier per iteration 351 / 388 / 409; four levels
// that way (98 KB, two blocks per SM) 352 / 392 / 365; four levels with 2-slot rings and the halo
// cells in each row warp 391 / 475 / 499, and 402 / 473 / 498 without the L2 prefetch; five levels
// (87 KB, two blocks per SM) 396 / 429 / 395; two warps per row 308 / 384 / 401.  Integer work is
// about as large as the floating-point work here, so the ring is addressed as an 8-row circular
// buffer per level (410 / 480 / 505) and the iteration loop is unrolled by two with the parity
// known at compile time, which makes every buffer row a per-thread constant (419 / 491 / 517);
// the fifth warp for the halo cells then takes a scalar collision per level off each row warp
// (426 / 498 / 525).  Giving the halo cells to one of the four row warps instead lost 5-18 %: the
// barriers then wait for that warp.  The kernel is bound by instruction issue and latency, not
// DRAM (ncu: issue slots half busy), so the level count that keeps three blocks resident wins.
template <class S, int K>
constexpr int tbk_smem_bytes() {
    return (K - 1) * 2 * 4 * S::Q * kTbRow * (int)sizeof(float);
}
constexpr int kTbRows = 4;                       // row warps per block
constexpr int kTbkThreads = (kTbRows + 1) * 32;  // plus the halo warp
template <int K>
constexpr int tbk_min_blocks() {
    return K == 3 ? 4 : 3;
}

// Global-memory side of a K-level tile: how level 1 reads S(t) and level K writes S(t+K).  The
// levels in between are FP32 in shared memory whatever the storage.  A policy gives
//   Elem        the stored element type;
//   Vec / One   what a lane's aligned 4-cell load, resp. a single-cell load, leaves in registers
//               (the loads are issued one iteration ahead and widened only when used);
//   ld4, ld1    the loads at element index idx of the state copy `base` (pitch between velocity
//               arrays), cvt4 / cvt1 the widening to FP32;
//   st4         the store of a lane's 4 cells at idx (every lane of the warp calls it; `store`
//               false for lanes that own no cells).
// FP32 storage: plain float4 / float accesses (the stored state is the FP32 state).
struct TileIoF32 {
    using Elem = float;
    using Vec = float4;
    using One = float;
    __device__ static __forceinline__ Vec ld4(const float *__restrict__ base, long long, long long idx) {
        return __ldg(reinterpret_cast<const float4 *>(base + idx));
    }
    __device__ static __forceinline__ One ld1(const float *__restrict__ base, long long, long long idx) {
        return __ldg(base + idx);
    }
    __device__ static __forceinline__ void cvt4(const Vec &t, float (&v)[4]) {
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static __forceinline__ float cvt1(const One &t) { return t; }
    __device__ static __forceinline__ void st4(float *__restrict__ base, long long, long long idx, const float (&v)[4],
                                               bool store) {
        if (store) tb_st(base + idx, v);
    }
};

// FP16 / BF16 storage (S g / f*; the storage scale is folded into the collision coefficients, as
// in the one-step kernel): 8-byte loads of a lane's four values, widened to FP32.  The levels in
// between stay FP32 (the storage's 11 or 8 significant bits would otherwise be lost at every
// level); S(t+K) is rounded to the storage once per launch, to nearest even like a one-step store.
template <class T>
struct TileIo16 {
    using Elem = T;
    using Vec = uint2;
    using One = unsigned short;
    __device__ static __forceinline__ float widen(unsigned bits) {
        if constexpr (std::is_same<T, __half>::value) {
            return __half2float(__ushort_as_half((unsigned short)bits));
        } else {
            return __bfloat162float(__ushort_as_bfloat16((unsigned short)bits));
        }
    }
    __device__ static __forceinline__ Vec ld4(const T *__restrict__ base, long long, long long idx) {
        return __ldg(reinterpret_cast<const uint2 *>(base + idx));
    }
    __device__ static __forceinline__ One ld1(const T *__restrict__ base, long long, long long idx) {
        return __ldg(reinterpret_cast<const unsigned short *>(base + idx));
    }
    __device__ static __forceinline__ void cvt4(const Vec &t, float (&v)[4]) {
        v[0] = widen(t.x & 0xFFFFu);  // element idx sits in the low half
        v[1] = widen(t.x >> 16);
        v[2] = widen(t.y & 0xFFFFu);
        v[3] = widen(t.y >> 16);
    }
    __device__ static __forceinline__ float cvt1(const One &t) { return widen(t); }
    __device__ static __forceinline__ void st4(T *__restrict__ base, long long, long long idx, const float (&v)[4],
                                               bool store) {
        if (store) store_vec<T, 4>(base + idx, v);
    }
};

template <class S, int K, class IO>
__device__ __forceinline__ void tbk_tile(const typename IO::Elem *__restrict__ src, typename IO::Elem *__restrict__ dst,
                                         int nx, int ny, long long pitch, int H, const CollideCoef<float> &cf, int x0,
                                         int y0, float *smem) {
    static_assert(S::D == 2 && K >= 3 && K <= 4, "deep tiles are 2D with three or four levels");
    constexpr int Q = S::Q;
    // The two 4-row slots of level l (1 .. K-1) form an 8-row circular buffer: row rr of the
    // level (counted from its first row) lives in buffer row rr & 7.  ring(l, r8) is velocity 0
    // of that row (velocity i at + i * kTbRow), column x0 at offset 4.
    auto ring = [&](int l, int r8) { return smem + ((l - 1) * 8 + r8) * Q * kTbRow; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Warps 0..3 compute the 128 columns of one row each; warp 4 computes the halo cells of all
    // four rows (h = K - l columns on each side at level l): lane L takes cell c = L mod 8h, on
    // row c / 2h of the block at offset hoff(h) from x0, and lanes L < 8h store it.
    const bool halo_warp = warp == kTbRows;
    const int iters = H / 4 + K - 1;
    auto wrap_x = [&](int x) {
        x %= nx;
        return x < 0 ? x + nx : x;
    };
    const int xa = wrap_x(x0 + kTbV * lane);
    // the element a lane's float4 lacks: column x0-1 for lane 0 (c_x = +1), x0+128 for lane 31
    // (c_x = -1)
    const int xedge = wrap_x(lane == 0 ? x0 - 1 : x0 + kTbW);
    auto hrow = [&](int h) { return (lane % (8 * h)) / (2 * h); };
    auto hoff = [&](int h) {
        const int c = (lane % (8 * h)) % (2 * h);
        return c < h ? c - h : kTbW + c - h;
    };
    constexpr int h1 = K - 1;
    const int w1 = halo_warp ? hrow(h1) : warp;  // the block row of this lane's level-1 work
    const int o1 = hoff(h1);
    // a level-1 halo cell pulls velocity i from column x0 + o1 - c_x = xh[1 - c_x]
    int xh[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) xh[e] = wrap_x(x0 + o1 - 1 + e);

    struct Pre {
        typename IO::Vec t[Q];     // row warps: the lane's four cells of velocity i from row a - c_y
        typename IO::One edge[Q];  // row warps, lanes 0 and 31: the element the four cells lack
        typename IO::One halo[Q];  // halo warp: the level-1 halo cell's pull of velocity i
    };
    Pre pre;
    const int lim1 = y0 + H + K - 2;  // last level-1 row the tile needs
    int rn = (y0 - (K - 1) + w1) % ny;
    if (rn < 0) rn += ny;
    auto load_a = [&](int k) {  // called once for each k = 0, 1, 2, ... in this order
        const int a = y0 - (K - 1) + 4 * k + w1;
        if (a <= lim1) {
            const int rows[3] = {rn == 0 ? ny - 1 : rn - 1, rn, rn + 1 == ny ? 0 : rn + 1};  // a-1, a, a+1
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = S::c(i, 0), cy = S::c(i, 1);
                const long long rb = (long long)i * pitch + (long long)rows[1 - cy] * nx;
                if (!halo_warp) {
                    pre.t[i] = IO::ld4(src, pitch, rb + xa);
                    if constexpr (cx == 1) {
                        if (lane == 0) pre.edge[i] = IO::ld1(src, pitch, rb + xedge);
                    } else if constexpr (cx == -1) {
                        if (lane == 31) pre.edge[i] = IO::ld1(src, pitch, rb + xedge);
                    }
                } else {
                    pre.halo[i] = IO::ld1(src, pitch, rb + xh[1 - cx]);
                }
            });
        }
        rn += 4;
        while (rn >= ny) rn -= ny;
    };
    load_a(0);

    // level l >= 2 (or K), block row w of block j: velocity i is pulled from row 4j + w + 1 - c_y
    // of level l-1 (whose rows start one earlier); rows[1 - c_y] points at those three rows.  JP
    // is the parity of j, known at compile time (the iteration loop is unrolled by two), so the
    // buffer rows are per-thread constants.
    auto src_rows = [&](int l, auto JP, int w, const float *(&rows)[3]) {
        constexpr int jp = decltype(JP)::value;
        rows[0] = ring(l - 1, (4 * jp + w) & 7);
        rows[1] = ring(l - 1, (4 * jp + w + 1) & 7);
        rows[2] = ring(l - 1, (4 * jp + w + 2) & 7);
    };
    auto pull_level = [&](const float *const (&rows)[3], float (&pb)[Q][kTbV]) {
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = S::c(i, 0), cy = S::c(i, 1);
            tb_pull<cx>(rows[1 - cy] + i * kTbRow, lane, pb[i]);
        });
    };
    // the halo cell at offset o, pulled from level l-1
    auto pull_halo = [&](const float *const (&rows)[3], int o, float (&hin)[Q][1]) {
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = S::c(i, 0), cy = S::c(i, 1);
            hin[i][0] = rows[1 - cy][i * kTbRow + 4 + o - cx];
        });
    };

    // iteration k; KP = k & 1 at compile time.  The conditions on rows are uniform in the row
    // warps (which shuffle) and per lane in the halo warp (which does not).
    auto iteration = [&](int k, auto KP) {
        constexpr int kp = decltype(KP)::value;
        // level 1, row 4k + w (rows of level l run to H - 1 + 2 (K - l) in that count)
        if (!halo_warp) {
            if (4 * k + warp <= H - 1 + 2 * (K - 1)) {
                float pa[Q][kTbV];
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int cx = S::c(i, 0);
                    float t[kTbV];
                    IO::cvt4(pre.t[i], t);
                    if constexpr (cx == 0) {
                        pa[i][0] = t[0]; pa[i][1] = t[1]; pa[i][2] = t[2]; pa[i][3] = t[3];
                    } else if constexpr (cx == 1) {
                        float left = __shfl_up_sync(kFull, t[3], 1);
                        if (lane == 0) left = IO::cvt1(pre.edge[i]);
                        pa[i][0] = left; pa[i][1] = t[0]; pa[i][2] = t[1]; pa[i][3] = t[2];
                    } else {
                        float right = __shfl_down_sync(kFull, t[0], 1);
                        if (lane == 31) right = IO::cvt1(pre.edge[i]);
                        pa[i][0] = t[1]; pa[i][1] = t[2]; pa[i][2] = t[3]; pa[i][3] = right;
                    }
                });
                float post[Q][kTbV];
                collide_chunk<S, kTbPacked>(pa, post, cf);
                float *dst1 = ring(1, 4 * kp + warp);
#pragma unroll
                for (int i = 0; i < Q; ++i) tb_st(dst1 + i * kTbRow + kTbV * lane + 4, post[i]);
            }
        } else if (4 * k + w1 <= H - 1 + 2 * (K - 1)) {
            float hin[Q][1], hout[Q][1];
#pragma unroll
            for (int i = 0; i < Q; ++i) hin[i][0] = IO::cvt1(pre.halo[i]);
            collide_chunk<S, kTbPacked>(hin, hout, cf);
            if (lane < 8 * h1) {
                float *dst1 = ring(1, (4 * kp + w1) & 7);
#pragma unroll
                for (int i = 0; i < Q; ++i) dst1[i * kTbRow + 4 + o1] = hout[i][0];
            }
        }
        if (k + 1 < iters) load_a(k + 1);
        __syncthreads();  // level-1 block k visible; every read of the slots written below is done
        static_for<K - 2>([&](auto Lx) {
            constexpr int l = 2 + decltype(Lx)::value;
            constexpr int h = K - l;
            constexpr int jp = (kp - (l - 1)) & 1;
            const int j = k - (l - 1);
            if (!halo_warp) {
                if (j >= 0 && 4 * j + warp <= H - 1 + 2 * (K - l)) {
                    const float *rows[3];
                    src_rows(l, std::integral_constant<int, jp>{}, warp, rows);
                    float pb[Q][kTbV], post[Q][kTbV];
                    pull_level(rows, pb);
                    collide_chunk<S, kTbPacked>(pb, post, cf);
                    float *dstl = ring(l, 4 * jp + warp);
#pragma unroll
                    for (int i = 0; i < Q; ++i) tb_st(dstl + i * kTbRow + kTbV * lane + 4, post[i]);
                }
            } else {
                const int wh = hrow(h), o = hoff(h);
                if (j >= 0 && 4 * j + wh <= H - 1 + 2 * (K - l)) {
                    const float *rows[3];
                    src_rows(l, std::integral_constant<int, jp>{}, wh, rows);
                    float hin[Q][1], hout[Q][1];
                    pull_halo(rows, o, hin);
                    collide_chunk<S, kTbPacked>(hin, hout, cf);
                    if (lane < 8 * h) {
                        float *dstl = ring(l, (4 * jp + wh) & 7);
#pragma unroll
                        for (int i = 0; i < Q; ++i) dstl[i * kTbRow + 4 + o] = hout[i][0];
                    }
                }
            }
            __syncthreads();  // level l block j visible to level l+1
        });
        const int m = k - (K - 1);
        if (!halo_warp && m >= 0) {
            const float *rows[3];
            src_rows(K, std::integral_constant<int, (kp - (K - 1)) & 1>{}, warp, rows);
            float pb[Q][kTbV], post[Q][kTbV];
            pull_level(rows, pb);
            collide_chunk<S, kTbPacked>(pb, post, cf);
            const int d = y0 + 4 * m + warp;
            const bool st = d < ny && x0 + kTbV * lane < nx;
            const long long ob = (long long)d * nx + x0 + kTbV * lane;
#pragma unroll
            for (int i = 0; i < Q; ++i) IO::st4(dst, pitch, (long long)i * pitch + ob, post[i], st);
        }
    };
    int k = 0;
    for (; k + 1 < iters; k += 2) {
        iteration(k, std::integral_constant<int, 0>{});
        iteration(k + 1, std::integral_constant<int, 1>{});
    }
    if (k < iters) iteration(k, std::integral_constant<int, 0>{});
}

template <class S, int K, class IO = TileIoF32>
__global__ void __launch_bounds__(kTbkThreads, tbk_min_blocks<K>()) k_stream_collide_kstep(
    const typename IO::Elem *__restrict__ src, typename IO::Elem *__restrict__ dst, int nx, int ny, long long pitch,
    int H, CollideCoef<float> cf) {
    extern __shared__ __align__(16) float tb_smem[];
    tbk_tile<S, K, IO>(src, dst, nx, ny, pitch, H, cf, blockIdx.x * kTbW, blockIdx.y * H, tb_smem);
}

// K fused steps over many periodic domains: block b works on tile tiles[b] = (domain, x0, y0)
// of height doms[domain].H, exactly as the two-step batched kernel.
template <class S, int K>
__global__ void __launch_bounds__(kTbkThreads, tbk_min_blocks<K>()) k_stream_collide_kstep_batched(
    const float *__restrict__ src, float *__restrict__ dst, const TbDomain *__restrict__ doms,
    const int3 *__restrict__ tiles) {
    extern __shared__ __align__(16) float tb_smem[];
    const int3 tl = tiles[blockIdx.x];
    const TbDomain &D = doms[tl.x];
    tbk_tile<S, K, TileIoF32>(src + D.offset, dst + D.offset, D.nx, D.ny, D.pitch, D.H, D.cf, tl.y, tl.z, tb_smem);
}

// Many independent periodic grids (one per domain) advanced by one launch.  Domain d owns the
// blocks [first_block[d], first_block[d+1]); its populations start at element offset[d] of the
// shared buffers, and it has its own extents and relaxation coefficients (its own tau).  The
// block -> domain map is a table, so a block never straddles two domains.
template <class C>
struct BatchDomain {
    GridDesc gd;
    CollideCoef<C> cf;
    long long offset;
    int first_block;
};

template <class S, class T, int V>
__global__ void __launch_bounds__(512) k_stream_collide_batched(const T *__restrict__ src, T *__restrict__ dst,
                                                                const BatchDomain<typename Store<T>::C> *__restrict__ doms,
                                                                const unsigned short *__restrict__ block_domain) {
    using C = typename Store<T>::C;
    const int d = block_domain[blockIdx.x];
    const BatchDomain<C> &D = doms[d];
    const long long raw = (long long)(blockIdx.x - D.first_block) * blockDim.x + threadIdx.x;
    const OpenEdge<C> none{0, C(0), nullptr, 0};
    stream_collide_chunk<S, T, V, false>(src + D.offset, dst + D.offset, D.gd, D.cf, none, raw);
}

}  // namespace lee

// onchip_cluster.cuh -- all steps of a small 1D grid in one launch of a thread-block cluster.
//
// The single-block on-chip kernel (k_onchip_1d) runs the whole grid on one SM; on GB300 that
// leaves an FP64 grid bound by one SM's FP64 pipe.  Here a cluster of kOnchipCluster CTAs splits
// the grid into contiguous segments, each double-buffered in its CTA's shared memory.  A cell
// whose pull source lies in another segment reads that CTA's shared memory (distributed shared
// memory, cluster.map_shared_rank); one cluster barrier per step makes every CTA's writes of the
// step visible before the next step reads them and keeps any CTA from overwriting a buffer that
// another one still reads.  The per-cell arithmetic is that of k_onchip_1d, so the result equals
// it (and single steps) bit for bit.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace lee {

constexpr int kOnchipCluster = 8;  // portable cluster size

template <class S, class T>
__global__ void __launch_bounds__(1024) k_onchip_1d_cluster(T *__restrict__ g, int nx, long long pitch,
                                                            CollideCoef<typename Store<T>::C> cf,
                                                            OpenEdge<typename Store<T>::C> ob, bool open,
                                                            long long nsteps) {
    namespace cg = cooperative_groups;
    using C = typename Store<T>::C;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int seg = (nx + kOnchipCluster - 1) / kOnchipCluster;  // cells per CTA (the last may hold fewer)
    const int xb = rank * seg;
    const int n_own = nx - xb < seg ? (nx - xb > 0 ? nx - xb : 0) : seg;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf0 = reinterpret_cast<T *>(smem_raw);  // [2][Q][seg]
    for (int k = threadIdx.x; k < S::Q * n_own; k += blockDim.x) {
        const int i = k / n_own, x = k % n_own;
        buf0[i * seg + x] = g[(long long)i * pitch + xb + x];
    }
    cluster.sync();  // every segment is in place before anyone pulls across
    const GridDesc gd{nx, 1, 1, nx, nx, nx};
    for (long long step = 0; step < nsteps; ++step) {
        T *src = buf0 + (size_t)(step & 1) * S::Q * seg;
        T *dst = buf0 + (size_t)((step + 1) & 1) * S::Q * seg;
        for (int xl = threadIdx.x; xl < n_own; xl += blockDim.x) {
            const int x = xb + xl;
            C pull[S::Q][1], post[S::Q][1];
            static_for<S::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                int xs = x - S::c(i, 0);
                bool out = false;
                if (xs < 0) { if (open) out = true; else xs += nx; }
                if (xs >= nx) { if (open) out = true; else xs -= nx; }
                C v = C(0);
                if (!out) {
                    const int owner = xs / seg;
                    const T *p = owner == rank ? src : cluster.map_shared_rank(src, owner);
                    v = Store<T>::load(p[i * seg + (xs - owner * seg)]);
                }
                pull[i][0] = v;
            });
            collide_cell<S, 0>(pull, post, cf);
            if (open && ob.sponge_w > 0) {
                const C damp = sponge_factor<C>(x, 0, 0, gd, 1, ob.sponge_w, ob.sponge_smax);
#pragma unroll
                for (int i = 0; i < S::Q; ++i) post[i][0] *= damp;
            }
#pragma unroll
            for (int i = 0; i < S::Q; ++i) dst[i * seg + xl] = Store<T>::make(post[i][0]);
        }
        cluster.sync();
    }
    const T *fin = buf0 + (size_t)(nsteps & 1) * S::Q * seg;
    for (int k = threadIdx.x; k < S::Q * n_own; k += blockDim.x) {
        const int i = k / n_own, x = k % n_own;
        g[(long long)i * pitch + xb + x] = fin[i * seg + x];
    }
}

}  // namespace lee

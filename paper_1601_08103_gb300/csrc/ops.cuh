// ops.cuh -- per-velocity-set launch table.  Each translation unit set_*.cu instantiates the
// kernels of a few sets (so that the library compiles in parallel) and exports one SetOps per
// set; lee_lbm.cu only sees these tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "aux_kernels.cuh"

namespace lee {

// Launch description of one fused time step.
struct StepLaunch {
    int storage;         // lee_storage
    const void *src;
    void *dst;
    int nx, ny, nz;
    long long pitch;
    bool open;
    double omega;        // 1 / tau, already rounded to the arithmetic type (see fold_coefficients)
    double coefM[4][4];  // see CollideCoef (FP64 values, split into hi + lo for FP32 arithmetic)
    double coefN[4][4];
    int sponge_w;
    double sponge_smax;
    const void *ghost;   // float (or double for F64) [4][ghost_L], or nullptr
    int ghost_L;
    int force_scalar;    // 1: use the one-cell-per-thread variant (testing)
    int slab;            // 1: a slab cut along the last axis (halo planes at src/dst -/+ one plane)
    int bfp_cells;       // BFP16 one-step kernel: cells per lane (4 or 8), 0 = the default for the set
    double store_scale;  // storage scale S of the 16-bit and split forms (1 otherwise)
    // 3D two-step tile: 1 = the TMA-fed kernel (tb3d_tma.cuh), 0 = the register-fed one (tb3d.cuh);
    // for the TMA-fed kernel, where a timed-out stage wait is recorded (device-visible word, or
    // nullptr), the wait limit in ns (0: one second) and the test injection of such a timeout
    int t3_tma;
    // open 2D grids: 1 = leave the border cells unwritten (the learned edge writes them)
    int skip_border;
    unsigned *wait_flag;
    long long wait_ns;
    int t3_inject;
    cudaStream_t stream;
};

struct SetOps {
    int D, Q;
    // one fused pull-stream + collide step
    cudaError_t (*step)(const StepLaunch &);
    // two fused steps per launch (periodic 2D FP32 grids with nx % 4 == 0; nullptr otherwise):
    // reads L.src, writes the state two steps later into L.dst
    cudaError_t (*step2)(const StepLaunch &);
    // one-time set-up of the two-step kernel on the current device (outside stream capture)
    cudaError_t (*step2_prepare)();
    // k = 3 or 4 fused steps per launch on the same grids (FP32, or BFP16 with nx % 8 == 0), and
    // its one-time set-up for a storage type
    cudaError_t (*stepk)(const StepLaunch &, int k);
    cudaError_t (*stepk_prepare)(int k, int storage);
    // two fused steps per launch for the 3D axis-velocity sets (periodic; FP32 with nx % 4 == 0
    // or BFP16 with nx % 8 == 0; nullptr for other sets), and its one-time set-up for a storage type
    // and kernel (tma = 1: the TMA-fed tile, which also needs t3t_eligible grids)
    cudaError_t (*step3d2)(const StepLaunch &);
    cudaError_t (*step3d2_prepare)(int storage, int tma);
    // g = g^eq(fields) (fields FP64 on device)
    cudaError_t (*init)(int storage, const double *rho, const double *u, const double *theta, void *g, long long cells,
                        long long pitch, const SetConsts &k, cudaStream_t st);
    // max |g^eq / f*| of the fields into *maxbits (float bits; caller zeroes it)
    cudaError_t (*init_maxabs)(const double *rho, const double *u, const double *theta, long long cells, const SetConsts &k,
                               unsigned int *maxbits, cudaStream_t st);
    cudaError_t (*moments)(int storage, const void *g, long long cells, long long pitch, const SetConsts &k, double *rho,
                           double *u, double *theta, cudaStream_t st);
    // partial sums: writes nblocks * kReduceMax doubles
    cudaError_t (*reduce_partial)(int storage, const void *g, long long cells, long long pitch, const SetConsts &k,
                                  double *partial, int nblocks, cudaStream_t st);
    cudaError_t (*export_f64)(int storage, const void *g, long long cells, long long pitch, const SetConsts &k, double *out,
                              cudaStream_t st);
    cudaError_t (*import_f64)(int storage, const double *in, long long cells, long long pitch, const SetConsts &k, void *g,
                              cudaStream_t st);
    // all steps of a small 1D grid in one launch, in place on g (nullptr for 2D/3D sets);
    // returns cudaErrorInvalidValue when the grid does not fit in shared memory
    cudaError_t (*onchip_1d)(const StepLaunch &L, void *g, long long nsteps);
    // the border cells of an open 2D grid for one step of the learned edge (k_edge_fixup): pulled
    // from L.src with the entering populations L.ghost, collided, stored in L.dst; nullptr for 1D/3D
    cudaError_t (*edge_fixup)(const StepLaunch &L);
    // slab halos: packs the populations that leave through the cut faces (first owned plane,
    // c_last = -1 -> send_lo; last owned plane, c_last = +1 -> send_hi), or unpacks the entering
    // ones into the halo planes (recv_lo -> plane -1, c_last = +1; recv_hi -> plane nl, c_last = -1).
    // g: the first owned cell of the state copy; plane: cells per plane; nl: owned planes.
    cudaError_t (*slab_pack)(int storage, const void *g, long long pitch, long long plane, int nl, void *send_lo,
                             void *send_hi, cudaStream_t st);
    cudaError_t (*slab_unpack)(int storage, void *g, long long pitch, long long plane, int nl, const void *recv_lo,
                               const void *recv_hi, cudaStream_t st);
    // sponge-frame damping of a stored state (after init_fields)
    cudaError_t (*sponge_damp)(int storage, void *g, int nx, int ny, int nz, long long pitch, int w, double smax,
                               cudaStream_t st);
    // description for lee_velset_info
    int c[27][3];
    int shell[27];
    int slab_crossing;  // velocities that cross a cut along the last axis, per direction
};

const SetOps *set_ops(int set);

// 1/tau rounded to the arithmetic type of the storage (FP64 storage: FP64, else FP32).
inline double omega_for(int storage, double tau) {
    const double w = 1.0 / tau;
    return storage == LEE_STORE_F64 ? w : (double)(float)w;
}

// CollideCoef for arithmetic type C from FP64 coefficients (M split into hi + lo for FP32).
template <class C>
CollideCoef<C> make_coef(double omega, const double M[4][4], const double N[4][4]) {
    CollideCoef<C> cf;
    cf.one_minus_omega = (C)1 - (C)omega;
    for (int t = 0; t < 4; ++t)
        for (int s = 0; s < 4; ++s) {
            cf.M[t][s] = (C)M[t][s];
            cf.Mlo[t][s] = (C)(M[t][s] - (double)cf.M[t][s]);
            cf.N[t][s] = (C)N[t][s];
        }
    return cf;
}

// Grids the TMA-fed 3D two-step tile (tb3d_tma.cuh) takes: whole 128-column tiles along x, ny a
// multiple of its kT3tRows-row tiles and at least two of them, and a pitch that keeps the BFP16
// exponent arrays' strides multiples of 16 bytes.
constexpr int kT3tRows = 8;
inline bool t3t_eligible(int nx, int ny, long long pitch) {
    return nx > 0 && nx % 128 == 0 && ny % kT3tRows == 0 && ny >= 2 * kT3tRows && pitch % 128 == 0;
}

// Largest dynamic shared memory a block may use on this GPU (227 KB on sm_103a).
constexpr int kMaxOnchipSmem = 227 * 1024;

// Host-side velocity-set constants (the same compile-time tables the kernels use).
template <class S>
SetConsts host_consts(double scale) {
    SetConsts k{};
    k.rho0 = S::rho0;
    k.theta0 = S::theta0;
    k.gamma = S::gamma;
    k.a1 = S::a1;
    k.a2 = S::a2;
    k.b = S::b;
    k.c1 = S::c1;
    k.c2 = S::c2;
    for (int s = 0; s < 4; ++s) {
        k.f[s] = S::fs(s);
        k.beta[s] = S::betas(s);
    }
    k.scale = scale;
    for (int s = 0; s < 4; ++s) {
        const double fa = k.a1 + 0.5 * s * k.c1, fb = k.a2 + 0.5 * s * k.c2;
        k.eqA[0][s] = k.f[s] * fa;
        k.eqB[0][s] = k.f[s] * fb;
        k.eqC[0][s] = k.f[s] * k.b;
        k.eqA[1][s] = fa;
        k.eqB[1][s] = fb;
        k.eqC[1][s] = k.b;
        k.dec[s] = k.f[s] / scale;
        k.enc[s] = k.f[s] > 0.0 ? scale / k.f[s] : 0.0;
        k.ew[s] = 0.5 * (s + k.beta[s]);
    }
    k.inv_rho0 = 1.0 / k.rho0;
    k.kE = (k.gamma - 1.0) / k.rho0;
    k.kR = k.theta0 / k.rho0;
    return k;
}

// Combination of the raw per-shell block sums of k_reduce_partial (see ReduceCombine).
inline ReduceCombine make_reduce_combine(const SetOps *o, const SetConsts &k, bool scaled) {
    ReduceCombine c{};
    bool present[4] = {false, false, false, false};
    for (int i = 0; i < o->Q; ++i) present[o->shell[i]] = true;
    int n = 0;
    for (int s = 0; s < 4; ++s) {
        if (!present[s]) continue;
        c.dec[n] = scaled ? k.dec[s] : 1.0;
        c.ew[n] = k.ew[s];
        c.f[n] = k.f[s];
        ++n;
    }
    c.D = o->D;
    c.ns = n;
    c.nraw = 2 * n + n * o->D + 1;
    return c;
}

// Most blocks a grid-stride auxiliary kernel is launched with (16 per SM on 152 SMs).  The
// reduction writes one row of partials per block, so this is also the row count of every
// partial-sum buffer, including the fixed scratch of the allocation-free reduction.
constexpr int kMaxAuxBlocks = 152 * 16;

// Grid size for grid-stride auxiliary kernels.
inline int aux_blocks(long long cells, int threads = 256) {
    long long b = (cells + threads - 1) / threads;
    if (b > kMaxAuxBlocks) b = kMaxAuxBlocks;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace lee

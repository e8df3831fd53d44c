/*
 * lee_lbm.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for the Linearized Euler
 * Equations without background velocity (Otte & Frank, "Derivation and Analysis of Lattice
 * Boltzmann Schemes for the Linearized Euler Equations", arXiv:1601.08103).
 *
 * The library advances the BGK lattice Boltzmann equation of Sec. 6 (eq. "LBE update scheme"),
 *     g_i(t+1, x + c_i) = (1 - 1/tau) g_i(t, x) + (1/tau) g_i^eq(t, x),
 * whose equilibrium (Sec. 4 eq. "equilibrium" for monoatomic gases, Sec. 5 general form for
 * polyatomic gases) is linear in the fluctuations (rho', u', theta').  Time, space and velocities
 * are in lattice units (epsilon = dx = dt = 1).
 *
 * Conventions shared by all entry points
 * -------------------------------------
 *  - Cell index: cell = x + nx * (y + ny * z); unused dimensions have extent 1.
 *  - Field layout (FP64): rho[cells], u[D][cells] (component-major), theta[cells].
 *  - Population layout (FP64 in the API): g[q][cells] in the library's velocity order, which
 *    lee_velset_info() reports.
 *  - State: the device buffer holds the POST-collision populations of the current time t,
 *    g*(t) = (1 - 1/tau) g(t) + (1/tau) g^eq(g(t)) (then damped inside a sponge frame); the next
 *    step pulls g_i(t+1, x) = g*_i(t, x - c_i) and collides it.  Right after init_fields,
 *    g*(0) = g(0) = g^eq(IC) (Sec. 7 initial condition), which is its own collision (times the
 *    frame damping inside a sponge frame).
 *  - Collision keeps rho', u' and theta' of every cell, so moments of g*(t) are those of g(t)
 *    (except inside a sponge frame, where they include that step's damping).
 *  - Ownership: the handle owns all device memory it allocates; caller buffers are only read or
 *    written during the call.  `on_device` = 1 means the pointer is CUDA device memory usable on
 *    the handle's stream, 0 means host memory (pageable or pinned).
 *  - Asynchrony: every call is enqueued on the handle's stream.  Calls that read or write host
 *    memory synchronise that stream before returning; device-pointer calls do not.
 *  - Host buffers of init_fields and moments that are page-locked and mapped into the device's
 *    address space (cudaHostAlloc, or cudaHostRegister with mapping) are read or written in place
 *    by the kernels -- over NVLink-C2C on a GB300 -- instead of through a staging copy; pageable
 *    host memory goes through device staging.  Either way the call returns after its work.
 *  - Errors: every call returns a lee_status; no call throws or aborts.  After LEE_ERR_CUDA or
 *    LEE_ERR_TIMEOUT the handle is poisoned: every later call except destroy returns
 *    LEE_ERR_POISONED.  lee_lbm_last_error() gives a one-line reason.
 */
#ifndef LEE_LBM_H
#define LEE_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LEE_OK = 0,
    LEE_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, enum value or combination          */
    LEE_ERR_UNSTABLE_TAU = 2,     /* tau < 1/2: |1 - 1/tau| > 1, outside the L2 stability bound */
    LEE_ERR_OUT_OF_MEMORY = 3,    /* device allocation failed                              */
    LEE_ERR_CUDA = 4,             /* a CUDA call failed; the handle is poisoned            */
    LEE_ERR_NONFINITE = 5,        /* a NaN/Inf was found by lee_lbm_check_finite           */
    LEE_ERR_TIMEOUT = 6,          /* a bounded device wait ran out; the handle is poisoned */
    LEE_ERR_UNSUPPORTED = 7,      /* valid but not implemented combination                 */
    LEE_ERR_POISONED = 8          /* handle unusable after an earlier CUDA error           */
} lee_status;

/* Velocity sets of Sec. 8 (values fixed by the paper; see lee_velset_info). */
typedef enum {
    LEE_D1Q3 = 0,          /* Sec. 8.1:   rho0 = 1,    theta0 = 1/3                      */
    LEE_D2Q5 = 1,          /* Sec. 8.2.1: rho0 = 1,    theta0 = 1/4                      */
    LEE_D2Q5_DIATOMIC = 2, /* Sec. 8.2.2: rho0 = 20/3, theta0 = 3/10, beta = (0, 1/2)     */
    LEE_D3Q7 = 3,          /* Sec. 8.3.1: rho0 = 1,    theta0 = 1/5,  alpha = 0           */
    LEE_D3Q9 = 4,          /* Sec. 8.3.1: rho0 = 1,    theta0 = 3/5,  alpha = 3/40        */
    LEE_D3Q13 = 5,         /* Sec. 8.3.1: rho0 = 1,    theta0 = 2/5,  alpha = 0           */
    LEE_D3Q19 = 6,         /* Sec. 8.3.1: rho0 = 1,    theta0 = 3/10, alpha = 0           */
    LEE_D3Q7_DIATOMIC = 7  /* Sec. 8.3.2: f1 = 5/42 (rho0 = 1), theta0 = 5/21, beta = (0, 2/3) */
} lee_velset;

/* Edge treatment.  The paper treats periodic domains only (Sec. 2.2); the open variants are
 * additions of this library:
 *   OPEN_ZERO:    a population that would stream in from outside is the rest state, g = 0.
 *   OPEN_SPONGE:  OPEN_ZERO, plus post-collision damping g* <- (1 - sigma(d)) g* in a frame of
 *                 sponge_width cells, sigma(d) = sponge_strength (d / sponge_width)^2, d = depth
 *                 of the cell in the frame (1 .. sponge_width, maximum over axes).
 *   OPEN_LEARNED: 2D five-velocity sets only; the entering population of each edge cell is
 *                 predicted by a small MLP from the 3-cell strip along the inward normal
 *                 (lee_lbm_set_boundary_mlp).  Until a network is installed -- or after
 *                 lee_lbm_set_boundary_mlp_for_tau found none trained for this tau -- the grid
 *                 runs the plain buffer instead: OPEN_SPONGE with the configured sponge_width and
 *                 sponge_strength, or OPEN_ZERO when sponge_width is 0 (lee_lbm_boundary_in_use
 *                 tells which).
 *   SLAB:         the grid is one slab of a larger periodic domain (Sec. 2.2) cut along its last
 *                 axis (y in 2D, z in 3D; ny resp. nz = the slab's own planes): periodic along the
 *                 other axes, and along the cut the populations that enter come from the
 *                 neighbouring slabs through halo planes (lee_lbm_slab_* below).  2D and 3D sets;
 *                 F64, F32, F16 and BF16 storage. */
typedef enum {
    LEE_BC_PERIODIC = 0,
    LEE_BC_OPEN_ZERO = 1,
    LEE_BC_OPEN_SPONGE = 2,
    LEE_BC_OPEN_LEARNED = 3,
    LEE_BC_SLAB = 4
} lee_bc;

/* Storage of the populations in device memory.  Collision arithmetic is FP64 for F64 storage and
 * FP32 otherwise.  The 16-bit forms store S * g_i / f*_i rounded to nearest-even, with S a power
 * of two (config.store_scale, or chosen by init_fields when 0) -- g is already the deviation from
 * the rest state, since F = M (1 + epsilon g) (Sec. 3).
 * SPLIT16 (periodic grids only) keeps per cell the conserved moments (rho', j, E) in FP32 and the
 * post-collision non-equilibrium parts n*_i = (1 - 1/tau) (g_i - g_i^eq) in FP16 as S n*_i / f*_i:
 * 4 (D + 2) + 2 q bytes per cell and copy (58 B for D3Q19 against 76 B in FP32), with only the
 * small non-equilibrium part rounded to 16 bits.  It pays for the q-heavy sets (D3Q19, D3Q13).
 * BFP16 (block floating point; periodic, zero-incoming and sponge edges) stores g itself with
 * 16-bit integer mantissas and one exponent byte per block of 8 consecutive cells of a velocity
 * array: value = (u - 32768) 2^(e - 127), u uint16, e uint8 (0: zero block; 255: the block held a
 * NaN/Inf and decodes to NaN).  A block of FP32 values v is encoded with e = b - 14, b the biased
 * exponent of M = max|v|, plus 1 when M's 23 mantissa bits are >= 8387840 (e = 0 if below 1), and
 * u = rint(v 2^(127 - e)) + 32768 (nearest-even): an error of at most 2^-15 M (1 + 2^-14) per
 * value; decoded values encode back to themselves.  Layout [q * pitch] uint16 mantissas, then [q * pitch / 8] uint8
 * exponents (2.125 bytes per value).  Widths that are a multiple of 8 use the multi-step kernels
 * with the intermediate states in FP32, so the state is rounded once per launch (see
 * lee_lbm_step). */
typedef enum {
    LEE_STORE_F64 = 0,
    LEE_STORE_F32 = 1,
    LEE_STORE_F16 = 2,
    LEE_STORE_BF16 = 3,
    LEE_STORE_SPLIT16 = 4,
    LEE_STORE_BFP16 = 5
} lee_storage;

typedef struct {
    int32_t set;            /* lee_velset                                                   */
    int32_t storage;        /* lee_storage                                                  */
    int64_t nx, ny, nz;     /* grid extents; ny = 1 in 1D, nz = 1 in 1D/2D                  */
    double tau;             /* BGK relaxation time (Sec. 4); must be >= 1/2                 */
    int32_t bc;             /* lee_bc                                                       */
    int32_t sponge_width;   /* frame width in cells for LEE_BC_OPEN_SPONGE                  */
    double sponge_strength; /* sigma at the outermost frame cell (0 .. 1)                   */
    double store_scale;     /* 16-bit storage scale S (power of two), 0 = choose at init    */
    void *cuda_stream;      /* cudaStream_t to run on; NULL = legacy default stream         */
} lee_lbm_config;

typedef struct lee_lbm lee_lbm; /* opaque solver handle */

/* One-line description of a status code (static string, never NULL). */
const char *lee_status_string(lee_status s);

/* Describes velocity set `set` in the library's order.  Sec. 8 tables; general-equilibrium
 * coefficients of Sec. 5 (monoatomic sets: a1 = 1/rho0, a2 = -D/(2 theta0), b = 1/theta0,
 * c1 = 0, c2 = 1/theta0^2, beta = 0, gamma = (D+2)/D).
 *   D, q:   dimension and number of velocities (q <= 27)
 *   c:      [q][3] integer velocities (host memory, may be NULL)
 *   f:      [q] weights f*_i (may be NULL);  beta: [q] additional energies (may be NULL)
 *   consts: [8] = {rho0, theta0, gamma, a1, a2, b, c1, c2} (may be NULL)
 * Returns LEE_ERR_INVALID_ARGUMENT for an unknown set or NULL D/q. */
lee_status lee_velset_info(int32_t set, int32_t *D, int32_t *q, int32_t *c, double *f, double *beta, double *consts);

/* Scales between a dimensional problem and the lattice (Sec. 2.1 non-dimensionalisation, Sec. 6
 * lattice with dx = dt).  A dimensional quantity is its scale times the non-dimensional one:
 * rho0_dim = rho_star rho0, theta0_dim = theta_star theta0, u_dim = u_star u, x_dim = x_star x,
 * t_dim = t_star t, with u_star = x_star / t_star and u_star^2 = theta_star; the velocity set
 * fixes the non-dimensional rho0, theta0 (Sec. 8). */
typedef struct {
    double rho_star, theta_star, u_star, x_star, t_star;
    double eps;       /* lattice spacing = time step, (length_dim / x_star) / n_cells */
    double t_end;     /* non-dimensional end time, t_end_dim / t_star */
    int64_t steps;    /* N_TS = round(t_end / eps), halves rounded away from zero */
    double mismatch;  /* t_end - steps * eps: the end-time error of the lattice run (Sec. 9, Table 1) */
} lee_units;

/* Fills *out for velocity set `set`, a dimensional background rho0_dim, theta0_dim (> 0), a length
 * scale x_star (> 0), a periodic domain of dimensional length length_dim (> 0) resolved by n_cells
 * (>= 1) cells per direction, and a dimensional end time t_end_dim (>= 0).  Host-only, no device
 * needed.  Initial fields convert as rho' = rho'_dim / rho_star, u' = u'_dim / u_star,
 * theta' = theta'_dim / theta_star.  LEE_ERR_INVALID_ARGUMENT for an unknown set, a NULL out, a
 * non-finite or out-of-range argument, or a step count beyond 2^62. */
lee_status lee_units_from_dimensional(int32_t set, double rho0_dim, double theta0_dim, double x_star,
                                      double length_dim, int64_t n_cells, double t_end_dim, lee_units *out);

/* Creates a solver for cfg on the current CUDA device.  Validates the configuration (tau >= 1/2,
 * extents >= 1 and consistent with the dimension, storage/bc/set combination), allocates the
 * ping-pong population buffers, field staging and reduction scratch on the device, and leaves the
 * populations at the rest state g = 0.  *out is NULL on failure. */
lee_status lee_lbm_create(const lee_lbm_config *cfg, lee_lbm **out);

/* Sets the state to the equilibrium of the given fields, g_i = g_i^eq(rho', u', theta')
 * (Sec. 7 initial condition; Sec. 4/5 equilibrium).  rho[cells], u[D][cells], theta[cells] in
 * FP64.  For 16-bit and split storage with store_scale = 0 the scale S is chosen here: the
 * largest power of two with S * max_i,x |g_i^eq / f*_i| <= 1024. */
lee_status lee_lbm_init_fields(lee_lbm *h, const double *rho, const double *u, const double *theta, int32_t on_device);

/* Advances n >= 0 time steps of the LBE update scheme (Sec. 6): one fused pull-stream + BGK
 * collision kernel per step.  Asynchronous.  For n >= 8 the launches are replayed from a CUDA
 * graph (one graph holding all n steps for n <= 4096, else repeated 100-step graphs), captured on
 * first use of that length on a private stream and cached in the handle; results are identical to
 * direct launches.  Every form below also gives the same bits as single one-step launches:
 *  - periodic 2D FP32 grids with nx a multiple of 4 advance four steps per launch, the three
 *    intermediate states kept in shared memory (temporal blocking; LEE_TB_STEPS=1..4 in the
 *    environment at create time picks another count; lee_lbm_steps_per_launch reports it); a
 *    run of n steps is n / 4 such launches and n % 4 single steps;
 *  - periodic 3D FP32 grids of D3Q7 and diatomic D3Q7 with nx a multiple of 4 advance two steps
 *    per launch (a z-marching tile; LEE_TB_STEPS=1 keeps one step per launch);
 *  - BFP16 storage on those periodic 2D grids with nx a multiple of 8 uses the same kernels (four
 *    steps, or three with LEE_TB_STEPS=3), but keeps the intermediate states in FP32 and encodes
 *    only the last one: a launch of k steps equals decoding the state, k FP32 steps and one
 *    encoding, bit for bit (LEE_TB_STEPS=1 or 2 keeps one step per launch, which equals decode,
 *    one FP32 step, encode).  On 3D grids BFP16 runs one step per launch unless LEE_TB_STEPS=2
 *    asks for the two-step tile (nx a multiple of 8), which is slower there;
 *  - FP16 and BF16 storage on periodic 2D grids with nx a multiple of 4 do the same: four (or
 *    three) steps per launch with the intermediate states in FP32, one rounding to the storage per
 *    launch (LEE_TB_STEPS=1 or 2 keeps one step per launch, rounding every step);
 *  - a 1D grid (not BFP16) whose two population copies fit in shared memory (2 q nx sizeof(storage) <= 227 KB,
 *    e.g. D1Q3 FP64 up to 4843 cells) runs all n >= 2 steps in one launch: one block, or from
 *    512 cells a thread-block cluster of 8 blocks;
 *  - OPEN_LEARNED: one launch per step whose first blocks run the boundary network and write the
 *    border cells (pulled with the network's entering populations and collided) while the other
 *    blocks step the interior cells; LEE_LEARNED_STREAMS=1 in the environment at create time runs
 *    the same work as three launches instead (network and border cells on a second stream beside
 *    the interior step, joined before the next step), with the same result bit for bit. */
lee_status lee_lbm_step(lee_lbm *h, int64_t n);

/* Per-cell moments of the current state (Sec. 4 discrete moments; Sec. 5 temperature for
 * polyatomic sets): rho'[cells], u'[D][cells], theta'[cells] in FP64.  Any pointer may be NULL
 * to skip that output. */
lee_status lee_lbm_moments(lee_lbm *h, double *rho, double *u, double *theta, int32_t on_device);

/* Global FP64 sums of the current state, out[D+4]:
 *   out[0]      sum_x rho'                             (conserved on periodic grids)
 *   out[1..D]   sum_x sum_i c_i g_i  = rho0 sum_x u'    (conserved)
 *   out[D+1]    sum_x sum_i (|c_i|^2 + beta_i) g_i / 2  (energy moment of Sec. 5, conserved)
 *   out[D+2]    sum_x sum_i g_i^2 / f*_i                (weighted energy, non-increasing for
 *                                                        tau >= 1/2; cf. A0 of Sec. 8.3.1)
 *   out[D+3]    number of non-finite stored populations
 * Deterministic: fixed per-block order, then one ordered pass over the block partials. */
lee_status lee_lbm_reduce(lee_lbm *h, double *out, int32_t on_device);

/* Returns LEE_ERR_NONFINITE if any stored population is NaN or Inf, else LEE_OK (host sync). */
lee_status lee_lbm_check_finite(lee_lbm *h);

/* Copies the state g*(t) out as FP64 g[q][cells] (decoded from 16-bit storage) -- checkpoint. */
lee_status lee_lbm_get_populations(lee_lbm *h, double *g, int32_t on_device);

/* Replaces the state with g[q][cells] (FP64, encoded into the storage type) -- resume.  Used
 * with get_populations a resumed run equals the uninterrupted one bit for bit. */
lee_status lee_lbm_set_populations(lee_lbm *h, const double *g, int32_t on_device);

/* Installs the boundary network for LEE_BC_OPEN_LEARNED on a LEE_D2Q5 grid (see lee_mlp.h for
 * the network and its parameter layout).  params: nparams = 5313 FP32 values, host memory.  With
 * the network installed, every step first evaluates it on the edge strips of the current state
 * and then streams with its predictions as the entering populations. */
lee_status lee_lbm_set_boundary_mlp(lee_lbm *h, const float *params, int64_t nparams);

/* Slab decomposition of a periodic domain along its last axis (a domain larger than one GPU, or
 * one spread over several processes).  The Sec. 6 update pulls g_i(t+1, x) from x - c_i: in a slab
 * handle (LEE_BC_SLAB) the pulls of the first and last owned planes along the cut reach one plane
 * beyond the slab, into halo planes the handle keeps there.  Before each step those halo planes
 * must hold the neighbouring slabs' post-collision populations that cross the cut (velocities
 * with c_last = +1 from the slab below, c_last = -1 from the slab above): one exchange of
 * `crossing` planes per face and step (D2Q5 1, D3Q7 1, D3Q19 5).  lee_lbm_step takes n <= 1 on
 * a slab handle, since every step needs a fresh exchange.
 *
 * Halo messages are device buffers the handle owns, `bytes` each: send_lo (from the first owned
 * plane, the populations leaving downward), send_hi (from the last owned plane, leaving upward),
 * recv_lo (what enters from below: the lower neighbour's send_hi) and recv_hi (the upper
 * neighbour's send_lo); each holds one plane per crossing velocity, in the library's velocity
 * order, in the storage type.  One exchange: lee_lbm_slab_pack on every slab, then any transport
 * that moves send_lo to the lower neighbour's recv_hi and send_hi to the upper neighbour's recv_lo
 * (NCCL, MPI, a P2P copy into the receiver's own buffer, ...), then lee_lbm_slab_unpack, then
 * lee_lbm_step(h, 1).  pack and unpack are asynchronous on the handle's stream. */
lee_status lee_lbm_slab_info(lee_lbm *h, int32_t *crossing, int64_t *plane_cells, int64_t *bytes);
lee_status lee_lbm_slab_buffers(lee_lbm *h, void **send_lo, void **send_hi, void **recv_lo, void **recv_hi);
lee_status lee_lbm_slab_pack(lee_lbm *h);
lee_status lee_lbm_slab_unpack(lee_lbm *h);

/* n steps of `count` slabs of one periodic domain held in this process on one device and one
 * stream, listed in order along the cut (slab k + 1 above slab k; the last one lies below the
 * first).  Each step: pack every slab, copy every message into its receiver's recv buffer
 * (cudaMemcpyAsync, device to device, on the shared stream), unpack, one step of every slab.  The
 * slabs must share set, storage, tau, the extents across the cut, device and stream, else
 * LEE_ERR_INVALID_ARGUMENT.  Bit for bit the single-domain result of the same storage. */
lee_status lee_lbm_slab_step(lee_lbm *const *slabs, int32_t count, int64_t n);

/* A boundary network trained at relaxation time trained_tau: installed (as lee_lbm_set_boundary_mlp)
 * only if |tau - trained_tau| <= tau_tolerance; otherwise the handle runs (or returns to) the
 * fallback edge of LEE_BC_OPEN_LEARNED.  *installed (may be NULL) receives 1 or 0.
 * LEE_ERR_INVALID_ARGUMENT for a non-learned handle, a non-finite trained_tau or a negative or
 * non-finite tolerance. */
lee_status lee_lbm_set_boundary_mlp_for_tau(lee_lbm *h, const float *params, int64_t nparams, double trained_tau,
                                            double tau_tolerance, int32_t *installed);

/* The edge treatment the next step runs (lee_bc): the configured one, except that OPEN_LEARNED
 * reports its fallback (OPEN_SPONGE or OPEN_ZERO) while no network is installed. */
lee_status lee_lbm_boundary_in_use(lee_lbm *h, int32_t *bc);

/* Number of time steps taken since the last init/set_populations. */
lee_status lee_lbm_steps_done(lee_lbm *h, int64_t *steps);

/* How lee_lbm_step runs this grid: *steps = 1 (one fused stream-collide launch per time step),
 * 2..4 (periodic 2D FP32 grids with nx a multiple of 4: that many time steps per launch, the
 * intermediate states kept in shared memory -- temporal blocking; 4 unless LEE_TB_STEPS was set
 * at create time; periodic 3D FP32 D3Q7 and diatomic D3Q7 grids with nx a multiple of 4: 2;
 * BFP16 storage: 3 or 4 in 2D on such grids with nx a multiple of 8, 2 in 3D only with
 * LEE_TB_STEPS=2; FP16 / BF16 storage: 3 or 4 in 2D on such grids) or 0 (small 1D
 * grid: all steps of a call in one on-chip launch).  All forms give bit-identical results, except
 * that BFP16, FP16 and BF16 storage round their state once per launch (see lee_lbm_step). */
lee_status lee_lbm_steps_per_launch(lee_lbm *h, int32_t *steps);

/* The 16-bit storage scale S in use (1 for F64/F32/BFP16 storage). */
lee_status lee_lbm_store_scale(lee_lbm *h, double *scale);

/* Blocks until all work on the handle's stream has finished. */
lee_status lee_lbm_sync(lee_lbm *h);

/* Last error message of the handle (empty string if none; never NULL for a non-NULL handle). */
const char *lee_lbm_last_error(lee_lbm *h);

/* Frees the handle and its device memory.  NULL-safe.  Synchronises the stream first. */
lee_status lee_lbm_destroy(lee_lbm *h);

/* Measures the current device's FP64 fused multiply-add rate (the paper has no counterpart): 8
 * blocks of 256 threads per SM each run 8 independent chains of `iters` FP64 fma; *flops_per_s =
 * 2 x fma count / elapsed time (CUDA events, after a warm-up launch).  The solver's FP64 storage
 * forms are bounded by this rate rather than by HBM.  Synchronous; allocates 2 KB of scratch.
 * LEE_ERR_INVALID_ARGUMENT for iters outside 1 .. 2^30 or a NULL output. */
lee_status lee_probe_fp64_fma(int64_t iters, double *flops_per_s);

/* Test hook for the failure path (the paper has no counterpart).  after >= 0 arms it: of the CUDA
 * calls that solver, batch and network handles check from now on, the (after+1)-th that succeeds
 * is reported as failed (cudaErrorUnknown), once; the handle that made it returns LEE_ERR_CUDA and
 * is poisoned exactly as after a real CUDA error.  after = -1 disarms it.  No GPU error is raised
 * (the call itself ran normally), so tests can exercise poisoning from the host.  Process-wide;
 * LEE_ERR_INVALID_ARGUMENT for after < -1. */
lee_status lee_test_inject_cuda_error(int32_t after);

/* Test hook for the bounded waits of the TMA-fed 3D two-step tile (the paper has no counterpart).
 * on = 1: every launch of that kernel from now on announces 16 bytes more than its first stage of
 * inputs receives, so that the wait for that stage runs out after wait_ns nanoseconds (0: the
 * default limit of one second); the kernel then records the timeout in its handle, lets its copies
 * in flight land and returns without touching the state.  The handle's next call (or the
 * synchronisation of the current one) returns LEE_ERR_TIMEOUT and poisons it.  The GPU itself
 * never faults or hangs.  on = 0 restores normal launches.  Graphs captured while it was on keep
 * it.  Process-wide; LEE_ERR_INVALID_ARGUMENT for on outside {0, 1} or wait_ns outside 0 .. 10^10. */
lee_status lee_test_inject_stage_timeout(int32_t on, int64_t wait_ns);

/* The global sums of lee_lbm_reduce (same out[D+4] layout and order, same result bit for bit)
 * for a population field the caller owns, computed WITHOUT ALLOCATING anything.  The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc (or any routine
 * that allocates) where they need these diagnostics -- code running under someone else's memory
 * budget or allocator, a process that reserves all its device memory up front, or a callback
 * that must not allocate -- and therefore cannot create a solver handle, whose creation
 * allocates the reduction scratch.
 *   set: as in lee_lbm_config; storage: LEE_STORE_F64, F32, F16 or BF16 (SPLIT16 and the other
 *   multi-array forms are rejected with LEE_ERR_INVALID_ARGUMENT); g: DEVICE pointer to the stored populations,
 *   g[i * pitch + cell] for i < q, in the storage type (16-bit storage holds S * g_i / f*_i);
 *   cells: 1 .. 2^31 - 1; pitch >= cells (elements between velocity arrays);
 *   store_scale: S for 16-bit storage (> 0), ignored otherwise;
 *   out: DEVICE pointer to D + 4 doubles; cuda_stream: stream to run on (NULL = default).
 * Scratch: a fixed file-scope device array of 2432 x 16 FP64 block partials (311,296 bytes) that
 * every GPU loading the library keeps until the process exits.  Sizes beyond it (more than
 * 2^31 - 1 cells) are rejected with LEE_ERR_INVALID_ARGUMENT; so are bad pointers or enums.
 * Set-up: the first call on a device (with that device current) looks up the array's device
 * address once and keeps it; make that first call before any stream capture.  The kept address
 * belongs to the device's primary context: after cudaDeviceReset on that device it is stale, and
 * this entry point must not be called again in that process.  All calls share the one array
 * and each call overwrites the entries it reads, so nothing needs clearing between calls -- but
 * calls that overlap on the GPU (e.g. on two streams at once) race on it.  Asynchronous: returns
 * after enqueueing; a CUDA failure returns LEE_ERR_CUDA (there is no handle to poison). */
lee_status lee_reduce_noalloc(int32_t set, int32_t storage, const void *g, int64_t cells, int64_t pitch,
                              double store_scale, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LEE_LBM_H */

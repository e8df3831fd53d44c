// lee_lbm.cu -- C ABI of the solver (include/lee_lbm.h): handle, memory, validation, dispatch.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lee_lbm.h"
#include "handles.cuh"
#include "split.cuh"

// fold_coefficients evaluates host-side constants in long double; the device pass of nvcc notes
// that long double would be double there, which does not apply to this host-only code.
#pragma nv_diag_suppress 20208

namespace lee {
cudaError_t launch_mlp_boundary(const void *packed, int storage, const void *g, long long pitch, int NX, int NY, void *ghost,
                                int L, cudaStream_t st);
cudaError_t launch_learned_step(const void *packed, int set, const StepLaunch &L, unsigned long long *corner);
cudaError_t mlp_pack(const float *params_dev, void *packed, cudaStream_t st);
extern const SetOps kOpsD1Q3, kOpsD2Q5, kOpsD2Q5Di, kOpsD3Q7, kOpsD3Q7Di, kOpsD3Q9, kOpsD3Q13, kOpsD3Q19;

const SetOps *set_ops(int set) {
    switch (set) {
    case LEE_D1Q3: return &kOpsD1Q3;
    case LEE_D2Q5: return &kOpsD2Q5;
    case LEE_D2Q5_DIATOMIC: return &kOpsD2Q5Di;
    case LEE_D3Q7: return &kOpsD3Q7;
    case LEE_D3Q9: return &kOpsD3Q9;
    case LEE_D3Q13: return &kOpsD3Q13;
    case LEE_D3Q19: return &kOpsD3Q19;
    case LEE_D3Q7_DIATOMIC: return &kOpsD3Q7Di;
    default: return nullptr;
    }
}

__global__ void k_reduce_final(const double *__restrict__ partial, int nblocks, ReduceCombine c, double *__restrict__ out) {
    __shared__ double raw[kReduceMax];
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (v < c.nraw) {
        double a = 0.0;
        for (int b = lane; b < nblocks; b += 32) a += partial[(long long)b * kReduceMax + v];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(kFull, a, off);
        if (lane == 0) raw[v] = a;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int ns = c.ns, D = c.D;
    double r = 0.0, e = 0.0, w = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < ns; ++k) {
        const double p = raw[k] * c.dec[k];
        r += p;
        e += c.ew[k] * p;
        w += raw[ns + k] * (c.dec[k] * c.dec[k]) / c.f[k];
        for (int a = 0; a < D; ++a) j[a] += raw[2 * ns + k * D + a] * c.dec[k];
    }
    out[0] = r;
    for (int a = 0; a < D; ++a) out[1 + a] = j[a];
    out[D + 1] = e;
    out[D + 2] = w;
    out[D + 3] = raw[c.nraw - 1];
}

SetConsts consts_for(int set, double scale) {
    SetConsts k{};
    dispatch_set(set, [&](auto s) {
        using S = decltype(s);
        k = host_consts<S>(scale);
    });
    return k;
}

// Folded collision coefficients (see CollideCoef in kernels.cuh):
//   rho' = sum_s w1_s P_s,  e = sum_s w2_s P_s,  theta' = kE e - kR rho',  j = sum_s w1_s J_s,
//   g*_i = (1 - w) g_i + w f'_t (alpha_t rho' + beta_t theta') + w f'_t (b / rho0) c_i . j
// with w1_s = f*_s for the scaled 16-bit storage (stored value S g / f*) and 1 otherwise,
// w2_s = w1_s (s + beta_s) / 2, f'_t = 1 (scaled) or f*_t, alpha_t = a1 + t c1 / 2,
// beta_t = a2 + t c2 / 2, kE = (gamma - 1) / rho0, kR = theta0 / rho0 (Secs. 4-6).
// `omega` must already be rounded to the arithmetic type (omega_for), so that every coefficient
// scales the same w that 1 - w is formed from.  The shell factors are evaluated in long double
// and snapped to a power of two when they are one to within rounding (the momentum factors
// f*_t b / rho0 are powers of two for every set of Sec. 8).
void fold_coefficients(int set, bool scaled, double omega, double M[4][4], double N[4][4]) {
    const SetConsts k = consts_for(set, 1.0);
    for (int t = 0; t < 4; ++t)
        for (int s = 0; s < 4; ++s) M[t][s] = N[t][s] = 0.0;
    typedef long double LD;
    const LD kE = ((LD)k.gamma - 1.0L) / (LD)k.rho0, kR = (LD)k.theta0 / (LD)k.rho0;
    auto snap = [](LD x) -> LD {
        if (x == 0.0L) return x;
        int e = 0;
        const LD m = std::frexp(std::fabs(x), &e);
        if (std::fabs(m - 0.5L) < 1e-15L) return std::copysign(std::ldexp(0.5L, e), x);
        return x;
    };
    for (int t = 0; t < 4; ++t) {
        const LD ft = scaled ? 1.0L : (LD)k.f[t];
        const LD alpha = (LD)k.a1 + 0.5L * t * (LD)k.c1, beta = (LD)k.a2 + 0.5L * t * (LD)k.c2;
        for (int s = 0; s < 4; ++s) {
            const LD w1 = scaled ? (LD)k.f[s] : 1.0L;
            const LD w2 = 0.5L * ((LD)s + (LD)k.beta[s]) * w1;
            const LD mhat = snap(ft * (alpha * w1 + beta * (kE * w2 - kR * w1)));
            const LD nhat = snap(ft * ((LD)k.b / (LD)k.rho0) * w1);
            M[t][s] = (double)((LD)omega * mhat);
            N[t][s] = (double)((LD)omega * nhat);
        }
    }
}

// Host-side failure injection for tests (lee_test_inject_cuda_error): number of successful
// checked calls still to pass before one is reported as failed; negative = disarmed.
std::atomic<int> g_inject_countdown{-1};
// lee_test_inject_stage_timeout: launches of the TMA-fed 3D tile announce more bytes than their
// first stage receives (so that its bounded wait runs out), with this wait limit in ns (0: default)
std::atomic<int> g_inject_stage{0};
std::atomic<long long> g_stage_wait_ns{0};

cudaError_t checked(cudaError_t e) {
    if (e != cudaSuccess) return e;
    int n = g_inject_countdown.load(std::memory_order_relaxed);
    while (n >= 0) {
        if (g_inject_countdown.compare_exchange_weak(n, n - 1, std::memory_order_relaxed))
            return n == 0 ? cudaErrorUnknown : cudaSuccess;
    }
    return cudaSuccess;
}

}  // namespace lee

using namespace lee;


namespace {

constexpr long long kGraphMinSteps = 8, kMaxGraphSteps = 4096, kChunkGraphSteps = 100;

lee_status fail(lee_lbm *h, lee_status s, const std::string &msg) {
    if (h) {
        h->err = msg;
        if (s == LEE_ERR_CUDA || s == LEE_ERR_TIMEOUT) h->poisoned = true;
    }
    return s;
}

// Time steps fused per launch (temporal blocking): tb_steps on periodic 2D FP32 grids whose width
// is a multiple of 4; two on periodic 3D FP32 grids of the axis-velocity sets whose width is a
// multiple of 4; one step otherwise (in 3D, FP16/BF16 storage moves half the bytes and stays on the
// one-step kernel, which measured faster there).
//
// BFP16 storage (widths a multiple of its 8-cell block) and FP16/BF16 storage on periodic 2D grids
// take the same K-step kernel, with the intermediate states in FP32 rather than rounded to the
// storage: a launch of k steps rounds once, so its results depend on k (deterministically) and stay
// within the storage error of single steps.  It has no two-step 2D kernel: LEE_TB_STEPS=2 keeps it on one step per launch.  In 3D its
// two-step tile is taken only when LEE_TB_STEPS=2 asks for it: the decoding and encoding make that
// latency-bound tile slower than the one-step kernel (D3Q7 384^3: 124 against 196 GLUPS).
//
// The two-step tile comes in two kernels: fed by per-thread loads (tb3d.cuh; any nx % 4 == 0), the
// default, or by TMA boxes (tb3d_tma.cuh; grids with nx % 128 == 0, ny a multiple of its 8-row
// tiles and at least 16, pitch % 128 == 0), taken when LEE_T3_TMA=1 asks for it.  The TMA-fed
// kernel measured slower on D3Q7 384^3 (FP32 166 against 217 GLUPS, BFP16 105 against 125 for the
// register-fed tile and 197 for the one-step kernel): with one block of ten computing warps per SM
// and one barrier per plane it is latency bound, although its stages arrive in time.
bool tma_tile(const lee_lbm *h) {
    if (!h->ops->step3d2 || h->cfg.bc != LEE_BC_PERIODIC || h->D != 3 || h->tb_steps < 2) return false;
    if (h->cfg.storage != LEE_STORE_BFP16 && h->cfg.storage != LEE_STORE_F32) return false;
    if (!t3t_eligible((int)h->cfg.nx, (int)h->cfg.ny, h->pitch)) return false;
    return h->t3_tma == 1;
}
bool tiled_3d(const lee_lbm *h) {
    if (!h->ops->step3d2 || h->cfg.bc != LEE_BC_PERIODIC) return false;
    if (tma_tile(h)) return true;
    if (h->cfg.storage == LEE_STORE_BFP16) return h->tb_env && h->tb_steps == 2 && h->cfg.nx % 8 == 0;
    return h->cfg.storage == LEE_STORE_F32 && h->cfg.nx % 4 == 0;
}
int fused_steps(const lee_lbm *h) {
    if (h->tb_steps <= 1) return 1;
    if (tiled_3d(h)) return 2;
    if (h->cfg.storage == LEE_STORE_BFP16) {
        const bool tiled = h->ops->stepk && h->cfg.bc == LEE_BC_PERIODIC && h->cfg.nx % 8 == 0 && h->cfg.ny >= 3;
        return tiled && h->tb_steps >= 3 ? h->tb_steps : 1;
    }
    if (h->cfg.storage == LEE_STORE_F16 || h->cfg.storage == LEE_STORE_BF16) {
        const bool tiled = h->ops->stepk && h->cfg.bc == LEE_BC_PERIODIC && h->cfg.nx % 4 == 0 && h->cfg.ny >= 3;
        return tiled && h->tb_steps >= 3 ? h->tb_steps : 1;
    }
    const bool tiled = h->ops->step2 && h->cfg.bc == LEE_BC_PERIODIC && h->cfg.storage == LEE_STORE_F32 &&
                       h->cfg.nx % 4 == 0 && h->cfg.ny >= 3;
    if (!tiled) return 1;
    return h->tb_steps >= 3 && h->ops->stepk ? h->tb_steps : 2;
}

// Whether the 1D on-chip path (all steps of a call in one launch) takes this grid.
bool onchip(const lee_lbm *h) {
    return h->ops->onchip_1d && h->cfg.storage != LEE_STORE_SPLIT16 && h->cfg.storage != LEE_STORE_BFP16 &&
           2 * h->elem * (size_t)h->Q * (size_t)h->cfg.nx <= (size_t)kMaxOnchipSmem;
}

lee_status cuda_fail(lee_lbm *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(h, LEE_ERR_OUT_OF_MEMORY, m);
    return fail(h, LEE_ERR_CUDA, m);
}

#define LEE_CK(h, call, what)                                 \
    do {                                                      \
        cudaError_t e_ = lee::checked(call);                  \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, what); \
    } while (0)

// Whether a kernel of this handle recorded a timed-out bounded wait (read without synchronising:
// the word is set by kernels that already finished, or will be seen after the next sync).
bool wait_timed_out(const lee_lbm *h) {
    return h->wait_host && *reinterpret_cast<volatile unsigned *>(h->wait_host) != 0u;
}
constexpr const char *kWaitMsg = "3D two-step tile: a bounded wait for a TMA stage ran out";

// Synchronises the handle's stream, then reports a timed-out wait recorded by its kernels.
#define LEE_SYNC(h)                                                                   \
    do {                                                                              \
        LEE_CK((h), cudaStreamSynchronize((h)->st), "sync");                          \
        if (wait_timed_out(h)) return fail((h), LEE_ERR_TIMEOUT, kWaitMsg);           \
    } while (0)

lee_status enter(lee_lbm *h) {
    if (!h) return LEE_ERR_INVALID_ARGUMENT;
    if (h->poisoned) return LEE_ERR_POISONED;
    if (wait_timed_out(h)) return fail(h, LEE_ERR_TIMEOUT, kWaitMsg);
    cudaError_t e = lee::checked(cudaSetDevice(h->device));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    return LEE_OK;
}

size_t elem_size(int storage) {
    switch (storage) {
    case LEE_STORE_F64: return 8;
    case LEE_STORE_F32: return 4;
    case LEE_STORE_F16:
    case LEE_STORE_BF16: return 2;
    case LEE_STORE_SPLIT16: return 2;  // the non-equilibrium arrays; the moments come on top
    case LEE_STORE_BFP16: return 2;    // the mantissas; one exponent byte per 8 values on top
    default: return 0;
    }
}

// Bytes of one state copy.
size_t state_bytes(int storage, int D, int Q, long long pitch) {
    if (storage == LEE_STORE_SPLIT16) return (size_t)split_bytes_per_cell(D, Q) * (size_t)pitch;
    if (storage == LEE_STORE_BFP16) return (size_t)Q * (size_t)pitch * 2 + (size_t)Q * (size_t)pitch / 8;
    return elem_size(storage) * (size_t)Q * (size_t)pitch;
}

// 16-bit forms whose storage scale S is chosen from the initial fields.
bool scaled_storage(int storage) {
    return storage == LEE_STORE_F16 || storage == LEE_STORE_BF16 || storage == LEE_STORE_SPLIT16;
}

void free_all(lee_lbm *h) {
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->fields);
    cudaFree(h->pops64);
    cudaFree(h->partial);
    cudaFree(h->red_out);
    cudaFree(h->maxbits);
    cudaFree(h->ghost);
    cudaFree(h->corner);
    cudaFree(h->mlp);
    for (void *p : h->halo) cudaFree(p);
    if (h->wait_host) cudaFreeHost(h->wait_host);
    h->wait_host = h->wait_dev = nullptr;
}

// A learned edge without a network runs its fallback: the sponge frame of the configuration
// (zero-incoming edges if its width is 0).
bool learned_active(const lee_lbm *h) { return h->cfg.bc == LEE_BC_OPEN_LEARNED && h->mlp_ready; }
bool sponge_active(const lee_lbm *h) {
    return h->cfg.bc == LEE_BC_OPEN_SPONGE || (h->cfg.bc == LEE_BC_OPEN_LEARNED && !h->mlp_ready && h->cfg.sponge_width > 0);
}

// Drops the captured step graphs (the launches they hold no longer match the edge treatment).
void drop_step_graphs(lee_lbm *h) {
    for (auto &kv : h->exec) cudaGraphExecDestroy(kv.second);
    h->exec.clear();
}

// The first owned cell of state copy `which` (one plane in for a slab, whose halo plane comes
// first in every velocity array).
void *state(lee_lbm *h, int which) {
    return static_cast<char *>(h->buf[which]) + (h->slab ? h->elem * (size_t)h->plane : 0);
}

// Device address of a host buffer that kernels can use in place: page-locked host memory mapped
// into the device address space (cudaHostAlloc, or cudaHostRegister with mapping), which a GB300
// reaches over NVLink-C2C.  nullptr for pageable memory, whose bytes go through a staging copy.
template <class T>
T *mapped_host(T *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<T *>(a.devicePointer);
}

lee_status ensure_fields(lee_lbm *h) {
    if (h->fields) return LEE_OK;
    LEE_CK(h, cudaMalloc(&h->fields, sizeof(double) * (size_t)(h->D + 2) * (size_t)h->cells), "cudaMalloc(fields)");
    return LEE_OK;
}

lee_status ensure_pops64(lee_lbm *h) {
    if (h->pops64) return LEE_OK;
    LEE_CK(h, cudaMalloc(&h->pops64, sizeof(double) * (size_t)h->Q * (size_t)h->cells), "cudaMalloc(pops64)");
    return LEE_OK;
}

}  // namespace

extern "C" {

const char *lee_status_string(lee_status s) {
    switch (s) {
    case LEE_OK: return "ok";
    case LEE_ERR_INVALID_ARGUMENT: return "invalid argument";
    case LEE_ERR_UNSTABLE_TAU: return "tau < 1/2 is outside the L2 stability bound";
    case LEE_ERR_OUT_OF_MEMORY: return "device out of memory";
    case LEE_ERR_CUDA: return "CUDA error (handle poisoned)";
    case LEE_ERR_NONFINITE: return "non-finite population found";
    case LEE_ERR_TIMEOUT: return "bounded device wait timed out (handle poisoned)";
    case LEE_ERR_UNSUPPORTED: return "unsupported combination";
    case LEE_ERR_POISONED: return "handle poisoned by an earlier CUDA error";
    default: return "unknown status";
    }
}

lee_status lee_test_inject_cuda_error(int32_t after) {
    if (after < -1) return LEE_ERR_INVALID_ARGUMENT;
    g_inject_countdown.store(after, std::memory_order_relaxed);
    return LEE_OK;
}

lee_status lee_test_inject_stage_timeout(int32_t on, int64_t wait_ns) {
    if ((on != 0 && on != 1) || wait_ns < 0 || wait_ns > 10000000000LL) return LEE_ERR_INVALID_ARGUMENT;
    g_inject_stage.store(on, std::memory_order_relaxed);
    g_stage_wait_ns.store(wait_ns, std::memory_order_relaxed);
    return LEE_OK;
}

lee_status lee_velset_info(int32_t set, int32_t *D, int32_t *q, int32_t *c, double *f, double *beta, double *consts) {
    const SetOps *o = set_ops(set);
    if (!o || !D || !q) return LEE_ERR_INVALID_ARGUMENT;
    *D = o->D;
    *q = o->Q;
    const SetConsts k = consts_for(set, 1.0);
    for (int i = 0; i < o->Q; ++i) {
        if (c)
            for (int a = 0; a < 3; ++a) c[3 * i + a] = o->c[i][a];
        if (f) f[i] = k.f[o->shell[i]];
        if (beta) beta[i] = k.beta[o->shell[i]];
    }
    if (consts) {
        const double v[8] = {k.rho0, k.theta0, k.gamma, k.a1, k.a2, k.b, k.c1, k.c2};
        for (int j = 0; j < 8; ++j) consts[j] = v[j];
    }
    return LEE_OK;
}

lee_status lee_units_from_dimensional(int32_t set, double rho0_dim, double theta0_dim, double x_star,
                                      double length_dim, int64_t n_cells, double t_end_dim, lee_units *out) {
    if (!out || !set_ops(set)) return LEE_ERR_INVALID_ARGUMENT;
    const double pos[4] = {rho0_dim, theta0_dim, x_star, length_dim};
    for (double v : pos)
        if (!std::isfinite(v) || !(v > 0.0)) return LEE_ERR_INVALID_ARGUMENT;
    if (n_cells < 1 || !std::isfinite(t_end_dim) || !(t_end_dim >= 0.0)) return LEE_ERR_INVALID_ARGUMENT;
    const SetConsts k = consts_for(set, 1.0);
    lee_units u;
    u.rho_star = rho0_dim / k.rho0;
    u.theta_star = theta0_dim / k.theta0;
    u.u_star = std::sqrt(u.theta_star);
    u.x_star = x_star;
    u.t_star = x_star / u.u_star;
    u.eps = (length_dim / x_star) / (double)n_cells;
    u.t_end = t_end_dim / u.t_star;
    const double r = std::round(u.t_end / u.eps);
    if (!std::isfinite(r) || r > 4.6e18) return LEE_ERR_INVALID_ARGUMENT;
    u.steps = (int64_t)r;
    u.mismatch = u.t_end - (double)u.steps * u.eps;
    *out = u;
    return LEE_OK;
}

lee_status lee_lbm_create(const lee_lbm_config *cfg, lee_lbm **out) {
    if (!out) return LEE_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (!cfg) return LEE_ERR_INVALID_ARGUMENT;
    const SetOps *o = set_ops(cfg->set);
    if (!o) return LEE_ERR_INVALID_ARGUMENT;
    if (elem_size(cfg->storage) == 0) return LEE_ERR_INVALID_ARGUMENT;
    if (!(cfg->tau == cfg->tau) || !std::isfinite(cfg->tau)) return LEE_ERR_INVALID_ARGUMENT;
    if (cfg->tau < 0.5) return LEE_ERR_UNSTABLE_TAU;
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return LEE_ERR_INVALID_ARGUMENT;
    if (o->D < 3 && cfg->nz != 1) return LEE_ERR_INVALID_ARGUMENT;
    if (o->D < 2 && cfg->ny != 1) return LEE_ERR_INVALID_ARGUMENT;
    if (cfg->nx > (1LL << 30) || cfg->ny > (1LL << 30) || cfg->nz > (1LL << 30)) return LEE_ERR_INVALID_ARGUMENT;
    const long long cells = cfg->nx * cfg->ny * cfg->nz;
    if (cells >= (1LL << 31)) return LEE_ERR_INVALID_ARGUMENT;
    if (cfg->bc < LEE_BC_PERIODIC || cfg->bc > LEE_BC_SLAB) return LEE_ERR_INVALID_ARGUMENT;
    if (cfg->bc == LEE_BC_SLAB) {
        if (o->D < 2) return LEE_ERR_UNSUPPORTED;
        if (cfg->storage == LEE_STORE_SPLIT16 || cfg->storage == LEE_STORE_BFP16) return LEE_ERR_UNSUPPORTED;
    }
    // a learned edge may name a sponge frame too: its fallback while no network is installed
    const bool frame = cfg->bc == LEE_BC_OPEN_SPONGE || (cfg->bc == LEE_BC_OPEN_LEARNED && cfg->sponge_width != 0);
    if (frame) {
        if (cfg->sponge_width < 1 || !(cfg->sponge_strength >= 0.0 && cfg->sponge_strength <= 1.0))
            return LEE_ERR_INVALID_ARGUMENT;
        for (int a = 0; a < o->D; ++a) {
            const long long n = a == 0 ? cfg->nx : (a == 1 ? cfg->ny : cfg->nz);
            if (2LL * cfg->sponge_width >= n) return LEE_ERR_INVALID_ARGUMENT;
        }
    }
    if (cfg->bc == LEE_BC_OPEN_LEARNED && !(o->D == 2 && o->Q == 5)) return LEE_ERR_UNSUPPORTED;
    if (cfg->bc == LEE_BC_OPEN_LEARNED && (cfg->nx < 3 || cfg->ny < 3)) return LEE_ERR_INVALID_ARGUMENT;
    if (cfg->storage == LEE_STORE_SPLIT16 && cfg->bc != LEE_BC_PERIODIC) return LEE_ERR_UNSUPPORTED;
    if (cfg->storage == LEE_STORE_BFP16 && cfg->bc == LEE_BC_OPEN_LEARNED) return LEE_ERR_UNSUPPORTED;
    if (cfg->store_scale < 0.0 || !std::isfinite(cfg->store_scale)) return LEE_ERR_INVALID_ARGUMENT;
    if (cfg->store_scale > 0.0) {
        int ex = 0;
        if (std::frexp(cfg->store_scale, &ex) != 0.5) return LEE_ERR_INVALID_ARGUMENT;  // power of two
    }

    lee_lbm *h = new (std::nothrow) lee_lbm();
    if (!h) return LEE_ERR_OUT_OF_MEMORY;
    h->cfg = *cfg;
    h->ops = o;
    h->D = o->D;
    h->Q = o->Q;
    h->cells = cells;
    h->pitch = (cells + 63) / 64 * 64;
    h->elem = elem_size(cfg->storage);
    if (cfg->bc == LEE_BC_SLAB) {  // the owned planes and a halo plane on each side
        h->slab = true;
        h->plane = o->D == 3 ? cfg->nx * cfg->ny : cfg->nx;
        h->nl = (int)(o->D == 3 ? cfg->nz : cfg->ny);
        h->crossing = o->slab_crossing;
        h->pitch = ((long long)(h->nl + 2) * h->plane + 63) / 64 * 64;
    }
    h->st = static_cast<cudaStream_t>(cfg->cuda_stream);
    if (const char *ev = std::getenv("LEE_TB_STEPS")) {
        if (ev[0] >= '1' && ev[0] <= '4' && ev[1] == 0) {
            h->tb_steps = ev[0] - '0';
            h->tb_env = true;
        }
    }
    if (const char *ev = std::getenv("LEE_SINGLE_STEP")) {
        if (ev[0] == '1') h->tb_steps = 1;
    }
    if (const char *ev = std::getenv("LEE_FORCE_SCALAR")) h->force_scalar = ev[0] == '1';
    if (const char *ev = std::getenv("LEE_BFP_CELLS")) {
        if ((ev[0] == '4' || ev[0] == '8') && ev[1] == 0) h->bfp_cells = ev[0] - '0';
    }
    if (const char *ev = std::getenv("LEE_T3_TMA")) {
        if ((ev[0] == '0' || ev[0] == '1') && ev[1] == 0) h->t3_tma = ev[0] - '0';
    }
    if (const char *ev = std::getenv("LEE_LEARNED_STREAMS")) h->learned_streams = ev[0] == '1';
    if (h->force_scalar) h->tb_steps = 1;
    h->scale = scaled_storage(cfg->storage) ? (cfg->store_scale > 0.0 ? cfg->store_scale : 1.0) : 1.0;
    cudaError_t e = cudaGetDevice(&h->device);
    const size_t bytes = state_bytes(cfg->storage, h->D, h->Q, h->pitch);
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[1], bytes);
    h->nblocks = aux_blocks(cells, kReduceThreads);
    if (e == cudaSuccess) e = cudaMalloc(&h->partial, sizeof(double) * kReduceMax * (size_t)h->nblocks);
    if (e == cudaSuccess) e = cudaMalloc(&h->red_out, sizeof(double) * kReduceMax);
    if (e == cudaSuccess) e = cudaMalloc(&h->maxbits, sizeof(unsigned int));
    for (int k = 0; k < 4 && h->slab && e == cudaSuccess; ++k)
        e = cudaMalloc(&h->halo[k], h->elem * (size_t)h->crossing * (size_t)h->plane);
    if (e == cudaSuccess && cfg->bc == LEE_BC_OPEN_LEARNED) {
        h->ghost_L = (int)(cfg->nx > cfg->ny ? cfg->nx : cfg->ny);
        e = cudaMalloc(&h->ghost, (cfg->storage == LEE_STORE_F64 ? 8 : 4) * 4 * (size_t)h->ghost_L);
        if (e == cudaSuccess) e = cudaMalloc(&h->corner, 4 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemsetAsync(h->corner, 0, 4 * sizeof(unsigned long long), h->st);
    }
    if (e == cudaSuccess && o->step2_prepare && cfg->bc == LEE_BC_PERIODIC && cfg->storage == LEE_STORE_F32)
        e = o->step2_prepare();
    if (e == cudaSuccess && o->stepk_prepare && h->tb_steps >= 3 && cfg->bc == LEE_BC_PERIODIC &&
        (cfg->storage == LEE_STORE_F32 || cfg->storage == LEE_STORE_BFP16 || cfg->storage == LEE_STORE_F16 ||
         cfg->storage == LEE_STORE_BF16))
        e = o->stepk_prepare(h->tb_steps, cfg->storage);
    if (e == cudaSuccess && h->tb_steps >= 2 && tiled_3d(h)) e = o->step3d2_prepare(cfg->storage, tma_tile(h) ? 1 : 0);
    if (e == cudaSuccess && tma_tile(h)) {
        e = cudaHostAlloc(reinterpret_cast<void **>(&h->wait_host), sizeof(unsigned), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            *h->wait_host = 0u;
            e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->wait_dev), h->wait_host, 0);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[0], 0, bytes, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, bytes, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        lee_status s = e == cudaErrorMemoryAllocation ? LEE_ERR_OUT_OF_MEMORY : LEE_ERR_CUDA;
        free_all(h);
        delete h;
        cudaGetLastError();
        return s;
    }
    *out = h;
    return LEE_OK;
}

lee_status lee_lbm_init_fields(lee_lbm *h, const double *rho, const double *u, const double *theta, int32_t on_device) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (!rho || !theta || (h->D > 0 && !u)) return fail(h, LEE_ERR_INVALID_ARGUMENT, "init_fields: NULL field");
    const double *dr = rho, *du = u, *dt = theta;
    const double *mr = on_device ? nullptr : mapped_host(rho), *mu = on_device ? nullptr : mapped_host(u),
                 *mt = on_device ? nullptr : mapped_host(theta);
    const bool in_place = mr && mt && (h->D == 0 || mu);
    if (in_place) {  // the kernels read the mapped host fields directly
        dr = mr;
        du = mu;
        dt = mt;
    } else if (!on_device) {
        if ((s = ensure_fields(h)) != LEE_OK) return s;
        const size_t n = sizeof(double) * (size_t)h->cells;
        double *fr = h->fields, *fu = h->fields + h->cells, *ft = h->fields + (size_t)(h->D + 1) * h->cells;
        LEE_CK(h, cudaMemcpyAsync(fr, rho, n, cudaMemcpyHostToDevice, h->st), "H2D rho");
        LEE_CK(h, cudaMemcpyAsync(fu, u, n * h->D, cudaMemcpyHostToDevice, h->st), "H2D u");
        LEE_CK(h, cudaMemcpyAsync(ft, theta, n, cudaMemcpyHostToDevice, h->st), "H2D theta");
        dr = fr;
        du = fu;
        dt = ft;
    }
    if (scaled_storage(h->cfg.storage) && h->cfg.store_scale == 0.0) {
        LEE_CK(h, cudaMemsetAsync(h->maxbits, 0, sizeof(unsigned int), h->st), "memset maxbits");
        LEE_CK(h, h->ops->init_maxabs(dr, du, dt, h->cells, consts_for(h->cfg.set, 1.0), h->maxbits, h->st), "init_maxabs");
        unsigned int bits = 0;
        LEE_CK(h, cudaMemcpyAsync(&bits, h->maxbits, sizeof(bits), cudaMemcpyDeviceToHost, h->st), "D2H maxbits");
        LEE_SYNC(h);
        float m;
        std::memcpy(&m, &bits, sizeof(m));
        double S = 1.0;
        if (m > 0.0f && std::isfinite(m)) {
            // largest power of two with S * m <= 1024
            int ex = (int)std::floor(std::log2(1024.0 / (double)m));
            S = std::ldexp(1.0, ex);
        }
        h->scale = S;
    }
    const SetConsts k = consts_for(h->cfg.set, h->scale);
    LEE_CK(h, h->ops->init(h->cfg.storage, dr, du, dt, state(h, 0), h->cells, h->pitch, k, h->st), "init kernel");
    if (sponge_active(h))
        LEE_CK(h, h->ops->sponge_damp(h->cfg.storage, h->buf[0], (int)h->cfg.nx, (int)h->cfg.ny, (int)h->cfg.nz, h->pitch,
                                      h->cfg.sponge_width, h->cfg.sponge_strength, h->st),
               "sponge damp");
    h->cur = 0;
    h->steps = 0;
    if (!on_device) LEE_SYNC(h);
    return LEE_OK;
}

lee_status lee_lbm_step(lee_lbm *h, int64_t n) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (n < 0) return fail(h, LEE_ERR_INVALID_ARGUMENT, "step: n < 0");
    if (h->slab && n > 1)
        return fail(h, LEE_ERR_INVALID_ARGUMENT, "step: a slab takes one step per halo exchange (lee_lbm_slab_step)");
    const bool learned = learned_active(h);
    StepLaunch L{};
    L.storage = h->cfg.storage;
    L.nx = (int)h->cfg.nx;
    L.ny = (int)h->cfg.ny;
    L.nz = (int)h->cfg.nz;
    L.pitch = h->pitch;
    L.open = h->cfg.bc != LEE_BC_PERIODIC && h->cfg.bc != LEE_BC_SLAB;
    L.slab = h->slab ? 1 : 0;
    L.omega = omega_for(h->cfg.storage, h->cfg.tau);
    const bool is16 = h->cfg.storage == LEE_STORE_F16 || h->cfg.storage == LEE_STORE_BF16;
    fold_coefficients(h->cfg.set, is16, L.omega, L.coefM, L.coefN);
    L.sponge_w = sponge_active(h) ? h->cfg.sponge_width : 0;
    L.sponge_smax = h->cfg.sponge_strength;
    L.ghost = learned ? h->ghost : nullptr;
    L.ghost_L = learned ? h->ghost_L : 0;
    L.force_scalar = h->force_scalar ? 1 : 0;
    L.bfp_cells = h->bfp_cells;
    L.store_scale = h->scale;
    L.t3_tma = tma_tile(h) ? 1 : 0;
    L.wait_flag = h->wait_dev;
    L.wait_ns = g_stage_wait_ns.load(std::memory_order_relaxed);
    L.t3_inject = g_inject_stage.load(std::memory_order_relaxed);
    // One time step's launches on stream `st`.  Learned edge: one launch of k_learned_step, whose
    // first blocks run the boundary network and write the border cells of the new state (pulled
    // with the entering populations and collided) while the others step the interior cells.  With
    // LEE_LEARNED_STREAMS=1 the same work runs as three launches instead: on a side stream the
    // network and k_edge_fixup (the border cells), meanwhile the step over the interior cells only
    // on `st` (it leaves the border cells unwritten), then `st` joins the side stream.  Either way
    // both parts read the same source state and write disjoint cells, and interior cells never
    // read the entering populations, so the state is that of a step run with them throughout.
    if (learned && h->learned_streams && !h->side) {
        LEE_CK(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "side stream");
        LEE_CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "fork event");
        LEE_CK(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "join event");
    }
    auto launch_step = [&](int from, cudaStream_t st) -> cudaError_t {
        L.src = state(h, from);
        L.dst = state(h, from ^ 1);
        L.stream = st;
        if (!learned) return h->ops->step(L);
        if (!h->learned_streams) return launch_learned_step(h->mlp, h->cfg.set, L, h->corner);
        cudaError_t e = cudaEventRecord(h->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
        if (e == cudaSuccess)
            e = launch_mlp_boundary(h->mlp, h->cfg.storage, h->buf[from], h->pitch, (int)h->cfg.nx, (int)h->cfg.ny,
                                    h->ghost, h->ghost_L, h->side);
        if (e == cudaSuccess) {
            StepLaunch F = L;
            F.stream = h->side;
            e = h->ops->edge_fixup(F);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side);
        if (e != cudaSuccess) return e;
        L.ghost = nullptr;  // the interior cells, which no ghost reaches
        L.skip_border = 1;
        e = h->ops->step(L);
        L.skip_border = 0;
        L.ghost = h->ghost;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_join, 0);
        return e;
    };
    int64_t left = n;
    // 1D grids that fit in shared memory: every step in one launch of the on-chip kernel
    if (n >= 2 && onchip(h)) {
        L.stream = h->st;
        LEE_CK(h, h->ops->onchip_1d(L, h->buf[h->cur], n), "on-chip 1D launch");
        h->steps += n;
        return LEE_OK;
    }
    // Periodic 2D FP32 grids whose width is a multiple of 4: several steps per launch
    // (temporal blocking; bit-identical to single steps).
    const int unit = fused_steps(h);
    auto launch_unit = [&](int from, cudaStream_t st) -> cudaError_t {
        if (unit == 1) return launch_step(from, st);
        L.src = h->buf[from];
        L.dst = h->buf[from ^ 1];
        L.stream = st;
        if (h->D == 3) return h->ops->step3d2(L);
        return unit == 2 ? h->ops->step2(L) : h->ops->stepk(L, unit);
    };
    int64_t units = n / unit;
    if (units * unit >= kGraphMinSteps) {
        // Runs of up to kMaxGraphSteps steps are one launch of a graph holding all of them;
        // longer runs replay a kChunkGraphSteps graph.  Graphs hold an even number of launches,
        // so a replay leaves the buffer parity unchanged; they are captured once per (parity,
        // length) on a private stream and replayed on the handle's stream.
        const long long gunits =
            units * unit <= kMaxGraphSteps ? (units & ~1LL) : (kChunkGraphSteps / unit) & ~1LL;
        while (gunits > 0 && units >= gunits) {
            const long long gsteps = gunits * unit;
            auto it = h->exec.find({h->cur, gsteps});
            cudaGraphExec_t ex = it == h->exec.end() ? nullptr : it->second;
            if (!ex) {
                if (!h->cap) LEE_CK(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "capture stream");
                cudaGraph_t g = nullptr;
                LEE_CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
                cudaError_t e = cudaSuccess;
                int w = h->cur;
                for (long long k = 0; k < gunits && e == cudaSuccess; ++k, w ^= 1) e = launch_unit(w, h->cap);
                cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
                if (g) cudaGraphDestroy(g);
                LEE_CK(h, e, "step graph capture");
                h->exec[{h->cur, gsteps}] = ex;
            }
            LEE_CK(h, cudaGraphLaunch(ex, h->st), "step graph launch");
            units -= gunits;
            h->steps += gsteps;
        }
    }
    for (; units > 0; --units) {
        LEE_CK(h, launch_unit(h->cur, h->st), "step launch");
        h->cur ^= 1;
        h->steps += unit;
    }
    left = n % unit;
    for (; left > 0; --left) {
        LEE_CK(h, launch_step(h->cur, h->st), "step launch");
        h->cur ^= 1;
        h->steps++;
    }
    return LEE_OK;
}

lee_status lee_lbm_moments(lee_lbm *h, double *rho, double *u, double *theta, int32_t on_device) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    const SetConsts k = consts_for(h->cfg.set, h->scale);
    if (on_device) {
        LEE_CK(h, h->ops->moments(h->cfg.storage, state(h, h->cur), h->cells, h->pitch, k, rho, u, theta, h->st), "moments");
        return LEE_OK;
    }
    {
        double *mr = mapped_host(rho), *mu = mapped_host(u), *mt = mapped_host(theta);
        if ((!rho || mr) && (!u || mu) && (!theta || mt)) {  // write the mapped host buffers directly
            LEE_CK(h, h->ops->moments(h->cfg.storage, state(h, h->cur), h->cells, h->pitch, k, mr, mu, mt, h->st),
                   "moments");
            LEE_SYNC(h);
            return LEE_OK;
        }
    }
    if ((s = ensure_fields(h)) != LEE_OK) return s;
    double *fr = h->fields, *fu = h->fields + h->cells, *ft = h->fields + (size_t)(h->D + 1) * h->cells;
    LEE_CK(h, h->ops->moments(h->cfg.storage, state(h, h->cur), h->cells, h->pitch, k, fr, fu, ft, h->st), "moments");
    const size_t n = sizeof(double) * (size_t)h->cells;
    if (rho) LEE_CK(h, cudaMemcpyAsync(rho, fr, n, cudaMemcpyDeviceToHost, h->st), "D2H rho");
    if (u) LEE_CK(h, cudaMemcpyAsync(u, fu, n * h->D, cudaMemcpyDeviceToHost, h->st), "D2H u");
    if (theta) LEE_CK(h, cudaMemcpyAsync(theta, ft, n, cudaMemcpyDeviceToHost, h->st), "D2H theta");
    LEE_SYNC(h);
    return LEE_OK;
}

lee_status lee_lbm_reduce(lee_lbm *h, double *out, int32_t on_device) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (!out) return fail(h, LEE_ERR_INVALID_ARGUMENT, "reduce: NULL out");
    const SetConsts k = consts_for(h->cfg.set, h->scale);
    const int nv = h->D + 4;
    LEE_CK(h, h->ops->reduce_partial(h->cfg.storage, state(h, h->cur), h->cells, h->pitch, k, h->partial, h->nblocks, h->st),
           "reduce_partial");
    double *dst = on_device ? out : h->red_out;
    const bool is16 = h->cfg.storage == LEE_STORE_F16 || h->cfg.storage == LEE_STORE_BF16;
    const ReduceCombine rc = make_reduce_combine(h->ops, k, is16);
    k_reduce_final<<<1, 32 * rc.nraw, 0, h->st>>>(h->partial, h->nblocks, rc, dst);
    LEE_CK(h, cudaGetLastError(), "reduce_final");
    if (!on_device) {
        LEE_CK(h, cudaMemcpyAsync(out, h->red_out, sizeof(double) * nv, cudaMemcpyDeviceToHost, h->st), "D2H reduce");
        LEE_SYNC(h);
    }
    return LEE_OK;
}

lee_status lee_lbm_check_finite(lee_lbm *h) {
    double out[kReduceMax];
    lee_status s = lee_lbm_reduce(h, out, 0);
    if (s != LEE_OK) return s;
    if (out[h->D + 3] != 0.0) return fail(h, LEE_ERR_NONFINITE, "non-finite populations present");
    return LEE_OK;
}

lee_status lee_lbm_get_populations(lee_lbm *h, double *g, int32_t on_device) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (!g) return fail(h, LEE_ERR_INVALID_ARGUMENT, "get_populations: NULL");
    const SetConsts k = consts_for(h->cfg.set, h->scale);
    double *dst = g;
    if (!on_device) {
        if ((s = ensure_pops64(h)) != LEE_OK) return s;
        dst = h->pops64;
    }
    LEE_CK(h, h->ops->export_f64(h->cfg.storage, state(h, h->cur), h->cells, h->pitch, k, dst, h->st), "export");
    if (!on_device) {
        LEE_CK(h, cudaMemcpyAsync(g, dst, sizeof(double) * (size_t)h->Q * h->cells, cudaMemcpyDeviceToHost, h->st), "D2H g");
        LEE_SYNC(h);
    }
    return LEE_OK;
}

lee_status lee_lbm_set_populations(lee_lbm *h, const double *g, int32_t on_device) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (!g) return fail(h, LEE_ERR_INVALID_ARGUMENT, "set_populations: NULL");
    const SetConsts k = consts_for(h->cfg.set, h->scale);
    const double *src = g;
    if (!on_device) {
        if ((s = ensure_pops64(h)) != LEE_OK) return s;
        LEE_CK(h, cudaMemcpyAsync(h->pops64, g, sizeof(double) * (size_t)h->Q * h->cells, cudaMemcpyHostToDevice, h->st),
               "H2D g");
        src = h->pops64;
    }
    h->cur = 0;
    LEE_CK(h, h->ops->import_f64(h->cfg.storage, src, h->cells, h->pitch, k, state(h, 0), h->st), "import");
    h->steps = 0;
    if (!on_device) LEE_SYNC(h);
    return LEE_OK;
}

lee_status lee_lbm_set_boundary_mlp(lee_lbm *h, const float *params, int64_t nparams) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (h->cfg.bc != LEE_BC_OPEN_LEARNED) return fail(h, LEE_ERR_INVALID_ARGUMENT, "set_boundary_mlp: bc is not learned");
    if (h->cfg.set != LEE_D2Q5) return fail(h, LEE_ERR_UNSUPPORTED, "set_boundary_mlp: five-velocity monoatomic set only");
    if (!params || nparams != 5313) return fail(h, LEE_ERR_INVALID_ARGUMENT, "set_boundary_mlp: need 5313 parameters");
    float *tmp = nullptr;
    if (!h->mlp) LEE_CK(h, cudaMalloc(&h->mlp, 20480), "cudaMalloc(network)");
    LEE_CK(h, cudaMalloc(&tmp, sizeof(float) * 5313), "cudaMalloc(params)");
    cudaError_t e = cudaMemcpyAsync(tmp, params, sizeof(float) * 5313, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = mlp_pack(tmp, h->mlp, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    cudaFree(tmp);
    LEE_CK(h, e, "install network");
    if (!h->mlp_ready) drop_step_graphs(h);  // from the fallback edge to the network
    h->mlp_ready = true;
    return LEE_OK;
}

lee_status lee_lbm_set_boundary_mlp_for_tau(lee_lbm *h, const float *params, int64_t nparams, double trained_tau,
                                            double tau_tolerance, int32_t *installed) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (!std::isfinite(trained_tau) || !(tau_tolerance >= 0.0) || !std::isfinite(tau_tolerance))
        return fail(h, LEE_ERR_INVALID_ARGUMENT, "set_boundary_mlp_for_tau: bad trained tau or tolerance");
    if (std::fabs(h->cfg.tau - trained_tau) > tau_tolerance) {  // not this network: keep or return to the fallback
        if (h->cfg.bc != LEE_BC_OPEN_LEARNED)
            return fail(h, LEE_ERR_INVALID_ARGUMENT, "set_boundary_mlp_for_tau: bc is not learned");
        if (h->mlp_ready) drop_step_graphs(h);
        h->mlp_ready = false;
        if (installed) *installed = 0;
        return LEE_OK;
    }
    s = lee_lbm_set_boundary_mlp(h, params, nparams);
    if (s == LEE_OK && installed) *installed = 1;
    return s;
}

lee_status lee_lbm_boundary_in_use(lee_lbm *h, int32_t *bc) {
    if (!h || !bc) return LEE_ERR_INVALID_ARGUMENT;
    if (h->cfg.bc != LEE_BC_OPEN_LEARNED) *bc = h->cfg.bc;
    else *bc = h->mlp_ready ? LEE_BC_OPEN_LEARNED : (h->cfg.sponge_width > 0 ? LEE_BC_OPEN_SPONGE : LEE_BC_OPEN_ZERO);
    return LEE_OK;
}

lee_status lee_lbm_slab_info(lee_lbm *h, int32_t *crossing, int64_t *plane_cells, int64_t *bytes) {
    if (!h) return LEE_ERR_INVALID_ARGUMENT;
    if (!h->slab) return fail(h, LEE_ERR_INVALID_ARGUMENT, "slab_info: not a slab");
    if (crossing) *crossing = h->crossing;
    if (plane_cells) *plane_cells = h->plane;
    if (bytes) *bytes = (int64_t)(h->elem * (size_t)h->crossing * (size_t)h->plane);
    return LEE_OK;
}

lee_status lee_lbm_slab_buffers(lee_lbm *h, void **send_lo, void **send_hi, void **recv_lo, void **recv_hi) {
    if (!h) return LEE_ERR_INVALID_ARGUMENT;
    if (!h->slab) return fail(h, LEE_ERR_INVALID_ARGUMENT, "slab_buffers: not a slab");
    if (send_lo) *send_lo = h->halo[0];
    if (send_hi) *send_hi = h->halo[1];
    if (recv_lo) *recv_lo = h->halo[2];
    if (recv_hi) *recv_hi = h->halo[3];
    return LEE_OK;
}

lee_status lee_lbm_slab_pack(lee_lbm *h) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (!h->slab) return fail(h, LEE_ERR_INVALID_ARGUMENT, "slab_pack: not a slab");
    LEE_CK(h, h->ops->slab_pack(h->cfg.storage, state(h, h->cur), h->pitch, h->plane, h->nl, h->halo[0], h->halo[1], h->st),
           "slab pack");
    return LEE_OK;
}

lee_status lee_lbm_slab_unpack(lee_lbm *h) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    if (!h->slab) return fail(h, LEE_ERR_INVALID_ARGUMENT, "slab_unpack: not a slab");
    LEE_CK(h, h->ops->slab_unpack(h->cfg.storage, state(h, h->cur), h->pitch, h->plane, h->nl, h->halo[2], h->halo[3],
                                  h->st),
           "slab unpack");
    return LEE_OK;
}

lee_status lee_lbm_slab_step(lee_lbm *const *slabs, int32_t count, int64_t n) {
    if (!slabs || count < 1 || n < 0) return LEE_ERR_INVALID_ARGUMENT;
    for (int k = 0; k < count; ++k) {
        lee_lbm *h = slabs[k];
        if (!h) return LEE_ERR_INVALID_ARGUMENT;
        if (h->poisoned) return LEE_ERR_POISONED;
        const lee_lbm *a = slabs[0];
        const bool same = h->slab && h->cfg.set == a->cfg.set && h->cfg.storage == a->cfg.storage &&
                          h->cfg.tau == a->cfg.tau && h->cfg.nx == a->cfg.nx && h->plane == a->plane &&
                          h->device == a->device && h->st == a->st;
        if (!same)
            return fail(h, LEE_ERR_INVALID_ARGUMENT,
                        "slab_step: slabs of one domain (same set, storage, tau, plane, device and stream) only");
        for (int j = 0; j < k; ++j)
            if (slabs[j] == h) return fail(h, LEE_ERR_INVALID_ARGUMENT, "slab_step: a slab is listed twice");
    }
    const size_t bytes = slabs[0]->elem * (size_t)slabs[0]->crossing * (size_t)slabs[0]->plane;
    for (int64_t t = 0; t < n; ++t) {
        lee_status s;
        for (int k = 0; k < count; ++k)
            if ((s = lee_lbm_slab_pack(slabs[k])) != LEE_OK) return s;
        // slab k + 1 lies above slab k, and the last one below the first (periodic domain); each
        // message is copied into the receiving slab's own buffer, in stream order
        for (int k = 0; k < count; ++k) {
            lee_lbm *h = slabs[k], *below = slabs[(k + count - 1) % count], *above = slabs[(k + 1) % count];
            LEE_CK(h, cudaMemcpyAsync(below->halo[3], h->halo[0], bytes, cudaMemcpyDeviceToDevice, h->st), "halo copy");
            LEE_CK(h, cudaMemcpyAsync(above->halo[2], h->halo[1], bytes, cudaMemcpyDeviceToDevice, h->st), "halo copy");
        }
        for (int k = 0; k < count; ++k)
            if ((s = lee_lbm_slab_unpack(slabs[k])) != LEE_OK) return s;
        for (int k = 0; k < count; ++k)
            if ((s = lee_lbm_step(slabs[k], 1)) != LEE_OK) return s;
    }
    return LEE_OK;
}

lee_status lee_lbm_steps_done(lee_lbm *h, int64_t *steps) {
    if (!h || !steps) return LEE_ERR_INVALID_ARGUMENT;
    *steps = h->steps;
    return LEE_OK;
}

lee_status lee_lbm_steps_per_launch(lee_lbm *h, int32_t *steps) {
    if (!h || !steps) return LEE_ERR_INVALID_ARGUMENT;
    *steps = onchip(h) ? 0 : fused_steps(h);
    return LEE_OK;
}

lee_status lee_lbm_store_scale(lee_lbm *h, double *scale) {
    if (!h || !scale) return LEE_ERR_INVALID_ARGUMENT;
    *scale = h->scale;
    return LEE_OK;
}

lee_status lee_lbm_sync(lee_lbm *h) {
    lee_status s = enter(h);
    if (s != LEE_OK) return s;
    LEE_SYNC(h);
    return LEE_OK;
}

const char *lee_lbm_last_error(lee_lbm *h) { return h ? h->err.c_str() : "NULL handle"; }

lee_status lee_lbm_destroy(lee_lbm *h) {
    if (!h) return LEE_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->st);
    for (auto &kv : h->exec) cudaGraphExecDestroy(kv.second);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    free_all(h);
    delete h;
    cudaGetLastError();
    return LEE_OK;
}

}  // extern "C"

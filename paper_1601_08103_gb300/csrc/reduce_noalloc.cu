// reduce_noalloc.cu -- lee_reduce_noalloc: the global sums of lee_lbm_reduce for a population
// field the caller owns, computed without allocating any memory.
//
// Who needs this: code that may not call cudaMalloc or any allocating routine at the point where
// it needs the diagnostics -- for instance a host callback or plugin running inside someone
// else's memory pool or allocator budget, a process that pins its device memory up front and
// forbids later allocations, or a caller between allocation-free phases of a larger application.
// The regular entry point needs a solver handle, whose creation allocates the block-partial
// scratch; this one takes the populations and the output directly and keeps its scratch in a
// fixed file-scope device array instead.
//
// The scratch: kMaxPartials block partials x kReduceMax values in FP64 (2432 x 16 x 8 B =
// 311,296 bytes).  Every GPU that loads the library holds this array until the process exits.
// The launch shape is the one lee_lbm_reduce uses (min(ceil(cells / 256), 2432) blocks of 256
// threads, grid-stride), so the two entry points sum in the same order and agree bit for bit.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lee_lbm.h"
#include "ops.cuh"

namespace lee {
SetConsts consts_for(int set, double scale);
}

using namespace lee;

namespace {

constexpr int kMaxPartials = kMaxAuxBlocks;  // rows of partials: the most blocks aux_blocks() gives
static_assert(kMaxPartials * kReduceMax * sizeof(double) == 311296, "scratch size as documented in lee_lbm.h");
constexpr int kMaxDevices = 64;

// Scratch for the block partials.  In host code this name is only a stand-in for the device
// array, not its address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_partials[kMaxPartials * kReduceMax];

std::mutex g_setup_mutex;
double *g_partials_addr[kMaxDevices] = {nullptr};

// Resolves the device address of the scratch on the current device, once per device.
cudaError_t partials_on_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_partials_addr[dev] == nullptr) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double *>(ptr);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lee_status lee_reduce_noalloc(int32_t set, int32_t storage, const void *g, int64_t cells, int64_t pitch,
                                         double store_scale, double *out, void *cuda_stream) {
    const SetOps *o = set_ops(set);
    if (!o || !g || !out) return LEE_ERR_INVALID_ARGUMENT;
    if (storage < LEE_STORE_F64 || storage > LEE_STORE_BF16) return LEE_ERR_INVALID_ARGUMENT;
    if (cells < 1 || cells >= (1LL << 31) || pitch < cells) return LEE_ERR_INVALID_ARGUMENT;
    const bool is16 = storage == LEE_STORE_F16 || storage == LEE_STORE_BF16;
    if (is16 && !(store_scale > 0.0)) return LEE_ERR_INVALID_ARGUMENT;
    const int nblocks = aux_blocks(cells, kReduceThreads);
    if (nblocks > kMaxPartials) return LEE_ERR_INVALID_ARGUMENT;  // beyond the fixed scratch
    double *partials = nullptr;
    if (partials_on_current_device(&partials) != cudaSuccess) return LEE_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const SetConsts k = consts_for(set, is16 ? store_scale : 1.0);
    // Each block overwrites its own partials before the final pass reads them, so nothing in the
    // shared scratch has to be cleared between calls.
    if (o->reduce_partial(storage, g, cells, pitch, k, partials, nblocks, st) != cudaSuccess) return LEE_ERR_CUDA;
    const ReduceCombine rc = make_reduce_combine(o, k, is16);
    k_reduce_final<<<1, 32 * rc.nraw, 0, st>>>(partials, nblocks, rc, out);
    if (cudaGetLastError() != cudaSuccess) return LEE_ERR_CUDA;
    return LEE_OK;
}

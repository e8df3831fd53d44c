// probe.cu -- lee_probe_fp64_fma (include/lee_lbm.h): the device's FP64 fused multiply-add rate,
// measured, so that the FP64 storage forms of the solver (whose collision is FP64 arithmetic) can
// be stated against a measured FP64 roofline instead of a nominal one.
//
// Every thread runs 8 independent dependency chains of FP64 fma (x = x * a + b, |a| < 1, so the
// values stay finite and normal), enough to hide the pipe latency; the grid is 8 blocks of 256
// threads per SM.  One fma counts as 2 floating-point operations.
#include <cuda_runtime.h>

#include "../../include/lee_lbm.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(long long iters, double a, double b, double *__restrict__ sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (long long k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) sink[threadIdx.x] = s;  // keeps the chains alive; never true
}

}  // namespace

extern "C" lee_status lee_probe_fp64_fma(int64_t iters, double *flops_per_s) {
    if (iters < 1 || iters > (1LL << 30) || !flops_per_s) return LEE_ERR_INVALID_ARGUMENT;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LEE_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LEE_ERR_CUDA;
    const int blocks = 8 * sms, threads = 256;
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(double) * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_fp64_fma<<<blocks, threads>>>(iters / 8 + 1, 0.999999, 1e-7, sink);  // warm-up
        e = cudaEventRecord(e0);
    }
    if (e == cudaSuccess) {
        k_fp64_fma<<<blocks, threads>>>(iters, 0.999999, 1e-7, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || !(ms > 0.f)) {
        cudaGetLastError();
        return LEE_ERR_CUDA;
    }
    *flops_per_s = 2.0 * kChains * (double)iters * (double)blocks * threads / (ms * 1e-3);
    return LEE_OK;
}

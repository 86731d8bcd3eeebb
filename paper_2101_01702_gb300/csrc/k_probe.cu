// Throughput probes of the GPU's double-precision arithmetic: the peak the
// step's kernels are measured against.  The step is bound by FP64 work
// (temperature iteration, Stefan-Maxwell solve, reaction rates), so its
// roofline needs the rate of a fused multiply-add in double and of the
// double exponential and logarithm, timed on the device itself rather than
// derived from unit counts and the nominal clock.
//
//   LBM_PROBE_DFMA : 8 independent chains a <- fma(a, b, c) per thread
//                    (b = 1 - 2^-20, c = 2^-20: every chain stays near 1,
//                    no denormals, no overflow); 2 flops per FMA.
//   LBM_PROBE_EXP  : 4 independent chains y <- exp(-y) (fixed point 0.567).
//   LBM_PROBE_LOG  : 4 independent chains y <- log(y + 2) (fixed point 1.146).
//
// The chains' results feed a store that never happens (their sum is never
// negative), so the compiler keeps every operation.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/lbm.h"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_probe_dfma(int iters, double *sink)
{
    const double b = 1.0 - 0x1p-20, c = 0x1p-20;
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s < 0.0) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_exp(int iters, double *sink)
{
    double y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) y[k] = 0.5 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < 4; ++k) y[k] = exp(-y[k]);
    if (y[0] + y[1] + y[2] + y[3] < 0.0) sink[blockIdx.x] = y[0];
}

__global__ void __launch_bounds__(kThreads) k_probe_log(int iters, double *sink)
{
    double y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) y[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < 4; ++k) y[k] = log(y[k] + 2.0);
    if (y[0] + y[1] + y[2] + y[3] < 0.0) sink[blockIdx.x] = y[0];
}

}  // namespace

extern "C" int lbm_fp64_probe(int kind, int blocks, int iters, double *sink, double *out, void *cuda_stream)
{
    if (!sink || !out || blocks < 1 || iters < 1) return LBM_ERR_ARG;
    if (kind != LBM_PROBE_DFMA && kind != LBM_PROBE_EXP && kind != LBM_PROBE_LOG) return LBM_ERR_ARG;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, sink) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return LBM_ERR_ARG;
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LBM_ERR_CUDA;
    }
    int st = LBM_OK;
    if (cudaEventRecord(e0, stream) != cudaSuccess) st = LBM_ERR_CUDA;
    if (st == LBM_OK) {
        if (kind == LBM_PROBE_DFMA) k_probe_dfma<<<blocks, kThreads, 0, stream>>>(iters, sink);
        else if (kind == LBM_PROBE_EXP) k_probe_exp<<<blocks, kThreads, 0, stream>>>(iters, sink);
        else k_probe_log<<<blocks, kThreads, 0, stream>>>(iters, sink);
        if (cudaGetLastError() != cudaSuccess) st = LBM_ERR_CUDA;
    }
    if (st == LBM_OK && cudaEventRecord(e1, stream) != cudaSuccess) st = LBM_ERR_CUDA;
    if (st == LBM_OK && cudaEventSynchronize(e1) != cudaSuccess) st = LBM_ERR_CUDA;
    float ms = 0.f;
    if (st == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = LBM_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    const double threads = (double)blocks * kThreads;
    // operations per thread: 32 FMA (2 flops each) per iteration, or 4 calls
    const double ops = kind == LBM_PROBE_DFMA ? threads * iters * 32.0 * 2.0 : threads * iters * 4.0;
    out[0] = ms;
    out[1] = ops / (ms * 1e-3);
    return LBM_OK;
}

// pp_measure_fp64_rate: the FP64 (non-tensor) FMA throughput of the current
// GPU, measured with a kernel of independent FMA chains, for the roofline of
// the FP64 kernels (the FP64 pass and sweeps are bound by FP64 arithmetic on
// this part, not by memory).  Not part of the method.
#include "pp_internal.h"

#include <cuda_runtime.h>

namespace {

// Written only when the chains reach an impossible value, so that the
// compiler keeps every FMA; nothing reads it.
__device__ double g_fma_sink;

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + 1) + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.2345e300) g_fma_sink = s;
}

}  // namespace

extern "C" pp_status pp_measure_fp64_rate(void *stream, double *flops_per_s) {
    if (!flops_per_s) return pp_fail(PP_EINVAL, "pp_measure_fp64_rate: null output");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "pp_measure_fp64_rate: %s", cudaGetErrorString(e));
    const int threads = 256, blocks = sms * 8, iters = 4096;
    // a = 1 - 2^-20, b small: the chains stay finite and normal for any iteration count
    const double a = 1.0 - 1.0 / (1 << 20), b = 1e-7;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return pp_fail(PP_ECUDA, "pp_measure_fp64_rate: event creation failed");
    double best = 0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, st);
        k_fp64_fma<<<blocks, threads, 0, st>>>(iters, a, b);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * kChains * 8.0 * iters * (double)threads * blocks;
        if (rep > 0 && ms > 0 && flops / (ms * 1e-3) > best) best = flops / (ms * 1e-3);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "pp_measure_fp64_rate: %s", cudaGetErrorString(e));
    *flops_per_s = best;
    return PP_OK;
}

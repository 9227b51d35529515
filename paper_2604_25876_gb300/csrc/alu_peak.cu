// alu_peak.cu -- measured fused multiply-add throughput of the device: the
// ALU roofline denominators for the step kernels (packed FP32 pairs for the
// streaming FP32 kernel, FP64 for the FP64 path).  A diagnostic, not part of
// the method: every thread runs independent FMA chains long enough that the
// launch overhead is negligible, and the sum of the chains is kept live.
#include <cuda_runtime.h>

#include <algorithm>

#include "skyrme.h"

namespace {

constexpr int kChains = 8;    // independent chains per thread
constexpr int kThreads = 256;

__device__ float g_sink32;
__device__ double g_sink64;

__global__ void __launch_bounds__(kThreads) k_ffma2(int iters, float2 a, float2 b)
{
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = make_float2(1e-3f * (threadIdx.x + c), 1e-3f * (blockIdx.x + c));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
    if (s == 1234.5f) g_sink32 = s;  // practically never: keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_dfma(int iters, double a, double b)
{
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = 1e-3 * (threadIdx.x + c + blockIdx.x);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 1234.5) g_sink64 = s;
}

}  // namespace

extern "C" skyrme_status skyrme_measure_fma_peak(int kind, double *tflops, void *stream)
{
    if (!tflops || (kind != SKYRME_PEAK_FP32 && kind != SKYRME_PEAK_FP64)) return SKYRME_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SKYRME_ECUDA;
    const int blocks = std::max(1, sms) * 8;
    // values that keep every chain finite: |a| < 1 contracts towards b / (1 - a)
    const int iters = kind == SKYRME_PEAK_FP32 ? 1 << 14 : 1 << 10;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return SKYRME_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SKYRME_ECUDA;
    }
    float best_ms = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {  // the first launch warms up
        ok = cudaEventRecord(e0, s) == cudaSuccess;
        if (kind == SKYRME_PEAK_FP32)
            k_ffma2<<<blocks, kThreads, 0, s>>>(iters, make_float2(0.999f, 0.998f),
                                                make_float2(1e-4f, 2e-4f));
        else
            k_dfma<<<blocks, kThreads, 0, s>>>(iters, 0.999, 1e-4);
        ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || !(best_ms > 0.f)) return SKYRME_ECUDA;
    // an FMA is 2 floating-point operations; an FP32 pair instruction does two
    const double fma_per_chain = kind == SKYRME_PEAK_FP32 ? 2.0 : 1.0;
    const double flops = 2.0 * fma_per_chain * kChains * (double)iters * kThreads * blocks;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return SKYRME_OK;
}

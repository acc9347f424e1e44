// FP32 FMA throughput microbenchmark: the roofline denominator of the
// spectral path, whose hot loops are FP32 FMA/MUL/ALU work.  Every thread
// runs 8 independent FMA chains (enough to cover the FMA latency), every SM
// holds 2048 threads, and the result is only stored when an impossible value
// appears, so no chain can be removed.
#include "cwth_internal.h"

namespace cwth {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 512;

__global__ void __launch_bounds__(kPeakThreads) ffma_kernel(float* sink, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j) * 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -12345.678f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace cwth

extern "C" cwth_status cwth_measure_fp32_fma(double* tflops, void* stream) {
    if (!tflops) return CWTH_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CWTH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&sink, sizeof(float) * 4 * sms);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 4 * sms;  // 2048 threads per SM
    const int iters = 4096;      // 4096 x 16 x 8 FMAs per thread
    float best_ms = 0.f;
    // b < 1 keeps the chains bounded (a -> c / (1 - b)).
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            cwth::ffma_kernel<<<blocks, cwth::kPeakThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess || best_ms <= 0.f) return CWTH_ERR_CUDA;
    const double flops = 2.0 * cwth::kChains * 16.0 * iters * (double)blocks * cwth::kPeakThreads;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return CWTH_OK;
}

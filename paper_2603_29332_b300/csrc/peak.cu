// peak.cu -- FP32 FMA throughput microbenchmark: the measured denominator of the step kernel's
// ALU roofline (beside the figure derived from SMs x 128 lanes x 2 FLOP x clock).
#include <cuda_runtime.h>

#include "../../include/msim.h"

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (hides the FMA latency)

__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1e-3f * (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

}  // namespace

extern "C" {

msim_status msim_measure_fp32_peak(int32_t device, double* tflops) {
    if (!tflops) return MSIM_ERR_ARG;
    *tflops = 0.0;
    if (cudaSetDevice(device) != cudaSuccess) return MSIM_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * 8, threads = 256, iters = 1 << 16;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(float) * blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first launch warms up
        e = cudaEventRecord(e0, 0);
        k_fma_peak<<<blocks, threads>>>(out, iters, 0.9999999f, 1e-7f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return MSIM_ERR_CUDA;
    *tflops = 2.0 * kChains * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
    return MSIM_OK;
}

}  // extern "C"

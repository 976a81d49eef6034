// Measured FP32-FMA and MUFU (ex2) throughput of the device: the denominators of the sweep's
// FP32-issue and SFU roofline terms (the paper has no counterpart).  Each thread runs eight
// independent dependency chains, so the pipes, not latency, bound the rate; the grid holds
// eight 256-thread blocks per SM.
#include <cuda_runtime.h>

#include "helios.h"

namespace {

constexpr int kChains = 8;

__global__ void fma_chains(float* out, int iters, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678f) out[blockIdx.x] = s;     // keeps the chains live; never true in practice
}

__global__ void ex2_chains(float* out, int iters)
{
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = -1.0f / (float)(threadIdx.x + j + 1);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            float r;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[j]));
            a[j] = -r;                             // stays in [-1, 0): 2^a in [0.5, 1)
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace

// defined in helios_api.cu
__attribute__((visibility("hidden"))) int helios_ctx_device(const helios_ctx* ctx);

extern "C" {

int helios_measure_peaks(helios_ctx* ctx, double* fp32_tflops, double* sfu_tops)
{
    if (!ctx || !fp32_tflops || !sfu_tops) return HELIOS_EINVAL;
    const int dev = helios_ctx_device(ctx);
    if (dev < 0 || cudaSetDevice(dev) != cudaSuccess) return HELIOS_ECUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HELIOS_ECUDA;
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HELIOS_OK;
    if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) return HELIOS_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = HELIOS_ECUDA;
    float ms_fma = 0.0f, ms_ex2 = 0.0f;
    if (!rc) {
        fma_chains<<<blocks, threads>>>(out, iters, 0.999f, 0.001f);     // warm-up
        ex2_chains<<<blocks, threads>>>(out, iters / 8);
        cudaEventRecord(e0);
        fma_chains<<<blocks, threads>>>(out, iters, 0.999f, 0.001f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms_fma, e0, e1);
        cudaEventRecord(e0);
        ex2_chains<<<blocks, threads>>>(out, iters / 8);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms_ex2, e0, e1);
        if (cudaGetLastError() != cudaSuccess || !(ms_fma > 0.0f) || !(ms_ex2 > 0.0f)) rc = HELIOS_ECUDA;
    }
    if (!rc) {
        const double n = (double)blocks * threads * kChains;
        *fp32_tflops = 2.0 * n * iters / (ms_fma * 1e-3) / 1e12;           // FMA = 2 flops
        *sfu_tops = n * (iters / 8) / (ms_ex2 * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

}  // extern "C"

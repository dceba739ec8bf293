// Measured FP32 arithmetic peak of the current device: the denominator of the
// "alu" roofline of the FFT kernels, taken on the GPU the kernels run on
// instead of from a datasheet.
//
// Every thread runs 8 independent chains of fused multiply-adds (enough
// independent work per warp to cover the pipeline latency), on a grid of 8
// blocks of 256 threads per SM.  Two forms are timed: the scalar fma.rn.f32
// (2 flops per lane and instruction) and the packed fma.rn.f32x2 (4 flops per
// lane and instruction, on pairs of FP32 values in one 64-bit register).  Each
// is launched once untimed and then timed with CUDA events over a fixed number
// of iterations; flops = threads x iterations x chains x flops per chain step.
#include <cstdint>

#include "common.cuh"
#include "profile.cuh"

namespace jdft {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) peak_ffma_kernel(float* out, int iters, float b, float c) {
    float a[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) a[i] = (float)(threadIdx.x + i);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[i]) : "f"(b), "f"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += a[i];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live; practically never true
}

__global__ void __launch_bounds__(kPeakThreads) peak_ffma2_kernel(float* out, int iters, float b, float c) {
    uint64_t a[kPeakChains];
    uint64_t bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) {
        const float x = (float)(threadIdx.x + i), y = x + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(x), "f"(y));
    }
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[i]));
        s += x + y;
    }
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace jdft

using namespace jdft;

extern "C" jdft_status jdft_measure_fp32_peak(double* ffma_tflops, double* ffma2_tflops, int* sms, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(ffma_tflops && ffma2_tflops && sms, "null output pointer");
    int dev = 0;
    JDFT_CUDA_TRY(cudaGetDevice(&dev));
    JDFT_CUDA_TRY(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    float* out = nullptr;
    const int blocks = *sms * 8;
    JDFT_CUDA_TRY(cudaMallocAsync((void**)&out, (size_t)blocks * sizeof(float), st));
    cudaEvent_t e0, e1;
    JDFT_CUDA_TRY(cudaEventCreate(&e0));
    JDFT_CUDA_TRY(cudaEventCreate(&e1));
    const int iters = 8192;
    const double steps = (double)blocks * kPeakThreads * iters * 16 * kPeakChains;
    jdft_status s = JDFT_OK;
    for (int form = 0; form < 2 && s == JDFT_OK; ++form) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {  // rep 0 untimed (set-up and clock ramp)
            cudaEventRecord(e0, st);
            {
                Trace tr_(form ? "peak_ffma2" : "peak_ffma", st);
                if (form == 0) peak_ffma_kernel<<<blocks, kPeakThreads, 0, st>>>(out, iters, 0.999f, 1e-3f);
                else peak_ffma2_kernel<<<blocks, kPeakThreads, 0, st>>>(out, iters, 0.999f, 1e-3f);
            }
            cudaEventRecord(e1, st);
            if ((s = check_launch("peak")) != JDFT_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                s = set_error(JDFT_ERR_CUDA, "peak kernel failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        const double flops = steps * (form ? 4.0 : 2.0);
        (form ? *ffma2_tflops : *ffma_tflops) = flops / (best * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    return s;
}

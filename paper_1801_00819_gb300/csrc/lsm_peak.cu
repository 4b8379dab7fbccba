// FP32 arithmetic peak of the current GPU, measured: the denominator of the depth sweeps' FP32
// roofline (the sweeps are bound by the FP32 pipe, so their achieved flop rate is reported against
// what this GPU's FMA pipe sustains rather than against a datasheet figure).
//
// Every thread runs independent chains of fused multiply-adds, enough of them that the pipe never
// waits on a dependency, on a grid of several blocks per SM; the rate is the flop count (2 per FMA)
// over the CUDA-event time of the launch, best of several launches.  Two forms are timed: scalar
// FFMA (one FMA per instruction) and the paired FP32 instructions of sm_100-class GPUs (two FMAs per
// instruction), which the sweeps' butterflies use.
#include <cuda_runtime.h>

#include "../../include/lsm.h"
#include "lsm_internal.h"

namespace lsm {

// written only when the chains produce an impossible value, so the arithmetic cannot be removed
static __device__ float g_peak_sink;

constexpr int kPeakChains = 8;
constexpr int kPeakIters = 2048;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float a, float b) {
    float acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = (float)(threadIdx.x + c);
#pragma unroll 1
    for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) acc[c] = fmaf(acc[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += acc[c];
    if (s == -1.2345678e30f) g_peak_sink = s;
}

__global__ void __launch_bounds__(kPeakThreads) ffma2_peak_kernel(float a, float b) {
    float2 acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = make_float2((float)(threadIdx.x + c), (float)(c - threadIdx.x));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
    for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) acc[c] = __ffma2_rn(acc[c], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += acc[c].x + acc[c].y;
    if (s == -1.2345678e30f) g_peak_sink = s;
}

}  // namespace lsm

extern "C" int lsm_measure_fp32_peak(double* tflops_ffma, double* tflops_ffma2, void* stream) {
    using namespace lsm;
    if (!tflops_ffma || !tflops_ffma2) return LSM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return LSM_ERR_CUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = sms * 8;  // eight 256-thread blocks per SM: 64 warps, the SM's maximum
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return LSM_ERR_CUDA;
    }
    int rc = LSM_OK;
    for (int form = 0; form < 2 && rc == LSM_OK; ++form) {
        // flops per thread: iterations x 8 x chains FMAs (two per paired instruction), 2 flop each
        const double flops = (double)blocks * kPeakThreads * kPeakIters * 8 * kPeakChains * 2.0 * (form ? 2.0 : 1.0);
        float best = 0.f;
        for (int rep = 0; rep < 6 && rc == LSM_OK; ++rep) {  // the first launch warms up, the best counts
            cudaEventRecord(e0, st);
            if (form == 0)
                fma_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(1.0000001f, 1e-7f);
            else
                ffma2_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(1.0000001f, 1e-7f);
            count_launch();
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = LSM_ERR_CUDA;
                break;
            }
            if (rep > 0 && (best == 0.f || ms < best)) best = ms;
        }
        if (rc == LSM_OK) *(form ? tflops_ffma2 : tflops_ffma) = flops / (best * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return rc;
}

// peak.cu -- measured FP32 fused-multiply-add throughput of the GPU, the
// denominator of the step kernel's roofline (no counterpart in the paper).
//
// Every SM is filled with threads, each running kChains independent chains of
// dependent FMAs (enough independent work per scheduler to hide the FMA
// latency); the kernel is timed with CUDA events and the flop count is
// 2 x chains x iterations x threads.  The chains' sums are stored only when a
// run-time value nothing sets says so, so that the compiler keeps every FMA.

#include <cuda_runtime.h>

#include "qtb.h"
#include "qtb_kernels.cuh"

namespace qtb {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float *out, int iters, float seed, int store)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.999999f, b = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (store) out[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

// The measurement behind qtb_fp32_peak (which reports errors by name): QTB_OK,
// QTB_ERR_CUDA or QTB_ERR_OOM.
int measure_fp32_peak(double *tflops, double *ms)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QTB_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QTB_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0) != cudaSuccess)
        return QTB_ERR_CUDA;
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)grid * kPeakThreads) != cudaSuccess) return QTB_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QTB_OK;
    const int iters = 4096;
    float best = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = QTB_ERR_CUDA;
    } else {
        k_fma_peak<<<grid, kPeakThreads>>>(out, iters / 8, 1.0f, 0);  // warm-up
        for (int r = 0; r < 5 && rc == QTB_OK; ++r) {
            cudaEventRecord(e0);
            k_fma_peak<<<grid, kPeakThreads>>>(out, iters, 1.0f, 0);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = QTB_ERR_CUDA;
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (best == 0.f || t < best) best = t;
        }
        if (rc == QTB_OK && cudaGetLastError() != cudaSuccess) rc = QTB_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != QTB_OK) return rc;
    const double flops = 2.0 * kChains * 16.0 * iters * (double)grid * kPeakThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return QTB_OK;
}

}  // namespace qtb

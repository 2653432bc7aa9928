// paco_probe.cu -- paco_probe_fp64_peak: the FP64 fused multiply-add rate of
// the current device, measured.  The complex128 transforms are bound by
// FP64 arithmetic on this GPU, so their roofline needs this denominator; the
// paper has no counterpart (its machine model counts operations, not rates).
#include <cuda_runtime.h>

#include "../../include/paco.h"
#include "paco_plan.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (covers the DFMA latency)
constexpr int kUnroll = 16;

__device__ double g_sink;       // written only if the chains ever sum to -1 (they cannot)

// Each thread runs kChains independent chains of `iters * kUnroll` FMAs
// a = a * m + c (positive, converging to c / (1 - m)); the sum is stored only
// if it equals -1, so the work cannot be removed and nothing is written.
__global__ void __launch_bounds__(256) dfma_peak_kernel(long long iters)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    const double m = 0.9999999, c = 1e-9;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) g_sink = s;
}

} // namespace

extern "C" paco_status_t paco_probe_fp64_peak(int64_t iters, double *gflops, float *ms, paco_stream_t stream)
{
    using paco::fail;
    if (iters < 1 || !gflops) return fail(PACO_ERR_INVALID_ARG, "paco_probe_fp64_peak: iters >= 1 and gflops required");
    int dev = 0, sms = 0;
    PACO_CUDA_TRY(cudaGetDevice(&dev));
    PACO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;           // 64 warps per SM
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    PACO_CUDA_TRY(cudaEventCreate(&a));
    PACO_CUDA_TRY(cudaEventCreate(&b));
    dfma_peak_kernel<<<blocks, threads, 0, s>>>(iters > 64 ? 64 : (long long)iters);   // warm-up
    PACO_CUDA_TRY(cudaGetLastError());
    PACO_CUDA_TRY(cudaEventRecord(a, s));
    dfma_peak_kernel<<<blocks, threads, 0, s>>>((long long)iters);
    PACO_CUDA_TRY(cudaGetLastError());
    PACO_CUDA_TRY(cudaEventRecord(b, s));
    PACO_CUDA_TRY(cudaEventSynchronize(b));
    float t = 0.f;
    PACO_CUDA_TRY(cudaEventElapsedTime(&t, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double flops = 2.0 * (double)blocks * threads * kChains * kUnroll * (double)iters;
    *gflops = flops / ((double)t * 1e-3) / 1e9;
    if (ms) *ms = t;
    return PACO_OK;
}

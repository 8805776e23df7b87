// FP32 FMA throughput of the current device: the denominator of the "alu"
// rooflines of the path's kernels.  Every thread runs 8 independent FMA chains
// (enough in flight to cover the FMA latency at 8 warps per scheduler), so the
// kernel measures issue-limited FP32 throughput, not latency.
#include <cuda_runtime.h>

#include "cf.h"
#include "cf_internal.cuh"

namespace cf {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace
}  // namespace cf

extern "C" int cf_fp32_peak(double *tflops) {
    if (!tflops) return cf::fail(CF_EINVAL, "tflops is NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cf::cuda_fail(e, "cf_fp32_peak: device query");
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *out = nullptr;
    int rc = CF_ECUDA;
    const int blocks = sms * 8, iters = 1 << 15;
    float ms = 0.f;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess && cudaMallocAsync((void **)&out, sizeof(float) * blocks, st) == cudaSuccess) {
        cf::k_fma_peak<<<blocks, cf::kPeakThreads, 0, st>>>(out, iters, 0.999999f, 1e-7f);  // warm-up
        cudaEventRecord(e0, st);
        cf::k_fma_peak<<<blocks, cf::kPeakThreads, 0, st>>>(out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
            const double flop = 2.0 * cf::kChains * (double)iters * blocks * cf::kPeakThreads;
            *tflops = flop / (ms * 1e-3) / 1e12;
            rc = CF_OK;
        }
        cudaFreeAsync(out, st);
        cudaStreamSynchronize(st);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (rc != CF_OK) return cf::fail(rc, "cf_fp32_peak: the timed FMA launch failed (%s)",
                                     cudaGetErrorString(cudaGetLastError()));
    return rc;
}

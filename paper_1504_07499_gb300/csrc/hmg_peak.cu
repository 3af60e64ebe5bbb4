// FP64 arithmetic rate of the device: the ceiling of the plain FP64 form of the solver,
// whose passes are bound by the FP64 pipe rather than by HBM.  A grid of threads runs
// long chains of dependent fused multiply-adds on eight independent accumulators each (no
// memory traffic in the loop); the rate is 2 flops per FMA over the CUDA-event time.
#include <cuda_runtime.h>

#include "../../include/hmg.h"
#include "hmg_runtime.h"

namespace hmg {
namespace {

constexpr int kAcc = 8;

__global__ void k_dfma(double* out, int iters, double a, double b) {
    double x[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kAcc; ++i) x[i] = fma(x[i], a, b);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += x[i];
    if (s == 12345.678) out[0] = s;   // keeps the chains alive; never true for these inputs
}

}  // namespace
}  // namespace hmg

using namespace hmg;

extern "C" hmg_status hmg_fp64_rate(hmg_ctx* ctx, double* flops_out) {
    g_last_error.clear();
    if (!ctx || !flops_out) {
        set_error("null argument");
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int threads = 256, blocks = 8 * sms, iters = 1 << 14;
    double* out = (double*)ctx->alloc(sizeof(double));
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_dfma<<<blocks, threads, 0, ctx->stream>>>(out, iters, 0.999999, 1e-7);   // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(a, ctx->stream);
        k_dfma<<<blocks, threads, 0, ctx->stream>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(b, ctx->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best) best = ms;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->release(out);
    if (e != cudaSuccess) {
        set_error("FP64 rate kernel: %s", cudaGetErrorString(e));
        return HMG_CUDA_ERROR;
    }
    *flops_out = 2.0 * kAcc * (double)iters * threads * blocks / (best * 1e-3);
    return HMG_OK;
}

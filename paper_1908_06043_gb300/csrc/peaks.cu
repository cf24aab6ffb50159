// Measured arithmetic peaks of this GPU (no paper counterpart): the denominators of the
// roofline fractions the benchmark reports for the CUDA-core kernels.  Each thread runs
// kIlp independent fused multiply-add chains; the grid fills every SM four times over.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.h"

namespace {

constexpr int kIlp = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(long long iters, T a, T b, T *sink) {
    T acc[kIlp];
#pragma unroll
    for (int i = 0; i < kIlp; ++i) acc[i] = (T)(threadIdx.x + i);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kIlp; ++i) acc[i] = acc[i] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kIlp; ++i) s += acc[i];
    if (s == (T)-12345.678) sink[blockIdx.x] = s;   // never true: keeps the chains live
}

template <typename T>
int run_chains(ss_ctx *ctx, long long iters, unsigned grid, void *sink, float *ms) {
    cudaEvent_t e0, e1;
    SS_CUDA_TRY(ctx, cudaEventCreate(&e0));
    SS_CUDA_TRY(ctx, cudaEventCreate(&e1));
    // a * x + b with a slightly below 1 keeps every chain finite for any iteration count
    SS_CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
    ss_launch(ctx, SS_K_MISC, k_fma_chains<T>, grid, 256, 0, ctx->stream, iters, (T)0.999999, (T)1e-7,
              (T *)sink);
    SS_CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
    SS_CUDA_TRY(ctx, cudaEventSynchronize(e1));
    SS_CUDA_TRY(ctx, cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

}  // namespace

extern "C" ss_status ss_measure_peak(ss_ctx *ctx, int32_t kind, double seconds, double *tflops) {
    if (!ctx) return SS_ERR_ARG;
    if (ctx->device < 0 || (kind != SS_PEAK_FP64_FMA && kind != SS_PEAK_FP32_FMA) || !tflops ||
        !(seconds > 0.0 && seconds <= 10.0))
        return ctx->set_error(SS_ERR_ARG, "ss_measure_peak: bad argument or host-only context");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const unsigned grid = (unsigned)ctx->sm_count * 4;
    void *sink = nullptr;
    SS_CUDA_TRY(ctx, cudaMallocAsync(&sink, sizeof(double) * grid, ctx->stream));
    long long iters = 1 << 12;
    float ms = 0.f;
    int rc = SS_OK;
    // grow the chain length until one launch takes the requested time (at most 2^34
    // iterations); the rate of the last launch is reported
    for (int round = 0; round < 24 && rc == SS_OK; ++round) {
        rc = kind == SS_PEAK_FP64_FMA ? run_chains<double>(ctx, iters, grid, sink, &ms)
                                      : run_chains<float>(ctx, iters, grid, sink, &ms);
        if (rc != SS_OK || ms >= 1e3 * seconds || iters >= (1ll << 34)) break;
        const double scale = ms > 0.05f ? 1e3 * seconds / ms : 16.0;
        iters = std::min<long long>(1ll << 34, (long long)(iters * std::min(16.0, std::max(1.1, scale * 1.05))));
    }
    cudaFreeAsync(sink, ctx->stream);
    if (rc != SS_OK) return rc;
    const double flops = 2.0 * kIlp * (double)iters * grid * 256.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return SS_OK;
}

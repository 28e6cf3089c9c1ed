/*
 * yk_peak.cu — FMA-rate microbenchmark (diagnostic; the paper has no counterpart).  Measures the
 * FP64 or FP32 FMA throughput of the device with independent FMA chains, and the rate of the
 * double-float multiply-add that the FP64 path's kernels are built from (df_mul_add and its
 * unnormalised form df_mul_add_lazy of yk_core.h, each counted as 2 FP64-equivalent flops), so
 * that ALU-bound kernels of the evaluator can be reported against a measured peak.
 */
#include <cuda_runtime.h>

#include "yk_internal.h"

namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chains(R *out, int iters, R a, R b)
{
    R x0 = (R)threadIdx.x, x1 = x0 + (R)1, x2 = x0 + (R)2, x3 = x0 + (R)3;
    R x4 = x0 + (R)4, x5 = x0 + (R)5, x6 = x0 + (R)6, x7 = x0 + (R)7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const R s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (R)-12345.678) out[blockIdx.x] = s; /* keep the chains alive */
}

/* double-float multiply-add chains: 8 independent accumulators per thread, acc <- acc + a * b */
template <bool LAZY>
__global__ void __launch_bounds__(256) k_df_chains(float *out, int iters, float ah, float al,
                                                   float bh, float bl)
{
    using yk::df32;
    const df32 a(ah, al), b(bh, bl);
    df32 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = df32((float)(threadIdx.x + k), 0.0f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            x[k] = LAZY ? yk::df_mul_add_lazy(x[k], a, b) : yk::df_mul_add(x[k], x[k], a);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k].hi + x[k].lo;
    if (s == -12345.678f) out[blockIdx.x] = s; /* keep the chains alive */
}

} /* namespace */

extern "C" YK_API yk_status yk_fma_peak(int precision, double *tflops)
{
    if (!tflops) return YK_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return YK_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return YK_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    if (precision < YK_FP64 || precision > YK_PEAK_DF_LAZY) return YK_ERR_ARG;
    const int iters = precision == YK_FP64 ? 4096 : precision == YK_FP32C ? 65536 : 8192;
    void *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) return YK_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        if (precision == YK_FP64)
            k_fma_chains<double><<<blocks, threads>>>((double *)out, iters, 0.999999, 1e-7);
        else if (precision == YK_FP32C)
            k_fma_chains<float><<<blocks, threads>>>((float *)out, iters, 0.999999f, 1e-7f);
        else if (precision == YK_PEAK_DF)
            /* x <- x + x * a with a ~ 1e-7: the chain stays bounded */
            k_df_chains<false><<<blocks, threads>>>((float *)out, iters, 1e-7f, 1e-15f, 0.0f, 0.0f);
        else
            k_df_chains<true><<<blocks, threads>>>((float *)out, iters, 0.5f, 1e-9f, 1e-7f, 1e-15f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms; /* first launch is a warm-up */
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return YK_ERR_CUDA;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return YK_OK;
}

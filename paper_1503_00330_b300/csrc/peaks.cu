// peaks.cu -- measured issue rates of the pipes the kernels lean on: packed
// FP32 FMA (FFMA2) and the MUFU base-2 exponential (the FP32 rollout), and
// FP64 FMA (the cost-to-go scan).  Every SM runs enough warps of independent
// dependency chains to saturate the pipe; the rates come from CUDA-event time.
// They are context for the rooflines (the FP32 denominator is the unit-count
// peak), not part of any update.
#include <cuda_runtime.h>

#include "pi2rh.h"
#include "pi2rh_ctx.h"

namespace {

constexpr int NT = 256;
constexpr int CHAINS = 8;

__global__ void __launch_bounds__(NT) ffma2_chains(int iters, float seed, float *sink)
{
    float2 acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = make_float2(seed + c, seed - c);
    const float2 m = make_float2(0.999999f, 0.999998f), a = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = __ffma2_rn(acc[c], m, a);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c].x + acc[c].y;
    if (s == 12345.678f) *sink = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(NT) ex2_chains(int iters, float seed, float *sink)
{
    float v[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = -0.5f - 0.01f * c - seed;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) v[c] = -pi2rh::ex2(v[c]);   // stays in (-1, 0)
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += v[c];
    if (s == 12345.678f) *sink = s;
}

__global__ void __launch_bounds__(NT) dfma_chains(int iters, double seed, double *sink)
{
    double acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = seed + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], 0.9999999999, 1e-12);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    if (s == 12345.678) *sink = s;
}

int rc_of(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PI_OK;
    return pi2rh_fail(e == cudaErrorMemoryAllocation ? PI_ERR_OOM : PI_ERR_CUDA, what);
}

}  // namespace

extern "C" int pi_debug_pipe_rates(int device, double *ffma_tflops, double *ex2_per_s)
{
    if (!ffma_tflops || !ex2_per_s) return pi2rh_fail(PI_ERR_INVALID_ARG, "NULL output");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return pi2rh_fail(PI_ERR_CUDA, "cudaSetDevice");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = rc_of(cudaMalloc(&sink, sizeof(float)), "probe buffer");
    if (!rc) rc = rc_of(cudaEventCreate(&e0), "event");
    if (!rc) rc = rc_of(cudaEventCreate(&e1), "event");
    const int blocks = sms * 8;   // 64 warps per SM
    const int fma_iters = 1 << 14, ex2_iters = 1 << 12;
    float ms = 0.0f;
    if (!rc) {
        ffma2_chains<<<blocks, NT>>>(256, 1.0f, sink);   // warm-up
        cudaEventRecord(e0);
        ffma2_chains<<<blocks, NT>>>(fma_iters, 1.0f, sink);
        cudaEventRecord(e1);
        rc = rc_of(cudaEventSynchronize(e1), "FFMA2 probe");
    }
    if (!rc) {
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = (double)blocks * NT * fma_iters * CHAINS * 4.0;   // FFMA2 = 2 FMA = 4 flop
        *ffma_tflops = flops / (ms * 1e-3) / 1e12;
        ex2_chains<<<blocks, NT>>>(64, 0.1f, sink);
        cudaEventRecord(e0);
        ex2_chains<<<blocks, NT>>>(ex2_iters, 0.1f, sink);
        cudaEventRecord(e1);
        rc = rc_of(cudaEventSynchronize(e1), "ex2 probe");
    }
    if (!rc) {
        cudaEventElapsedTime(&ms, e0, e1);
        *ex2_per_s = (double)blocks * NT * ex2_iters * CHAINS / (ms * 1e-3);
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}

extern "C" int pi_debug_fp64_rate(int device, double *dfma_per_s)
{
    if (!dfma_per_s) return pi2rh_fail(PI_ERR_INVALID_ARG, "NULL output");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return pi2rh_fail(PI_ERR_CUDA, "cudaSetDevice");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = rc_of(cudaMalloc(&sink, sizeof(double)), "probe buffer");
    if (!rc) rc = rc_of(cudaEventCreate(&e0), "event");
    if (!rc) rc = rc_of(cudaEventCreate(&e1), "event");
    const int blocks = sms * 8;   // 64 warps per SM
    const int iters = 1 << 10;
    float ms = 0.0f;
    if (!rc) {
        dfma_chains<<<blocks, NT>>>(16, 1.0, sink);   // warm-up
        cudaEventRecord(e0);
        dfma_chains<<<blocks, NT>>>(iters, 1.0, sink);
        cudaEventRecord(e1);
        rc = rc_of(cudaEventSynchronize(e1), "DFMA probe");
    }
    if (!rc) {
        cudaEventElapsedTime(&ms, e0, e1);
        *dfma_per_s = (double)blocks * NT * iters * CHAINS / (ms * 1e-3);
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}

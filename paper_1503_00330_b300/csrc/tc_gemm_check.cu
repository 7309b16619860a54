// tc_gemm_check.cu -- staged check of the tensor-core GEMM core used by the
// tensor-core rollout form: one CTA computes D[128 x 64] = A[128 x K] B[64 x K]^T
// with fp16 operands in the K-major core-matrix shared-memory layout, fp32
// accumulation in tensor memory (tcgen05.mma, kind::f16), read back with
// tcgen05.ld.  Exposed as pi_debug_tc_gemm so the operand descriptors and the
// TMEM handling are verified on their own against a host product.
#include <cuda_fp16.h>

#include "pi2rh_kernels.h"
#include "tc_ptx.cuh"

namespace pi2rh {

namespace {

constexpr int GM = 128, GN = 64, GKMAX = 160;
constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + GM * GKMAX * 2;          // 40960
constexpr int OFF_BAR = OFF_B + GN * GKMAX * 2;        // 61440
constexpr int OFF_SLOT = OFF_BAR + 8;
constexpr int OFF_ABORT = OFF_SLOT + 8;
constexpr int GEMM_SMEM = OFF_ABORT + 16;

__global__ void __launch_bounds__(128, 1) tc_gemm_check_kernel(const __half *__restrict__ A,
                                                               const __half *__restrict__ B, int K,
                                                               float *__restrict__ D, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + OFF_SLOT);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + OFF_ABORT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < GM * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        *reinterpret_cast<__half *>(smem + OFF_A + kmajor_offset(r, k, K)) = A[i];
    }
    for (int i = tid; i < GN * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        *reinterpret_cast<__half *>(smem + OFF_B + kmajor_offset(r, k, K)) = B[i];
    }
    if (warp == 0) {
        tmem_alloc(slot, GN);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *slot;

    if (tid == 0) {
        const uint32_t idesc = idesc_f16_f32(GM, GN);
        const uint32_t a0 = smem_u32(smem + OFF_A), b0 = smem_u32(smem + OFF_B);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = smem_desc_kmajor(a0 + ks * 256, 128, 16 * K);
            const uint64_t bd = smem_desc_kmajor(b0 + ks * 256, 128, 16 * K);
            mma_f16(tbase, ad, bd, idesc, ks > 0);
        }
        mma_commit(bar);
    }
    __syncwarp();
    if (!mbar_wait_bounded(bar, 0, abort_flag)) {
        if (lane == 0) atomicOr(err, DEVERR_TIMEOUT_FULL);
        mbar_wait_drain(bar, 0);      // the MMAs may still be writing TMEM
    }
    tc_fence_after();
#pragma unroll
    for (int c = 0; c < GN / 16; ++c) {
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c * 16, v);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) D[(size_t)(warp * 32 + lane) * GN + c * 16 + i] = v[i];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, GN);
}

bool g_gemm_attr = false;

}  // namespace

cudaError_t launch_tc_gemm_check(const void *A, const void *B, int K, float *D, int *err, cudaStream_t s)
{
    if (K < 16 || K > GKMAX || K % 16) return cudaErrorInvalidValue;
    if (!g_gemm_attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_check_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GEMM_SMEM);
        if (e != cudaSuccess) return e;
        g_gemm_attr = true;
    }
    tc_gemm_check_kernel<<<1, 128, GEMM_SMEM, s>>>(static_cast<const __half *>(A), static_cast<const __half *>(B),
                                                    K, D, err);
    return cudaGetLastError();
}

}  // namespace pi2rh

// tc_ptx.cuh -- inline-PTX wrappers for the 5th-generation tensor cores
// (tcgen05: MMA into tensor memory, TMEM allocation, TMEM loads) and the
// shared-memory operand descriptors they read, for sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pi2rh_device.cuh"

namespace pi2rh {

// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor (64 bit) for K-major operands without
// swizzling.  The operand is tiled in "core matrices" of 8 rows x 16 bytes
// (8 x 8 fp16), each stored as 128 contiguous bytes (row r at +16 r).
//   start   byte address of the first core matrix            bits  0-13 (>>4)
//   lbo     byte distance between core matrices adjacent in K bits 16-29 (>>4)
//   sbo     byte distance between core matrices adjacent in
//           the M/N (row) direction                          bits 32-45 (>>4)
//   bits 46-47 = 1 (descriptor version), base offset 0, no swizzle (bits 61-63 = 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor for kind::f16 with fp16 A and B, fp32 accumulator,
// both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N)
{
    return (1u << 4)                          // D format: f32
           | (0u << 7) | (0u << 10)           // A, B format: f16
           | (0u << 15) | (0u << 16)          // A, B K-major
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

// Byte offset of element (r, k) of a K-major fp16 tile with `kdim` columns in
// the core-matrix layout above (lbo = 128, sbo = 16 * kdim).
__host__ __device__ constexpr uint32_t kmajor_offset(int r, int k, int kdim)
{
    return (uint32_t)((r >> 3) * (16 * kdim) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// ---------------------------------------------------------------------------
// TMEM allocation (one full warp executes these).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_result, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_result)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// MMA: D[tmem] (+)= A[smem] x B[smem]^T, issued by one thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// The three MMAs of one K step of the split-precision product,
//   D (+)= A_hi B_hi + A_hi B_lo + A_lo B_hi,
// executed by a whole converged warp and issued by the one lane that
// elect.sync picks (the same lane on every call with all lanes active).  The
// first MMA overwrites D when acc_first is 0.
__device__ __forceinline__ void mma3_elect(uint32_t d_tmem, uint64_t a_hi, uint64_t a_lo, uint64_t b_hi,
                                           uint64_t b_lo, uint32_t idesc, uint32_t acc_first)
{
    asm volatile(
        "{\n\t.reg .pred p, t, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.u32 p, %6, 0;\n\t"
        "setp.eq.u32 t, %6, %6;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %5, p;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %5, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %5, t;\n\t}" ::"r"(d_tmem),
        "l"(a_hi), "l"(a_lo), "l"(b_hi), "l"(b_lo), "r"(idesc), "r"(acc_first)
        : "memory");
}

// Two of the split products of one K step, D += A_hi B_hi + A_hi B_lo (the
// A operand at its fp16 rounding, the B operand split), issued like mma3_elect;
// always accumulates.
__device__ __forceinline__ void mma2_elect(uint32_t d_tmem, uint64_t a_hi, uint64_t b_hi, uint64_t b_lo,
                                           uint32_t idesc)
{
    asm volatile(
        "{\n\t.reg .pred t, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.eq.u32 t, %4, %4;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %4, t;\n\t}" ::"r"(d_tmem),
        "l"(a_hi), "l"(b_hi), "l"(b_lo), "r"(idesc)
        : "memory");
}

// tcgen05.commit from the lane elect.sync picks (the lane that issued the
// MMAs of mma3_elect): arrives on the mbarrier once they complete.
__device__ __forceinline__ void commit_elect(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

// Arrives on an mbarrier once all prior tcgen05 async operations of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Makes generic-proxy shared-memory writes visible to the async proxy (MMA operands).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// TMEM -> registers: each thread of the warp reads its lane (32 lanes per
// warp quarter) and 16 consecutive 32-bit columns starting at taddr.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Two 16-column loads and the wait in one asm statement, so that no use of
// the destination registers can be scheduled before the loads have landed.
__device__ __forceinline__ void tmem_ld16x2_wait(uint32_t ta, uint32_t tb, float (&va)[16], float (&vb)[16])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        va[i] = __uint_as_float(r[i]);
        vb[i] = __uint_as_float(r[16 + i]);
    }
}

}  // namespace pi2rh

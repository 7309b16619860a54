// pi2rh_device.cuh -- device-side building blocks shared by the kernels of the
// PI^2-RH / LWPR library: counter-based noise, the cost function, the packed
// LWPR field-pair record, mbarrier / bulk-copy (1-D TMA) primitives with
// bounded waits, and the device error word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pi2rh {

constexpr int NX = 12, NU = 4, NZ = 16, NY = 12;

// ---------------------------------------------------------------------------
// Device error word (bit flags), read and cleared by pi_sync.
// ---------------------------------------------------------------------------
constexpr int DEVERR_TIMEOUT_FULL = 1;   // consumer waited too long for a stage
constexpr int DEVERR_TIMEOUT_EMPTY = 2;  // producer waited too long for a free slot
constexpr int DEVERR_TIMEOUT_DRAIN = 4;  // copies still in flight at exit
constexpr int DEVERR_BAD_CONFIG = 8;     // launch configuration inconsistent
constexpr int DEVERR_TIMEOUT_PEER = 16;  // a CTA waited too long for another CTA's step (split launch)

// Upper bound on any single device-side wait (nanoseconds of %globaltimer).
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

// ---------------------------------------------------------------------------
// Packed LWPR record: two receptive fields of the same output side by side
// (float2 = {field 2p, field 2p+1}), so that the per-field arithmetic runs on
// the packed FP32x2 FMA datapath.  Quadratic-form coefficients are stored in
// the base-2 exponent domain: s = bias + sum_i d_i sum_{j>=i} A_ij d_j equals
// -(1/2) log2(e) (z-c)^T D (z-c), with A_ii = -k D_ii, A_ij = -k (D_ij + D_ji),
// k = log2(e)/2, and d = z - c.
// ---------------------------------------------------------------------------
constexpr int REC_NEGC = 0;      // 16 entries: -c
constexpr int REC_A = 16;        // 136 entries: upper triangle of A, row-major
constexpr int REC_BETA = 152;    // 16 entries: beta
constexpr int REC_B = 168;       // b (value of the local model at its center)
constexpr int REC_VAR = 169;     // sigma_j^2
constexpr int REC_BIAS = 170;    // 0 for a real field, -inf for padding
constexpr int REC_LEN = 172;     // float2 entries per record (1376 bytes)
constexpr int REC_BYTES = REC_LEN * 8;
static_assert(REC_BYTES % 16 == 0, "bulk copies need 16-byte multiples");

// Offset of entry (i, j >= i) of the upper triangle, row-major.
__host__ __device__ constexpr int tri_index(int i, int j) { return i * NZ - (i * (i - 1)) / 2 + (j - i); }

// ---------------------------------------------------------------------------
// Cost parameters as seen by the kernels (copied by value into the launch).
// ---------------------------------------------------------------------------
struct CostDev {
    float goal[3];
    float Q_pos[3];
    float Q_vel, Q_ang, w_obs, obs_sharp, radius, w_crash, w_var, w_T;
    int obs_kind, n_obs;
    const float2 *obs;   // device [n_obs]
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// published definition: per round, two 32x32 -> 64-bit products of counter
// words 0 and 2 with the round multipliers; the key advances by the Weyl
// increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0 = __umulhi(mul0, c.x), lo0 = mul0 * c.x;
        uint32_t hi1 = __umulhi(mul1, c.z), lo1 = mul1 * c.z;
        uint4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += weyl0;
        k1 += weyl1;
    }
    return c;
}

__device__ __forceinline__ uint4 noise_block(uint64_t seed, uint32_t k, uint32_t t, uint32_t blk,
                                             uint32_t m)
{
    return philox4x32_10(make_uint4(k, t, blk, m), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform in (0, 1): odd multiples of 2^-24, exact in FP32.
__device__ __forceinline__ float uniform24(uint32_t r)
{
    return (float)(2u * (r >> 9) + 1u) * 0x1p-24f;
}

// Box-Muller on (u0, u1) and (u2, u3).
__device__ __forceinline__ float4 box_muller4(uint4 r)
{
    float u0 = uniform24(r.x), u1 = uniform24(r.y), u2 = uniform24(r.z), u3 = uniform24(r.w);
    float ra = sqrtf(-2.0f * logf(u0)), rb = sqrtf(-2.0f * logf(u2));
    float sa, ca, sb, cb;
    sincospif(2.0f * u1, &sa, &ca);
    sincospif(2.0f * u3, &sb, &cb);
    return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

// ---------------------------------------------------------------------------
// Cost (Sec. 5 form).  The obstacle indicator is an integer decision made in
// FP32 with separately rounded operations (no contraction).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int inside_any(const CostDev &C, const float2 *obs_s, float px, float py)
{
    float r2 = __fmul_rn(C.radius, C.radius);
    int inside = 0;
    for (int i = 0; i < C.n_obs; ++i) {
        float2 o = obs_s[i];
        float dx = __fsub_rn(px, o.x), dy = __fsub_rn(py, o.y);
        float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        inside |= (d2 < r2) ? 1 : 0;
    }
    return inside;
}

__device__ __forceinline__ float running_cost(const CostDev &C, const float2 *obs_s, const float *x,
                                              const float *var)
{
    float q = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float e = x[d] - C.goal[d];
        q = fmaf(C.Q_pos[d] * e, e, q);
    }
    float v2 = x[3] * x[3] + x[4] * x[4] + x[5] * x[5];
    float a2 = x[6] * x[6] + x[7] * x[7] + x[8] * x[8];
    q = fmaf(C.Q_vel, v2, q);
    q = fmaf(C.Q_ang, a2, q);
    int inside = inside_any(C, obs_s, x[0], x[1]);
    if (C.obs_kind == 0) {
        q += inside ? C.w_obs : 0.0f;
    } else {
        float bump = 0.0f;
        for (int i = 0; i < C.n_obs; ++i) {
            float2 o = obs_s[i];
            float dx = x[0] - o.x, dy = x[1] - o.y;
            bump += expf(-C.obs_sharp * (dx * dx + dy * dy));
        }
        q = fmaf(C.w_obs, bump, q);
    }
    q += inside ? C.w_crash : 0.0f;
    float vs = 0.0f;
#pragma unroll
    for (int o = 0; o < NY; ++o) vs += var[o];
    return fmaf(C.w_var, vs, q);
}

__device__ __forceinline__ float terminal_cost(const CostDev &C, const float *x)
{
    float phi = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float e = x[d] - C.goal[d];
        phi = fmaf(C.Q_pos[d] * e, e, phi);
    }
    return C.w_T * phi;
}

// ---------------------------------------------------------------------------
// Base-2 exponential on the MUFU unit (ex2.approx, ftz): 2^x, 2^-inf = +0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk asynchronous copy (1-D TMA) primitives.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity to complete.  Gives up (returns
// false) when *abort is set or after WAIT_LIMIT_NS.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  volatile int *abort,
                                                  unsigned long long limit_ns = WAIT_LIMIT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31u) == 0u) {
            if (*abort) return false;
            if (globaltimer() - t0 > limit_ns) return false;
        }
    }
}

// True in the one lane of a converged warp that elect.sync picks.
__device__ __forceinline__ bool elect_one()
{
    uint32_t e;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(e));
    return e != 0;
}

// Bounded wait with no abort check (used to drain copies at exit).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t *bar, uint32_t parity)
{
    unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31u) == 31u && globaltimer() - t0 > WAIT_LIMIT_NS) return false;
    }
}

// Global -> shared bulk copy completing on an mbarrier (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Arrival (without waiting) at named barrier `id`, whose instance counts
// `count` threads in all (those that arrive and those that sync).
__device__ __forceinline__ void named_bar_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier over `count` threads (multiple of 32), id 1..15.
__device__ __forceinline__ void named_bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier that also returns the OR of `pred` over the participants.
__device__ __forceinline__ bool bar_sync_or(int id, int count, bool pred)
{
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return out != 0;
}

// ---------------------------------------------------------------------------
// Thread-block cluster primitives (distributed shared memory).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_size()
{
    uint32_t n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(const void *p, uint32_t rank)
{
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
    return a;
}

__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Arrive (release, cluster scope) on an mbarrier of another CTA of the cluster.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_wait_bounded, with acquire at cluster scope (the arrivals come from
// other CTAs of the cluster, after their distributed shared-memory stores).
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try_wait_cluster(bar, parity)) return true;
    unsigned long long t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 31u) == 0u) {
            if (*abort) return false;
            if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
        }
    }
}

// Every thread of every CTA of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

}  // namespace pi2rh

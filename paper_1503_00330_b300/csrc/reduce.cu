// reduce.cu -- cost-to-go scan and the per-timestep weighted average (Eq. 2).
//
// scan_lse_kernel: one CTA per RS_KC = 64 rollouts.  The timesteps are walked
// from T-1 down to 0 in chunks of TC, through a two-deep shared-memory buffer:
// - producer warps 0-1, one thread per rollout, prefetch the next chunk's
//   costs and extend the suffix sum S_{k,i} = phi_k + dt sum_{j>=i} q_{k,j}
//   in FP64 (Sec. 3.1), serially from T-1 down;
// - consumer warps 2-7 take whole timesteps of the previous chunk (their eps
//   loaded before they wait) and form, over the CTA's 64 rollouts, the
//   log-sum-exp partial
//     m_c = min_k S,  Z_c = sum_k 2^((m_c - S) log2(e)/lambda),
//     V_c = sum_k 2^(...) eps_k
// (exponent in FP64; exponential, the 2-term lane sums and the pairwise warp
// sums in FP32; each partial row is 6 doubles wide: m_c as a double, then Z_c
// and V_c as five floats, widened to FP64 by the merge).  The halves hand chunks over through
// named barriers (full / empty per buffer).  cost and eps are read once,
// coalesced and vectorised ([T][K] layout, eps as float4).  costs_out[k] = S_{k,0}.
// B300 runs FP64 at about 2 lanes per clock per SM, 1/64 of FP32, so the
// kernel keeps FP64 to the suffix sum (convert + FMA) and the exponent
// (subtract, multiply, convert) -- five FP64-pipe instructions per
// rollout-step: the exact minimum over the rollouts is taken on integer keys
// of the doubles (warp redux), and the FP32 sums are stored as they are (a
// conversion by lane 0 alone still holds the FP64 pipe for a whole warp).
//
// lse_merge_kernel: one warp per timestep (one warp per CTA, so that the FP64
// exponentials spread over T SMs) merges the per-CTA partials in a fixed order
// (deterministic) in FP64 and writes u_out = u_nom + V / Z.
#include "pi2rh_kernels.h"

namespace pi2rh {

namespace {

constexpr int KC = RS_KC;
constexpr int TC = 32;
constexpr int NT = 256;

__device__ __forceinline__ double warp_min_d(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Order-preserving unsigned key of a double (not NaN): the smaller key is the
// smaller value, so a minimum over keys is the exact minimum of the values.
__device__ __forceinline__ unsigned long long dkey(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double dkey_value(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

// Exact minimum over a warp of one key per lane: the minimum high word, then
// the minimum low word among the lanes holding it (integer warp reductions).
__device__ __forceinline__ double warp_min_key(unsigned long long k)
{
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? lo : 0xffffffffu);
    return dkey_value(((unsigned long long)mhi << 32) | mlo);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Pairwise (5-level butterfly) sum over a warp in FP32: at most 5 roundings.
__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Named barriers of the scan's two-deep buffer (compile-time ids): full[b]
// (producers arrive, consumers wait) and empty[b] (the other way round).
__device__ __forceinline__ void scan_full_arrive(int b)
{
    if (b) named_bar_arrive(2, NT);
    else named_bar_arrive(1, NT);
}
__device__ __forceinline__ void scan_full_wait(int b)
{
    if (b) named_bar_sync(2, NT);
    else named_bar_sync(1, NT);
}
__device__ __forceinline__ void scan_empty_arrive(int b)
{
    if (b) named_bar_arrive(4, NT);
    else named_bar_arrive(3, NT);
}
__device__ __forceinline__ void scan_empty_wait(int b)
{
    if (b) named_bar_sync(4, NT);
    else named_bar_sync(3, NT);
}

__device__ __forceinline__ void scan_lse_block(const float *__restrict__ cost_tk, const float *__restrict__ phi,
                                               const float4 *__restrict__ eps_tk, int K, int T, double dt,
                                               double inv_lam_log2e, float *__restrict__ costs_out,
                                               double *__restrict__ part, int blk)
{
    constexpr int NPROD = KC;                 // producer threads (warps 0-1)
    constexpr int NCW = (NT - NPROD) / 32;    // consumer warps
    __shared__ double S_s[2][TC][KC];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k0 = blk * KC;
    const int nchunk = (T + TC - 1) / TC;     // chunk c covers [max(T - (c+1) TC, 0), T - c TC)
    if (tid < NPROD) {
        const int k = k0 + tid;
        double acc = k < K ? (double)phi[k] : 0.0;
        float cb[TC];
        auto load_chunk = [&](int c) {
            const int hi = T - c * TC, lo = hi > TC ? hi - TC : 0;
#pragma unroll
            for (int r = 0; r < TC; ++r) {
                const int i = hi - 1 - r;
                cb[r] = (k < K && i >= lo) ? cost_tk[(size_t)i * K + k] : 0.0f;
            }
        };
        load_chunk(0);
        for (int c = 0; c < nchunk; ++c) {
            const int b = c & 1;
            const int hi = T - c * TC, lo = hi > TC ? hi - TC : 0;
            float cur[TC];
#pragma unroll
            for (int r = 0; r < TC; ++r) cur[r] = cb[r];
            if (c + 1 < nchunk) load_chunk(c + 1);   // in flight while this chunk is summed
            if (c >= 2) scan_empty_wait(b);   // the consumers are done with buffer b
            // the chunk's costs, summed backwards in FP64 in the same order as ever
#pragma unroll
            for (int r = 0; r < TC; ++r) {
                const int i = hi - 1 - r;
                if (i >= lo) {
                    double s = INFINITY;
                    if (k < K) {
                        acc += (double)cur[r] * dt;
                        s = acc;
                    }
                    S_s[b][i - lo][tid] = s;
                }
            }
            if (lo == 0 && k < K) costs_out[k] = (float)acc;
            scan_full_arrive(b);
        }
        // the last one or two buffers: wait for their consumers before leaving
        for (int c = nchunk > 2 ? nchunk - 2 : 0; c < nchunk; ++c) scan_empty_wait(c & 1);
        return;
    }
    const int cw = warp - NPROD / 32;          // consumer warp 0..NCW-1
    constexpr int RPW = (TC + NCW - 1) / NCW;  // rows per consumer warp and chunk
    const int ka = k0 + lane, kb = k0 + lane + 32;
    for (int c = 0; c < nchunk; ++c) {
        const int b = c & 1;
        const int hi = T - c * TC, lo = hi > TC ? hi - TC : 0;
        // this warp's timesteps of the chunk: rows cw, cw + NCW, ...; their eps first
        float4 ea[RPW], eb[RPW];
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
            const int r = cw + u * NCW, i = lo + r;
            const bool ok = r < hi - lo;
            ea[u] = ok && ka < K ? eps_tk[(size_t)i * K + ka] : make_float4(0.f, 0.f, 0.f, 0.f);
            eb[u] = ok && kb < K ? eps_tk[(size_t)i * K + kb] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        scan_full_wait(b);
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
            const int r = cw + u * NCW, i = lo + r;
            if (r >= hi - lo) break;
            const double sa = S_s[b][r][lane], sb = S_s[b][r][lane + 32];
            // exact minimum (a rounded shift can put exponents hundreds of
            // binary orders off when S is large and lambda small), on keys
            const unsigned long long ka2 = dkey(sa), kb2 = dkey(sb);
            const double mn = warp_min_key(ka2 < kb2 ? ka2 : kb2);
            const float wa = exp2f((float)((mn - sa) * inv_lam_log2e));
            const float wb = exp2f((float)((mn - sb) * inv_lam_log2e));
            // the 64 rollouts' FP32 terms are summed by a pairwise warp tree in
            // FP32 (B300 has little FP64 throughput); the partials are stored
            // and merged over K in FP64
            const float4 xa = ea[u], xb = eb[u];
            const float z = warp_sum_f(wa + wb);
            const float v0 = warp_sum_f(fmaf(wa, xa.x, wb * xb.x));
            const float v1 = warp_sum_f(fmaf(wa, xa.y, wb * xb.y));
            const float v2 = warp_sum_f(fmaf(wa, xa.z, wb * xb.z));
            const float v3 = warp_sum_f(fmaf(wa, xa.w, wb * xb.w));
            if (lane == 0) {
                // the minimum as a double, the five FP32 sums as floats (the
                // merge widens them, exactly): no conversion on the FP64 pipe here
                double *p = part + ((size_t)blk * T + i) * 6;
                float *pf = reinterpret_cast<float *>(p + 1);
                p[0] = mn;
                pf[0] = z;
                pf[1] = v0;
                pf[2] = v1;
                pf[3] = v2;
                pf[4] = v3;
            }
        }
        scan_empty_arrive(b);
    }
}

__global__ void __launch_bounds__(NT) scan_lse_kernel(const float *__restrict__ cost_tk,
                                                      const float *__restrict__ phi,
                                                      const float4 *__restrict__ eps_tk, int K, int T,
                                                      double dt, double inv_lam_log2e,
                                                      float *__restrict__ costs_out,
                                                      double *__restrict__ part)
{
    scan_lse_block(cost_tk, phi, eps_tk, K, T, dt, inv_lam_log2e, costs_out, part, blockIdx.x);
}

// Batched: block b handles item items[b] = (controller, rollout block).
__global__ void __launch_bounds__(NT) scan_lse_batch_kernel(const ReduceArgs *__restrict__ args,
                                                            const int2 *__restrict__ items)
{
    const int2 it = items[blockIdx.x];
    const ReduceArgs &r = args[it.x];
    scan_lse_block(r.cost_tk, r.phi, r.eps_tk, r.K, r.T, r.dt, r.inv_lam_log2e, r.costs_out, r.part, it.y);
}

__device__ __forceinline__ void lse_merge_warp(const double *__restrict__ part, int nblk, int T, double inv_lam_log2e,
                                               const float *u_nom, float *u_out, int i)
{
    const int lane = threadIdx.x & 31;
    if (i >= T) return;
    double mn = INFINITY;
    for (int c = lane; c < nblk; c += 32) mn = fmin(mn, part[((size_t)c * T + i) * 6]);
    mn = warp_min_d(mn);
    double z = 0.0, v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = lane; c < nblk; c += 32) {
        const double *p = part + ((size_t)c * T + i) * 6;
        const float *pf = reinterpret_cast<const float *>(p + 1);
        const double sc = exp2((mn - p[0]) * inv_lam_log2e);
        z = fma((double)pf[0], sc, z);
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = fma((double)pf[1 + a], sc, v[a]);
    }
    z = warp_sum_d(z);
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = warp_sum_d(v[a]);
    if (lane < 4) {
        const double va = lane == 0 ? v[0] : lane == 1 ? v[1] : lane == 2 ? v[2] : v[3];
        u_out[(size_t)i * 4 + lane] = (float)((double)u_nom[(size_t)i * 4 + lane] + va / z);
    }
}

__global__ void __launch_bounds__(256) lse_merge_kernel(const double *__restrict__ part, int nblk, int T,
                                                        double inv_lam_log2e, const float *u_nom, float *u_out)
{
    lse_merge_warp(part, nblk, T, inv_lam_log2e, u_nom, u_out, blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
}

// Batched: block b handles 8 timesteps of controller items[b].x starting at items[b].y.
__global__ void __launch_bounds__(256) lse_merge_batch_kernel(const ReduceArgs *__restrict__ args,
                                                              const int2 *__restrict__ items)
{
    const int2 it = items[blockIdx.x];
    const ReduceArgs &r = args[it.x];
    lse_merge_warp(r.part, (r.K + KC - 1) / KC, r.T, r.inv_lam_log2e, r.u_nom, r.u_out, it.y + (threadIdx.x >> 5));
}

__global__ void noise_raw_kernel(uint64_t seed, int K, int T, int m, uint4 *raw)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)K * T) return;
    const int k = (int)(idx / T), t = (int)(idx % T);
    for (int blk = 0; blk < 4; ++blk)
        raw[idx * 4 + blk] = noise_block(seed, (uint32_t)k, (uint32_t)t, (uint32_t)blk,
                                         blk == 0 ? 0u : (uint32_t)m);
}

__global__ void noise_normals_kernel(uint64_t seed, int K, int T, int m, float4 *ctrl, float4 *model)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)K * T) return;
    const int k = (int)(idx / T), t = (int)(idx % T);
    ctrl[idx] = box_muller4(noise_block(seed, (uint32_t)k, (uint32_t)t, 0u, 0u));
    for (int blk = 1; blk < 4; ++blk)
        model[idx * 3 + blk - 1] =
            box_muller4(noise_block(seed, (uint32_t)k, (uint32_t)t, (uint32_t)blk, (uint32_t)m));
}

// One bounded wait on an mbarrier that no thread ever arrives at: the wait
// gives up after limit_ns, the kernel flags the timeout in the error word and
// returns (the failure path of every device-side wait, without a fault).
__global__ void wait_timeout_kernel(int *err, unsigned long long limit_ns)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, &abort_flag, limit_ns)) atomicOr(err, DEVERR_TIMEOUT_FULL);
}

}  // namespace

cudaError_t launch_wait_timeout(int *err, unsigned long long limit_ns, cudaStream_t s)
{
    wait_timeout_kernel<<<1, 32, 0, s>>>(err, limit_ns);
    return cudaGetLastError();
}

int scan_blocks(int K) { return (K + KC - 1) / KC; }

cudaError_t launch_scan_lse(const float *cost_tk, const float *phi, const float4 *eps_tk, int K,
                            int T, float dt, double inv_lam_log2e, float *costs_out, double *part,
                            cudaStream_t s)
{
    scan_lse_kernel<<<scan_blocks(K), NT, 0, s>>>(cost_tk, phi, eps_tk, K, T, (double)dt,
                                                  inv_lam_log2e, costs_out, part);
    return cudaGetLastError();
}

cudaError_t launch_lse_merge(const double *part, int nblk, int T, double inv_lam_log2e,
                             const float *u_nom, float *u_out, cudaStream_t s)
{
    // one warp per CTA: the FP64 exponentials of the merge spread over T SMs
    lse_merge_kernel<<<T, 32, 0, s>>>(part, nblk, T, inv_lam_log2e, u_nom, u_out);
    return cudaGetLastError();
}

cudaError_t launch_scan_lse_batch(const ReduceArgs *args, const int2 *items, int n_items, cudaStream_t s)
{
    if (n_items <= 0) return cudaErrorInvalidValue;
    scan_lse_batch_kernel<<<n_items, NT, 0, s>>>(args, items);
    return cudaGetLastError();
}

cudaError_t launch_lse_merge_batch(const ReduceArgs *args, const int2 *items, int n_items, cudaStream_t s)
{
    if (n_items <= 0) return cudaErrorInvalidValue;
    lse_merge_batch_kernel<<<n_items, 256, 0, s>>>(args, items);
    return cudaGetLastError();
}

cudaError_t launch_noise_raw(uint64_t seed, int K, int T, int m, uint32_t *raw, cudaStream_t s)
{
    const long long n = (long long)K * T;
    noise_raw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, K, T, m,
                                                                 reinterpret_cast<uint4 *>(raw));
    return cudaGetLastError();
}

cudaError_t launch_noise_normals(uint64_t seed, int K, int T, int m, float *ctrl, float *model,
                                 cudaStream_t s)
{
    const long long n = (long long)K * T;
    noise_normals_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        seed, K, T, m, reinterpret_cast<float4 *>(ctrl), reinterpret_cast<float4 *>(model));
    return cudaGetLastError();
}

}  // namespace pi2rh

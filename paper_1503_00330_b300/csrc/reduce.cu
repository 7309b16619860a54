// reduce.cu -- cost-to-go scan and the per-timestep weighted average (Eq. 2).
//
// scan_lse_kernel: one CTA per RS_KC = 64 rollouts.  The timesteps are walked
// from T-1 down to 0 in chunks of TC: one thread per rollout loads the chunk's
// costs (all loads in flight at once), extends its suffix sum
// S_{k,i} = phi_k + dt sum_{j>=i} q_{k,j} in FP64 (Sec. 3.1) and parks the
// chunk in shared memory; then each warp takes whole timesteps of the chunk
// (their eps loaded up front) and forms, over the CTA's 64 rollouts, the log-sum-exp partial
//     m_c = min_k S,  Z_c = sum_k 2^((m_c - S) log2(e)/lambda),
//     V_c = sum_k 2^(...) eps_k
// (exponent in FP64; exponential, the 2-term lane sums and the pairwise warp
// sums in FP32; partials stored in FP64).  cost and eps are read once, coalesced and vectorised ([T][K]
// layout, eps as float4).  costs_out[k] = S_{k,0}.
//
// lse_merge_kernel: one warp per timestep merges the per-CTA partials in a
// fixed order (deterministic) in FP64 and writes u_out = u_nom + V / Z.
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

__device__ __forceinline__ void scan_lse_block(const float *__restrict__ cost_tk, const float *__restrict__ phi,
                                               const float4 *__restrict__ eps_tk, int K, int T, double dt,
                                               double inv_lam_log2e, float *__restrict__ costs_out,
                                               double *__restrict__ part, int blk)
{
    __shared__ double S_s[TC][KC];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k0 = blk * KC;
    const int k = k0 + tid;
    double acc = 0.0;
    if (tid < KC && k < K) acc = (double)phi[k];

    for (int hi = T; hi > 0; hi -= TC) {
        const int lo = hi > TC ? hi - TC : 0;
        if (tid < KC) {
            // the chunk's costs are loaded first (independent loads in flight),
            // then summed backwards in FP64 in the same order as ever
            float cb[TC];
#pragma unroll
            for (int r = 0; r < TC; ++r) {
                const int i = hi - 1 - r;
                cb[r] = (k < K && i >= lo) ? cost_tk[(size_t)i * K + k] : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < TC; ++r) {
                const int i = hi - 1 - r;
                if (i >= lo) {
                    double s = INFINITY;
                    if (k < K) {
                        acc += (double)cb[r] * dt;
                        s = acc;
                    }
                    S_s[i - lo][tid] = s;
                }
            }
            if (lo == 0 && k < K) costs_out[k] = (float)acc;
        }
        __syncthreads();
        // each warp takes timesteps warp, warp + 8, ... of the chunk; the eps of
        // all of them are loaded before the reductions
        constexpr int RPW = TC / (NT / 32);
        float4 ea[RPW], eb[RPW];
        const int ka = k0 + lane, kb = k0 + lane + 32;
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
            const int r = warp + u * (NT / 32), i = lo + r;
            const bool ok = r < hi - lo;
            ea[u] = ok && ka < K ? eps_tk[(size_t)i * K + ka] : make_float4(0.f, 0.f, 0.f, 0.f);
            eb[u] = ok && kb < K ? eps_tk[(size_t)i * K + kb] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
            const int r = warp + u * (NT / 32), i = lo + r;
            if (r >= hi - lo) break;
            const double sa = S_s[r][lane], sb = S_s[r][lane + 32];
            // exact FP64 minimum: a rounded shift can put exponents hundreds of
            // binary orders off when S is large and lambda small
            const double mn = warp_min_d(fmin(sa, sb));
            const float wa = exp2f((float)((mn - sa) * inv_lam_log2e));
            const float wb = exp2f((float)((mn - sb) * inv_lam_log2e));
            // the 64 rollouts' FP32 terms are summed by a pairwise warp tree in
            // FP32 (B300 has little FP64 throughput); the partials are stored
            // and merged over K in FP64
            const float4 xa = ea[u], xb = eb[u];
            const double z = (double)warp_sum_f(wa + wb);
            const double v0 = (double)warp_sum_f(fmaf(wa, xa.x, wb * xb.x));
            const double v1 = (double)warp_sum_f(fmaf(wa, xa.y, wb * xb.y));
            const double v2 = (double)warp_sum_f(fmaf(wa, xa.z, wb * xb.z));
            const double v3 = (double)warp_sum_f(fmaf(wa, xa.w, wb * xb.w));
            if (lane == 0) {
                double *p = part + ((size_t)blk * T + i) * 6;
                p[0] = mn;
                p[1] = z;
                p[2] = v0;
                p[3] = v1;
                p[4] = v2;
                p[5] = v3;
            }
        }
        __syncthreads();
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
        const double sc = exp2((mn - p[0]) * inv_lam_log2e);
        z = fma(p[1], sc, z);
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = fma(p[2 + a], sc, v[a]);
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
    lse_merge_kernel<<<(T + 7) / 8, 256, 0, s>>>(part, nblk, T, inv_lam_log2e, u_nom, u_out);
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

// pi2rh_kernels.h -- host-side launch interface of the kernels (internal).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "pi2rh_device.cuh"

namespace pi2rh {

// Raises a kernel's dynamic shared-memory limit to `bytes` once per device
// (devices 0-63 are remembered in `done`; concurrent first calls both set the
// same value, which is harmless).
template <typename Kernel>
inline cudaError_t set_smem_once(std::atomic<uint64_t> &done, Kernel *kernel, int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Arguments of the fused rollout kernel (also of the prediction kernel).
struct RolloutArgs {
    const float2 *rec;       // packed model [NY][P][REC_LEN]
    int P;                   // field pairs per output
    int stages_per_out;      // ceil(P / pairs per stage)
    CostDev cost;
    float dt;
    int K, T, M;             // rollouts, steps, sub-rollouts per rollout
    int model_noise;         // 1 = sampled next state, 0 = mean only
    float sqrt_sigma_u[4];   // control-noise standard deviations
    uint64_t seed;
    const float *x0;         // [NX]
    const float *u_nom;      // [T][NU]
    float *cost_tk;          // [T][K] running cost (mean over sub-rollouts)
    float4 *eps_tk;          // [T][K] control perturbations
    float *phi;              // [K] terminal cost (mean over sub-rollouts)
    const float *z_in;       // prediction: [n_pred][NZ]
    float *y_out, *var_out;  // prediction: [n_pred][NY]
    int n_pred;
    int *err;                // device error word
    // Output-split launch of the FP32 rollout (see launch_rollout_fp32):
    // exchange area of split_bytes(split_max_blocks) bytes (null: never
    // split), its mode, and a tag that differs between launches on one area.
    unsigned char *split;
    int split_max_blocks;
    int split_mode;          // PI_SPLIT_OFF / _AUTO / _ALWAYS
    uint32_t split_epoch;    // >= 1, new for every launch on `split`
    int split_upc;           // set by the launcher: (block, output) units per CTA,
    int split_b0, split_blocks;  // and the 64-slot blocks [b0, b0 + blocks) the split launch covers
    int split_drop;          // failure-path checks (0 normally): 1 = leave the split grid's last CTA
                             // out, 2 = treat the split launch as refused by the runtime
    int block0;              // first 64-slot block of a plain launch (set by the launcher)
};

// Rollout slots (rollout x sub-rollout) per CTA of the FP32 rollout kernel.
constexpr int RF_SLOTS = 64;
constexpr int RF_CONSUMER_WARPS = 8;
// Field-pair records per stage of the FP32 kernel's record ring: 8 per
// consumer warp, so each warp's waits and arrivals are amortized over 8 records.
constexpr int RF_PAIRS_PER_STAGE = 8 * RF_CONSUMER_WARPS;

// Work list of the persistent batched rollout kernels: item = (controller,
// slot block); CTAs claim items through *counter (zeroed before the launch).
struct BatchArgs {
    const RolloutArgs *args;   // [n_ctrl] per-controller arguments (FP32 form)
    const int2 *items;         // [n_items] (controller, block of RF_SLOTS slots)
    int n_items;
    int *counter;
    int *err;
};

// Exchange area of the output-split FP32 launch: a 128-byte header, then per
// 64-slot block its flags (z published, outputs done per non-owner CTA) and
// its z, y and var rows.
constexpr size_t SPLIT_HDR_BYTES = 128;
constexpr size_t SPLIT_BLOCK_BYTES = 128 + (size_t)(NZ + 2 * NY) * RF_SLOTS * 4;
inline size_t split_bytes(int max_blocks) { return SPLIT_HDR_BYTES + (size_t)max_blocks * SPLIT_BLOCK_BYTES; }

// How an FP32 rollout is launched: plain_blocks 64-slot blocks [0, plain_blocks)
// one CTA each (whole waves), then, when upc > 0, the remaining split_blocks
// blocks [split_b0, split_b0 + split_blocks) of a last, partial wave as the
// output-split launch: their (block, output) units dealt out upc at a time
// to split_ctas co-resident CTAs (one per SM).
struct Fp32Launch {
    int plain_blocks;
    int split_b0, split_blocks, upc, split_ctas;
};
// (A stream that is capturing a CUDA graph always gets the plain launch.)
Fp32Launch fp32_launch_plan(const RolloutArgs &a, cudaStream_t s);
// The plan for `blocks` 64-slot blocks on nsm SMs, P field pairs per output,
// split mode `mode` and an exchange area of max_blocks blocks (host only).
Fp32Launch fp32_plan_blocks(long long blocks, int nsm, int P, int mode, int max_blocks);
// The segments the split kernel's CTA `cta` evaluates (the kernel's own
// partition, run on the host): seg[5 i ..] = {block, first output, end output,
// owned, owned ? CTAs before it holding the block : its index among them}, in
// evaluation order; returns the count (0 for an invalid CTA).
int fp32_split_partition(int blocks, int upc, int cta, int *seg);

// The FP32 rollout (one or two launches, as fp32_launch_plan says; *n_launched
// = how many).  The results are those of the one-CTA-per-block launch bit for
// bit whatever the split.
cudaError_t launch_rollout_fp32(const RolloutArgs &a, cudaStream_t s, int *n_launched = nullptr);
cudaError_t launch_rollout_fp32_batch(const BatchArgs &b, int grid, cudaStream_t s);
// Plain-launch form of the batch: one item per CTA (b.counter unused).
cudaError_t launch_rollout_fp32_group(const BatchArgs &b, cudaStream_t s);
cudaError_t launch_predict_fp32(const RolloutArgs &a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Tensor-core form.  Coefficient tiles of 128 fields are pre-packed at context
// creation as 11 chunks of 8 KB in the exact shared-memory image the MMAs
// read (fp16, K-major core-matrix layout, 128 rows x 16 K per half-chunk):
// chunk 0 = [S hi of K step 0 | Y hi], chunk 1 = [S lo of K step 0 | Y lo]
// (one N = 256 MMA serves K step 0 of S and the whole Y GEMM, which share
// the A operand z), chunk j + 1 = [S hi | S lo] of K step j = 1..9; the
// per-field constants (cy, sigma^2; 2 x 128 floats) are packed separately.
// ---------------------------------------------------------------------------
constexpr int TC_SLOTS = 128;           // rollout slots per CTA (MMA M)
constexpr int TC_TILE_FIELDS = 128;     // fields per tile (MMA N)
constexpr int TC_KF = 160;              // feature columns: z (16), z_a z_b (136), 1, 0 (7)
constexpr int TC_HALF_CHUNK = TC_TILE_FIELDS * 16 * 2;                 // 4 KB
constexpr int TC_CHUNK_BYTES = 2 * TC_HALF_CHUNK;                      // 8 KB
constexpr int TC_CHUNKS_PER_TILE = TC_KF / 16 + 1;                     // 11
constexpr int TC_TILE_BYTES = TC_CHUNKS_PER_TILE * TC_CHUNK_BYTES;     // 90,112
constexpr int TC_CONST_BYTES = 2 * TC_TILE_FIELDS * 4;                 // 1,024
// Chunks 2..TC_QUAD_LAST_CHUNK carry K steps 1..8 of the exponent GEMM, whose
// features (16..143) are all quadratic z_a z_b.
constexpr int TC_QUAD_LAST_CHUNK = 9;
constexpr int TC_CONST_FEATURE = 152;   // feature column holding the constant 1 (+ 2^-14 in the lo part)

// Quadratic feature k (16 <= k < 152) is z_a z_b with (a, b) the (k-16)-th
// entry of the row-major upper triangle; features k < 16 are z_k.
__host__ __device__ constexpr int tc_feat_row(int k)
{
    int t = k - 16, a = 0;
    while (a < 16 && t >= 16 - a) { t -= 16 - a; ++a; }
    return a;
}
__host__ __device__ constexpr int tc_feat_col(int k)
{
    int t = k - 16, a = 0;
    while (a < 16 && t >= 16 - a) { t -= 16 - a; ++a; }
    return a + t;
}

struct TcArgs {
    const unsigned char *wtiles;   // [NY][tiles_per_out][TC_TILE_BYTES]
    const unsigned char *wconst;   // [NY][tiles_per_out][TC_CONST_BYTES]
    int tiles_per_out;
    CostDev cost;
    float dt;
    int K, T, M;
    int model_noise;
    float sqrt_sigma_u[4];
    uint64_t seed;
    const float *x0;
    const float *u_nom;
    float *cost_tk;
    float4 *eps_tk;
    float *phi;
    const float *z_in;
    float *y_out, *var_out;
    int n_pred;
    int *err;
    int qprod;   // split products on the quadratic-feature K steps: 3 or 2 (selects the kernel)
};

struct TcBatchArgs {
    const TcArgs *args;        // [n_ctrl] per-controller arguments (tensor-core form)
    const int2 *items;         // [n_items] (controller, block of TC_SLOTS slots)
    int n_items;
    int *counter;
    int qprod;                 // split products of every controller in the launch (3 or 2)
};

cudaError_t launch_rollout_tc(const TcArgs &a, cudaStream_t s);
cudaError_t launch_rollout_tc_batch(const TcBatchArgs &b, int grid, cudaStream_t s);
// Non-persistent form of the batch launch: one item per CTA or per cluster of
// `split` CTAs (outputs split as in the single-controller kernel), one wave.
// tc_group_split(n) = the split that keeps n items in one wave (1 = none fits).
int tc_group_split(int n_items);
cudaError_t launch_rollout_tc_group(const TcBatchArgs &b, int split, cudaStream_t s);
cudaError_t launch_predict_tc(const TcArgs &a, cudaStream_t s);
const char *tc_launch_diag();   // resources of the tensor-core kernel (for error messages)

// Cost-to-go scan + per-CTA log-sum-exp partials, then the merge over CTAs.
constexpr int RS_KC = 64;   // rollouts per CTA of the scan kernel
int scan_blocks(int K);
cudaError_t launch_scan_lse(const float *cost_tk, const float *phi, const float4 *eps_tk, int K,
                            int T, float dt, double inv_lam_log2e, float *costs_out, double *part,
                            cudaStream_t s);
cudaError_t launch_lse_merge(const double *part, int nblk, int T, double inv_lam_log2e,
                             const float *u_nom, float *u_out, cudaStream_t s);

// Receding-horizon advance.
cudaError_t launch_rh_build_z(const float *x0, const float *u_out, float *z, cudaStream_t s);
cudaError_t launch_rh_apply(float *x0, const float *y, float dt, const float *u_out, int T, float *u_next,
                            cudaStream_t s);

// Staged check of the tensor-core GEMM core: D[128x64] = A[128xK] B[64xK]^T, fp16 in, fp32 out.
cudaError_t launch_tc_gemm_check(const void *A, const void *B, int K, float *D, int *err, cudaStream_t s);

// Per-controller arguments of the batched reduction kernels.
struct ReduceArgs {
    const float *cost_tk;
    const float *phi;
    const float4 *eps_tk;
    int K, T;
    double dt, inv_lam_log2e;
    float *costs_out;
    double *part;
    const float *u_nom;
    float *u_out;
};
// scan items: (controller, block of RS_KC rollouts); merge items: (controller, first of 8 timesteps)
cudaError_t launch_scan_lse_batch(const ReduceArgs *args, const int2 *items, int n_items, cudaStream_t s);
cudaError_t launch_lse_merge_batch(const ReduceArgs *args, const int2 *items, int n_items, cudaStream_t s);

// One bounded device-side wait that is never satisfied (failure-path check).
cudaError_t launch_wait_timeout(int *err, unsigned long long limit_ns, cudaStream_t s);

// Staged noise kernels.
cudaError_t launch_noise_raw(uint64_t seed, int K, int T, int m, uint32_t *raw, cudaStream_t s);
cudaError_t launch_noise_normals(uint64_t seed, int K, int T, int m, float *ctrl, float *model,
                                 cudaStream_t s);

}  // namespace pi2rh

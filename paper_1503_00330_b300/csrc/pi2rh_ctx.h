// pi2rh_ctx.h -- definition of the context object behind the opaque pi_ctx
// handle of the C ABI (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "pi2rh.h"
#include "pi2rh_device.cuh"
#include "pi2rh_kernels.h"

struct pi_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    pi_opts opts{};
    int L = 0, P = 0, spo = 0;
    float dt = 0.f;
    float2 *d_rec = nullptr;   // packed model [NY][P][REC_LEN]
    unsigned char *d_wtiles = nullptr;   // tensor-core coefficient tiles (precision TC)
    unsigned char *d_wconst = nullptr;   // tensor-core per-field constants
    int tiles_per_out = 0;
    float2 *d_obs = nullptr;
    pi2rh::CostDev cost{};
    int *d_err = nullptr;
    // per-update scratch
    float *d_cost = nullptr;   // [T][K]
    float4 *d_eps = nullptr;   // [T][K]
    float *d_phi = nullptr;    // [K]
    double *d_part = nullptr;  // [nblk][T][6]
    size_t cap_cost = 0, cap_eps = 0, cap_phi = 0, cap_part = 0;
    // staging for the host-buffer path
    float *d_x0 = nullptr, *d_unom = nullptr, *d_uout = nullptr, *d_costs = nullptr;
    size_t cap_x0 = 0, cap_unom = 0, cap_uout = 0, cap_costs = 0;
    // receding-horizon advance scratch: z [16], y [12], var [12]
    float *d_rh = nullptr;
    // per-kernel timing: a ring of event sets, timed update n records into set
    // n % PI2RH_TIMING_RING (start, after the rollout, after the scan, end)
    bool timing = false;
    cudaEvent_t ev[PI2RH_TIMING_RING][4] = {};
    uint64_t n_timed = 0;
    uint64_t launches = 0;
    // exchange area of the output-split FP32 rollout launch (FP32 contexts)
    unsigned char *d_split = nullptr;
    int split_max_blocks = 0;
    int split_mode = PI_SPLIT_AUTO;
    uint32_t split_epoch = 0;
    int split_drop = 0;   // pi_debug_split_drop_cta
};

// Scoped NVTX range on the calling host thread (shown by profilers that attach
// to NVTX; a few nanoseconds otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// True for the tensor-core precisions (one packed model, the tensor-core rollout kernel).
inline bool pi2rh_is_tc(int precision)
{
    return precision == PI_PRECISION_TC_FP16X3 || precision == PI_PRECISION_TC_FP16X2;
}

// Split products on the quadratic-feature K steps of a tensor-core precision.
inline int pi2rh_tc_qprod(int precision) { return precision == PI_PRECISION_TC_FP16X2 ? 2 : 3; }

// The event set the next timed update records into, or nullptr with timing off.
inline cudaEvent_t *timing_slot(pi_ctx *c)
{
    return c->timing ? c->ev[c->n_timed % PI2RH_TIMING_RING] : nullptr;
}

// Records msg as the calling thread's last error (pi_last_error) and returns code.
int pi2rh_fail(int code, const char *msg);

// Kernel arguments that depend only on the context (model, cost, options).
inline pi2rh::RolloutArgs ctx_rollout_args(const pi_ctx *c)
{
    pi2rh::RolloutArgs a{};
    a.rec = c->d_rec;
    a.P = c->P;
    a.stages_per_out = c->spo;
    a.cost = c->cost;
    a.dt = c->dt;
    a.M = c->opts.M;
    a.model_noise = c->opts.model_noise == PI_NOISE_SAMPLED ? 1 : 0;
    a.err = c->d_err;
    return a;
}

// Output-split fields of the next FP32 rollout launch on the context's own
// exchange area: a fresh epoch per launch (the area starts zeroed, so epochs
// start at 1; before the counter wraps, the area is cleared on the stream).
inline cudaError_t ctx_split_args(pi_ctx *c, pi2rh::RolloutArgs &a)
{
    a.split = c->d_split;
    a.split_max_blocks = c->split_max_blocks;
    a.split_mode = c->split_mode;
    a.split_drop = c->split_drop;
    if (!c->d_split) return cudaSuccess;
    if (c->split_epoch == 0xffffffffu) {
        cudaError_t e = cudaMemsetAsync(c->d_split, 0, pi2rh::split_bytes(c->split_max_blocks), c->stream);
        if (e != cudaSuccess) return e;
        c->split_epoch = 0;
    }
    a.split_epoch = ++c->split_epoch;
    return cudaSuccess;
}

inline pi2rh::TcArgs ctx_tc_args(const pi_ctx *c)
{
    pi2rh::TcArgs t{};
    t.wtiles = c->d_wtiles;
    t.wconst = c->d_wconst;
    t.tiles_per_out = c->tiles_per_out;
    t.cost = c->cost;
    t.dt = c->dt;
    t.M = c->opts.M;
    t.model_noise = c->opts.model_noise == PI_NOISE_SAMPLED ? 1 : 0;
    t.err = c->d_err;
    t.qprod = pi2rh_tc_qprod(c->opts.precision);
    return t;
}

/*
 * pi2rh.h -- C ABI of the B300 (sm_103a) implementation of one receding-horizon
 * path-integral (PI^2-RH) control update over a learned LWPR dynamics model
 * ("GPU based Path Integral Control with Learned Dynamics", arXiv 1503.00330).
 *
 * One update (pi_update) computes, on the GPU:
 *   1. K perturbed control sequences u_{k,t} = u_nom_t + eps_{k,t},
 *      eps ~ N(0, diag(sigma_u)), drawn in-kernel from Philox4x32-10
 *      (Sec. 3.1, "sample possible trajectories").
 *   2. K rollouts of T Euler steps through the probabilistic LWPR model:
 *      normalized Gaussian receptive-field weights, local linear mean, variance
 *      (Sec. 2, Eq. 1), and a sampled next state x + dt (y + sigma n)
 *      (Sec. 3.2; Euler integration as in Table 1). With M > 1 each rollout is
 *      M sub-rollouts that share eps and average their cost (Sec. 3.2).
 *   3. the running cost q(x_t, z_t) per step and the terminal cost phi(x_T)
 *      (Sec. 5 obstacle-navigation cost; indicator or Gaussian-bump form).
 *   4. the cost-to-go S_{k,i} = phi + dt sum_{j>=i} q_{k,j} (Sec. 3.1), in FP64.
 *   5. per timestep i, the weights exp(-S_{k,i}/lambda) / sum_k and
 *      u_out_i = u_nom_i + sum_k P_{k,i} eps_{k,i} (Sec. 3.1, Eq. 2), with the
 *      normalization over k in FP64.
 *
 * Fixed dimensions: state NX = 12 (position, velocity, roll/pitch/yaw, body
 * rates), control NU = 4 (thrust, roll, pitch, yaw-rate), LWPR input
 * z = [x, u] (NZ = 16), LWPR outputs NY = 12 (the state derivatives).
 *
 * Conventions for every entry point:
 *   - Return value 0 (PI_OK) or a PI_ERR_* code; pi_last_error() gives a
 *     message for the calling thread.  No entry point aborts the process.
 *   - "device" pointers are CUDA global-memory pointers on the context's
 *     device; "host" pointers are ordinary CPU memory.  The caller owns every
 *     buffer it passes; the library never frees or retains caller memory.
 *   - Work is enqueued asynchronously on the context's stream (pi_set_stream,
 *     default: the legacy default stream) unless stated otherwise.  Results are
 *     valid once that stream is synchronized; pi_sync() does that and reports
 *     device-side errors.
 *   - Float inputs must be finite; non-finite inputs give unspecified (but
 *     memory-safe) outputs.
 */
#ifndef PI2RH_H
#define PI2RH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PI2RH_NX 12
#define PI2RH_NU 4
#define PI2RH_NZ 16
#define PI2RH_NY 12
#define PI2RH_MAX_OBS 256
#define PI2RH_MAX_M 64

enum {
    PI_OK = 0,
    PI_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range       */
    PI_ERR_OOM = 2,         /* device allocation failed                           */
    PI_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed         */
    PI_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired (see pi_sync)    */
    PI_ERR_INTERNAL = 5,    /* a device-side consistency check failed              */
    PI_ERR_UNSUPPORTED = 6, /* option not available in this build                  */
    PI_ERR_BUSY = 7,        /* the object has work in flight that the call needs finished */
    PI_ERR_CANCELLED = 8    /* a serving request was cancelled before it reached the GPU */
};

/* PI_PRECISION_FP32: receptive fields evaluated on the FP32 FMA pipe.
 * PI_PRECISION_TC_FP16X3: quadratic forms and local predictions as tensor-core
 * GEMMs (tcgen05, fp16 hi/lo split, three products per term, fp32 accumulate);
 * requires every LWPR input |z_a| < 255 so the fp16 features stay finite.
 * Accurate to the FP32 form's level.
 * PI_PRECISION_TC_FP16X2: the same GEMMs with two split products (features at
 * their fp16 rounding, weights split hi + lo) on the 128 quadratic features
 * z_a z_b of the exponent, three on the linear and constant features and on
 * the local predictions.  Each quadratic term then carries an fp16 rounding
 * (2^-11 relative) instead of ~2^-22: about 11-16 % faster than FP16X3 and
 * held to the tensor-core form's stated bound (2e-3 on u_out per channel)
 * rather than the FP32 one.  Both tensor-core forms share one packed model. */
enum { PI_PRECISION_FP32 = 0, PI_PRECISION_TC_FP16X3 = 1, PI_PRECISION_TC_FP16X2 = 2 };
enum { PI_NOISE_MEAN_ONLY = 0, PI_NOISE_SAMPLED = 1 };
enum { PI_SPLIT_OFF = 0, PI_SPLIT_AUTO = 1, PI_SPLIT_ALWAYS = 2 };
enum { PI_OBS_INDICATOR = 0, PI_OBS_GAUSSIAN = 1 };

typedef struct pi_ctx pi_ctx;

/* LWPR model (Sec. 2, Eq. 1).  All arrays host, float32, row-major, copied at
 * pi_create.  n_in must be 16 and n_out 12; L >= 1 fields per output.
 *   c     [n_out][L][n_in]        receptive-field centers c_j
 *   D     [n_out][L][n_in][n_in]  distance metrics D_j (used through the
 *                                 quadratic form, so only D + D^T matters)
 *   beta  [n_out][L][n_in]        local slopes: y_j(z) = b_j + beta_j . (z - c_j)
 *   b     [n_out][L]              local offsets (value at the center)
 *   sigma [n_out][L]              per-field noise standard deviation sigma_j
 *   dt                            Euler step (s), > 0                          */
typedef struct {
    int n_in;
    int n_out;
    int L;
    float dt;
    const float *c;
    const float *D;
    const float *beta;
    const float *b;
    const float *sigma;
} pi_lwpr_params;

/* Running cost (Sec. 5 form, generalized):
 *   q(x, z) = sum_d Q_pos[d] (p_d - goal_d)^2 + Q_vel |v|^2 + Q_ang |angles|^2
 *           + (obs_kind == PI_OBS_INDICATOR ? w_obs * C
 *                                           : w_obs * sum_i exp(-obs_sharp d_i^2))
 *           + w_crash * C + w_var * sum_o var_o(z)
 *   C = 1 if (p_x, p_y) is strictly inside any vertical cylinder of the given
 *   radius around obs_xy[i] (decided in FP32), else 0.
 * Terminal cost phi(x_T) = w_T * sum_d Q_pos[d] (p_{T,d} - goal_d)^2.
 * obs_xy: host [n_obs][2], 0 <= n_obs <= PI2RH_MAX_OBS, copied at pi_create. */
typedef struct {
    float goal[3];
    float Q_pos[3];
    float Q_vel;
    float Q_ang;
    float w_obs;
    float obs_sharp;
    float radius;
    float w_crash;
    float w_var;
    float w_T;
    int obs_kind;
    int n_obs;
    const float *obs_xy;
} pi_cost_params;

/* Options.  precision: PI_PRECISION_FP32, PI_PRECISION_TC_FP16X3 or
 * PI_PRECISION_TC_FP16X2.  model_noise: PI_NOISE_SAMPLED
 * (draw x' = x + dt (y + sigma n)) or PI_NOISE_MEAN_ONLY (x' = x + dt y).
 * M: sub-rollouts per rollout (Sec. 3.2), a power of two in [1, 64].
 * device: CUDA device ordinal. */
typedef struct {
    int precision;
    int model_noise;
    int M;
    int device;
} pi_opts;

/* Fills *opts with FP32, sampled noise, M = 1, device 0. */
void pi_default_opts(pi_opts *opts);

/* Creates a context: validates and packs the model into the kernel's record
 * layout and copies model, obstacles and options to the device (synchronous).
 * opts may be NULL (defaults).  On success *out owns device memory until
 * pi_destroy.  Errors: INVALID_ARG (bad dims / NULL / ranges), OOM, CUDA. */
int pi_create(const pi_lwpr_params *lwpr, const pi_cost_params *cost, const pi_opts *opts,
              pi_ctx **out);

/* Sets the cudaStream_t (passed as void*) used by later calls; NULL = legacy
 * default stream.  The stream must belong to the context's device. */
int pi_set_stream(pi_ctx *ctx, void *stream);

/* Pre-allocates the per-update scratch for K rollouts and T steps so that later
 * pi_update calls with K' <= K, T' <= T allocate nothing. */
int pi_reserve(pi_ctx *ctx, int K, int T);

/* One control update (Sec. 3.1 / Eq. 2 over the rollouts of Sec. 3.2).
 *   x0        device [12]      initial state
 *   u_nominal device [T][4]    nominal controls (may alias u_out)
 *   K >= 1 rollouts, T >= 1 steps; lambda > 0 (temperature of Eq. 2)
 *   sigma_u   host [4]         control-noise variances (>= 0), Sigma_u = diag
 *   seed                       Philox key; noise of rollout k, step t, block b,
 *                              sub-rollout m uses counter (k, t, b, m)
 *   u_out     device [T][4]    u_nom + sum_k P_k eps_k per timestep
 *   costs_out device [K]       S_{k,0}, the cost-to-go of each whole rollout
 * Asynchronous on the context's stream.  Scratch (about K*T*20 bytes) is
 * grown with stream-ordered allocation when needed.  Errors: INVALID_ARG,
 * OOM, CUDA; device-side errors are reported by pi_sync. */
int pi_update(pi_ctx *ctx, const float *x0, const float *u_nominal, int K, int T, float lambda,
              const float *sigma_u, uint64_t seed, float *u_out, float *costs_out);

/* Limits of pi_update_noalloc's fixed scratch. */
#define PI2RH_NOALLOC_MAX_K 65536
#define PI2RH_NOALLOC_MAX_T 4096
#define PI2RH_NOALLOC_MAX_KT 1048576

/* pi_update for callers that cannot allocate device memory once they are
 * running: a real-time control loop that must not call cudaMalloc after
 * start-up (allocation can block, synchronize the device or fail at any
 * moment), or a host program that owns all GPU memory through its own pool.
 * There is no counterpart in the paper; it is a deployment variant.
 *
 * Same arguments, results and stream semantics as pi_update, in either form
 * (it runs the rollout kernel of the context's opts.precision, FP32 or tensor
 * cores, and the same reduction kernels, so its results equal pi_update's bit
 * for bit), but it calls no
 * allocating routine: the per-update scratch lives in one fixed device array
 * of about 21 MiB inside the library, held by every GPU that loads the library
 * until the process exits.  Limits: K <= PI2RH_NOALLOC_MAX_K,
 * T <= PI2RH_NOALLOC_MAX_T, K*T <= PI2RH_NOALLOC_MAX_KT; larger sizes return
 * PI_ERR_INVALID_ARG with a message and launch nothing.  On an FP32 context
 * the output-split launch of the rollout (pi_set_output_split) exchanges its
 * per-step state through the context's own 1.5 MB area, which pi_create
 * allocated, so it too needs no allocation here.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it.  Under CUDA's lazy module loading
 * (the default) that lookup is also when the runtime loads the array onto the
 * device, which commits its memory: make the first call on each device during
 * set-up (a small update will do), before the real-time loop starts and
 * before any stream capture.  Stage times (pi_set_timing / pi_stage_times)
 * cover this entry point as they cover pi_update.  All calls on a device share the one array: calls whose
 * work overlaps on the GPU (different streams or contexts without ordering
 * between them) race and corrupt each other's results; order them on one
 * stream or synchronize between them.  Every scratch element a call reads is
 * written earlier in the same call, so no clearing is needed between calls. */
int pi_update_noalloc(pi_ctx *ctx, const float *x0, const float *u_nominal, int K, int T,
                      float lambda, const float *sigma_u, uint64_t seed, float *u_out,
                      float *costs_out);

/* Same update with HOST buffers (x0 [12], u_nominal [T][4], u_out [T][4],
 * costs_out [K]): copies inputs to context-owned device buffers, runs
 * pi_update, copies results back and synchronizes the stream before
 * returning.  This is the end-to-end path (host<->device copies included). */
int pi_update_host(pi_ctx *ctx, const float *x0, const float *u_nominal, int K, int T,
                   float lambda, const float *sigma_u, uint64_t seed, float *u_out,
                   float *costs_out);

/* Receding-horizon advance (Sec. 3.1: execute one step of the plan, then
 * warm-start the next update with the unexecuted remainder).  On the context's
 * stream, with device buffers:
 *   x0        [12] in/out   x0 <- x0 + dt * y(z), y the LWPR mean (Eq. 1) at
 *                           z = [x0, u_out[0]] (the synthetic plant)
 *   u_out     [T][4] in     plan returned by pi_update
 *   u_nom_next[T][4] out    u_out shifted left by one step, last step repeated;
 *                           must not overlap u_out */
int pi_rh_advance(pi_ctx *ctx, float *x0, const float *u_out, int T, float *u_nom_next);

/* How the FP32 rollout kernel of pi_update (and pi_update_noalloc) is
 * launched on an FP32 context (no effect on tensor-core contexts).  The plain
 * launch gives each block of 64 rollout slots (rollout x sub-rollout) one CTA
 * for all T steps; with fewer blocks than the GPU has SMs some SMs then stay
 * idle (K = 8192, M = 1: 128 blocks on 148 SMs).  The output-split launch
 * deals the blocks' (block, output) pairs out to one co-resident CTA per SM
 * (a cooperative launch), which exchange each step's state through a 1.5 MB
 * area in device memory allocated by pi_create; every output is still
 * evaluated by one CTA in the same order, so the results are identical bit
 * for bit (Sec. 2, Eq. 1: the split changes which SM evaluates which
 * receptive fields, not the arithmetic).  With more blocks than SMs, whole
 * waves of blocks keep the plain launch and only the blocks of the last,
 * partial wave are split (two launches).
 *   PI_SPLIT_OFF     always the plain launch
 *   PI_SPLIT_AUTO    (default) split the partial wave where that takes work
 *                    off the busiest SM: fewer than ~11/12 as many blocks in
 *                    it as SMs and (12 - outputs per CTA) * ceil(L / 2) >= 64
 *   PI_SPLIT_ALWAYS  split it whenever that takes work off the busiest SM
 * An update enqueued on a stream that is capturing a CUDA graph always takes
 * the plain launch (a replayed split launch would reuse the flags' tag).
 * A bounded wait of one CTA on another that expires shows as PI_ERR_TIMEOUT
 * from pi_sync.  Errors: INVALID_ARG (mode). */
int pi_set_output_split(pi_ctx *ctx, int mode);

/* Per-kernel timing of pi_update (and pi_update_noalloc) with CUDA events on
 * the context's stream (off by default).  The context keeps the events of the
 * last PI2RH_TIMING_RING timed updates, so a caller can enqueue many updates
 * back to back and read their times afterwards.
 *   pi_stage_times     waits for the last timed update and writes ms[0] =
 *                      rollout kernel, ms[1] = cost-to-go/LSE kernel, ms[2] =
 *                      merge kernel (milliseconds)
 *   pi_stage_times_at  the same for the timed update `back` calls before the
 *                      last (back = 0 is the last); INVALID_ARG unless
 *                      0 <= back < min(timed updates so far, PI2RH_TIMING_RING)
 * Host memory ms[3]; both block until that update's kernels have finished. */
#define PI2RH_TIMING_RING 64
int pi_set_timing(pi_ctx *ctx, int enable);
int pi_stage_times(pi_ctx *ctx, float *ms);
int pi_stage_times_at(pi_ctx *ctx, int back, float *ms);

/* ---------------------------------------------------------------------------
 * Batched form: many independent controllers of uneven size (own model, cost,
 * K, T, M, seed) updated by ONE persistent rollout launch over a work list of
 * (controller, rollout block) items, plus one batched cost-to-go launch and one
 * batched merge launch, captured in a CUDA graph on the first update and
 * replayed afterwards (Sec. 3.1 update, per controller, as pi_update).
 * ------------------------------------------------------------------------- */
typedef struct pi_batch pi_batch;

/* One controller of a batch.  ctx is borrowed (must outlive the batch); the
 * device buffers x0 [12], u_nominal [T][4], u_out [T][4], costs_out [K] are
 * fixed for the life of the batch (their contents may change between updates). */
typedef struct {
    pi_ctx *ctx;
    int K;
    int T;
    const float *x0;
    const float *u_nominal;
    float *u_out;
    float *costs_out;
} pi_batch_item;

enum {
    PI_BATCH_ORDER_AS_GIVEN = 0,       /* items in controller order                     */
    PI_BATCH_ORDER_LONGEST_FIRST = 1,  /* default: largest per-block work first (LPT)    */
    PI_BATCH_ORDER_ROUND_ROBIN = 2     /* one block of each controller in turn           */
};

/* Creates a batch over n items, all of whose contexts live on one device.
 * precision PI_PRECISION_FP32 uses the FP32 rollout kernel; PI_PRECISION_TC_FP16X3
 * or PI_PRECISION_TC_FP16X2 the tensor-core one with that many split products
 * (every context must then have been created with the same precision).
 * Allocates the per-controller scratch (about K*T*20 bytes each) and the
 * device tables; synchronous.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
int pi_batch_create(const pi_batch_item *items, int n, int precision, pi_batch **out);

/* Schedule knobs (used by the autotuner): work-list order and the number of
 * persistent CTAs (0 = one per SM).  Re-captures the graph on the next update. */
int pi_batch_set_schedule(pi_batch *b, int order, int grid);

/* Tile shape of the batch (used by the autotuner).  split = 0 (default): the
 * persistent work list above, one CTA per item (128 slots x 12 outputs with
 * tensor cores, 64 slots x 12 outputs in FP32).  split = 1: a plain launch
 * with one item per CTA.  split = 2..4 (tensor cores only): one item per
 * cluster of `split` CTAs, each evaluating 12/split of the item's outputs for
 * its 128 slots.  Every shape gives the same results, bitwise.  INVALID_ARG
 * for split > 1 on an FP32 batch.  Re-captures the graph on the next update. */
int pi_batch_set_tile(pi_batch *b, int split);

/* Stream the batch's work is ordered after (and that waits for it); NULL = legacy default stream. */
int pi_batch_set_stream(pi_batch *b, void *stream);

/* One update of every controller: lambda [n], sigma_u [n][4] (variances) and
 * seed [n] are host arrays.  Asynchronous with respect to the host. */
int pi_batch_update(pi_batch *b, const float *lambda, const float *sigma_u, const uint64_t *seed);

/* Waits for the batch and reports device-side errors of its contexts (as pi_sync). */
int pi_batch_sync(pi_batch *b);

/* Kernel launches enqueued by the batch (3 per update). */
uint64_t pi_batch_launch_count(const pi_batch *b);

/* Frees the batch (not its contexts or item buffers).  NULL is accepted. */
void pi_batch_destroy(pi_batch *b);

/* ---------------------------------------------------------------------------
 * Serving form: a receding-horizon request loop for many simulated vehicles
 * that share one LWPR model and cost (one pi_ctx).  Each request is one
 * control update of one vehicle ("agent") followed, on the device, by the
 * receding-horizon advance of that agent (Sec. 3.1, PI^2-RH: execute the
 * first control of the plan on the simulated plant -- one Euler step of the
 * LWPR mean at [x0, u_out_0] -- and warm-start the next plan with the shifted
 * remainder, the last control held).  The paper runs one controller; serving
 * many of them is an engineering extension with no counterpart there.
 *
 * Per-agent state stays in device memory for the life of the server: the
 * state x0 [12], the warm-start plan [T_max][4] and an update counter.  The
 * noise seed of an agent's n-th update is agent_seed + n * 0x9E3779B97F4A7C15
 * (mod 2^64), formed on the device from that counter.
 *
 * A native scheduler thread admits queued requests in arrival order when a
 * launch lane (a CUDA stream) is free and the request's scratch (about
 * K*T*20 bytes) fits in the server's HBM pool; the requests admitted together
 * form one group, updated by one persistent batched rollout launch plus the
 * batched cost-to-go, merge and advance launches.  Groups on different lanes
 * overlap on the device.  An agent has at most one request on the GPU; later
 * requests of a busy agent wait in the queue without holding back others.
 * Every result equals, bitwise, the result of the same update run alone
 * (pi_update followed by pi_rh_advance with the same seed).
 * ------------------------------------------------------------------------- */
typedef struct pi_server pi_server;

typedef struct {
    int n_agents;       /* simulated vehicles (device-resident state slots), >= 1          */
    int K_max;          /* largest K a request may ask for                                  */
    int T_max;          /* longest horizon a request may ask for (warm-start plan length)   */
    int max_inflight;   /* launch lanes: groups that may be on the GPU at once (>= 1)       */
    int max_group;      /* most requests packed into one group (>= 1)                       */
    size_t hbm_budget;  /* bytes of the scratch pool; 0 = half the free device memory,
                           at most 32 GiB                                                   */
    int want_costs;     /* 1: each kept result also holds the K per-rollout costs           */
} pi_server_opts;

/* One control update request of one agent. */
typedef struct {
    int agent;          /* 0 .. n_agents-1                                                   */
    int K, T;           /* rollouts and horizon: 1 <= K <= K_max, 1 <= T <= T_max            */
    float lambda;       /* temperature (> 0)                                                 */
    float sigma_u[4];   /* control-noise variances (>= 0)                                    */
    const float *x0;    /* host [12]: measured state replacing the agent's device state
                           before the update; NULL = use the device-resident state          */
    int keep_result;    /* 1: hold u_out (and costs) on the host for pi_server_result        */
} pi_serve_request;

/* Completion record of one request.  Times are host monotonic-clock
 * nanoseconds: submission, the group's launch, and the moment the scheduler
 * saw the result in host memory. */
typedef struct {
    uint64_t ticket;
    int agent, K, T;
    int status;         /* PI_OK, or PI_ERR_TIMEOUT / PI_ERR_INTERNAL / PI_ERR_CUDA, or
                           PI_ERR_CANCELLED (t_launch_ns is then 0)                         */
    int group_size;     /* requests in the launch that carried this one                      */
    int64_t t_submit_ns, t_launch_ns, t_result_ns;
} pi_serve_done;

/* One arrival of a replayed trace: at t_ns after the replay starts, agent asks
 * for an update of size (K, T). */
typedef struct {
    int64_t t_ns;
    int agent, K, T;
} pi_serve_arrival;

typedef struct {
    uint64_t submitted, completed, groups, launches;
    uint64_t memory_waits;      /* scheduler passes whose next eligible request did not fit the pool */
    size_t pool_bytes, pool_peak_bytes;
    int peak_inflight_requests, peak_group_size;
} pi_server_stats;

/* Defaults: n_agents 1, K_max 16384, T_max 128, max_inflight 2, max_group 64,
 * hbm_budget 0, want_costs 0. */
void pi_server_default_opts(pi_server_opts *opts);

/* Creates a server over ctx's model and cost (ctx is borrowed and must
 * outlive the server; its stream and scratch are not used) in the context's
 * precision, and starts the scheduler thread.  Agents start at x0 = 0, a zero
 * plan, counter 0 and seed = agent index.  Synchronous.
 * Errors: INVALID_ARG, OOM (pool or tables do not fit), CUDA. */
int pi_server_create(pi_ctx *ctx, const pi_server_opts *opts, pi_server **out);

/* Sets an agent's device state: x0 [12] (host), plan u_warm [T_max][4] (host,
 * NULL = zeros) and seed; resets its counter to 0.  The agent must have no
 * request queued or in flight (else PI_ERR_BUSY).  Synchronous. */
int pi_server_set_agent(pi_server *s, int agent, const float *x0, const float *u_warm, uint64_t seed);

/* Queues a request (copies it, including *x0); returns at once with its
 * ticket.  Errors: INVALID_ARG (sizes, parameters, or a request whose scratch
 * exceeds the whole pool). */
int pi_server_submit(pi_server *s, const pi_serve_request *req, uint64_t *ticket);

/* Cancels a request that is still queued: it never reaches the GPU, its
 * agent's state and counter are untouched, and a completion record with status
 * PI_ERR_CANCELLED is queued for it.  PI_ERR_BUSY if the request is already on
 * the GPU or finished; PI_ERR_INVALID_ARG for an unknown ticket. */
int pi_server_cancel(pi_server *s, uint64_t ticket);

/* Moves up to max completion records into out (oldest first), waiting up to
 * timeout_us microseconds for the first one (0 = do not wait); *n_out = count. */
int pi_server_poll(pi_server *s, pi_serve_done *out, int max, int64_t timeout_us, int *n_out);

/* Copies a kept result and releases it: u_out [T][4] (host) and, if the server
 * keeps costs, costs [K] (host, may be NULL).  INVALID_ARG if the ticket has no
 * kept result (unknown, not finished, not kept, or already fetched). */
int pi_server_result(pi_server *s, uint64_t ticket, float *u_out, float *costs);

/* Waits until nothing is queued or on the GPU; PI_ERR_TIMEOUT after timeout_ms. */
int pi_server_drain(pi_server *s, int64_t timeout_ms);

/* Replays a trace in real time (arrivals sorted by t_ns) in the calling
 * thread: an arrival whose agent still waits for its previous result is
 * dropped (a controller that has no new plan yet keeps its old one); the rest
 * are submitted with the parameters of proto (agent, K, T and x0 taken from
 * the arrival / the device state, results not kept).  Returns when every
 * submitted request has completed.  done [n] receives the completion records
 * in completion order; *n_done and *n_dropped count them.  The server must
 * be idle when the replay starts (else PI_ERR_BUSY); PI_ERR_TIMEOUT if no
 * request completes for 60 s. */
int pi_server_replay(pi_server *s, const pi_serve_arrival *arrivals, int n, const pi_serve_request *proto,
                     pi_serve_done *done, int *n_done, int *n_dropped);

/* Checkpoint / resume of every agent's state (host arrays): x0 [n][12],
 * plan [n][T_max][4], counter [n], seed [n].  The server must be idle
 * (PI_ERR_BUSY otherwise).  Synchronous. */
int pi_server_state_save(pi_server *s, float *x0, float *u_warm, uint64_t *counter, uint64_t *seed);
int pi_server_state_load(pi_server *s, const float *x0, const float *u_warm, const uint64_t *counter,
                         const uint64_t *seed);

int pi_server_get_stats(const pi_server *s, pi_server_stats *out);

/* Stops the scheduler, waits for the groups on the GPU, drops queued requests
 * and frees the server.  NULL is accepted. */
void pi_server_destroy(pi_server *s);

/* Measured issue rates of the pipes the FP32 form leans on, on `device`: packed
 * FP32 FMA (FFMA2) in TFLOP/s and the MUFU base-2 exponential in results/s.
 * Independent dependency chains on every SM, CUDA-event timed; synchronous.
 * Context for the roofline (the paper has no counterpart). */
int pi_debug_pipe_rates(int device, double *ffma_tflops, double *ex2_per_s);

/* Measured FP64 FMA rate of `device` in lane results per second (each is 2
 * flop): independent DFMA chains on every SM, CUDA-event timed; synchronous.
 * The denominator of the cost-to-go scan's roofline, which B300's low FP64
 * throughput bounds. */
int pi_debug_fp64_rate(int device, double *dfma_per_s);

/* Host-only ABI check (no GPU): writes, for the public structs in this order
 * -- pi_lwpr_params, pi_cost_params, pi_opts, pi_batch_item, pi_server_opts,
 * pi_serve_request, pi_serve_done, pi_serve_arrival, pi_server_stats -- their
 * sizeof followed by the byte offset of each member in declaration order, into
 * out [max]; *n = entries written.  INVALID_ARG if max is too small. */
int pi_debug_struct_layout(size_t *out, int max, int *n);

/* Host-only check of the server's pool allocator (no GPU): runs n operations
 * on a pool of `capacity` bytes -- op[i] = 1 allocates size[i] bytes, op[i] = 0
 * frees the block allocated by operation size[i] -- and writes each
 * allocation's offset (or -1 if it did not fit) to offset[i] and, at the end,
 * the number of free extents to *free_extents. */
int pi_debug_pool(size_t capacity, const int *op, const size_t *size, int n, int64_t *offset, int *free_extents);

/* Synchronizes the context's stream and reports device-side errors raised by
 * earlier work: PI_ERR_TIMEOUT if a bounded wait in a kernel expired (the
 * kernel returned early and its outputs are invalid), PI_ERR_INTERNAL for a
 * failed device-side check.  Clears the device error word. */
int pi_sync(pi_ctx *ctx);

/* Frees the context and its device memory (synchronizes its stream first).
 * NULL is accepted. */
void pi_destroy(pi_ctx *ctx);

/* Message of the last error on the calling thread ("" if none). */
const char *pi_last_error(void);

/* Number of kernel launches enqueued through this context since creation. */
uint64_t pi_launch_count(const pi_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Staged entry points (same device code as pi_update, exposed for parity
 * tests of each step).  All pointers are device pointers; asynchronous on the
 * context's stream (pi_debug_noise / pi_debug_normals take a stream).
 * ------------------------------------------------------------------------- */

/* Raw Philox4x32-10 blocks: raw[k][t][blk][4] = Philox(counter (k, t, blk,
 * blk == 0 ? 0 : m), key (seed lo, seed hi)), blk = 0..3. */
int pi_debug_noise(uint64_t seed, int K, int T, int m, uint32_t *raw, void *stream);

/* Standard normals from those blocks by Box-Muller on (u0,u1), (u2,u3) with
 * u = (2 (r >> 9) + 1) 2^-24: ctrl[k][t][4] from block 0, model[k][t][12] from
 * blocks 1..3. */
int pi_debug_normals(uint64_t seed, int K, int T, int m, float *ctrl, float *model, void *stream);

/* LWPR prediction (Eq. 1) of the context's model at n inputs:
 * z [n][16] -> y [n][12], var [n][12]. */
int pi_debug_lwpr(pi_ctx *ctx, const float *z, int n, float *y, float *var);

/* Rollout stage only: writes cost [T][K] (running cost averaged over the
 * sub-rollouts), eps [T][K][4] and phi [K] (terminal cost, averaged). */
int pi_debug_rollout(pi_ctx *ctx, const float *x0, const float *u_nominal, int K, int T,
                     const float *sigma_u, uint64_t seed, float *cost, float *eps, float *phi);

/* Cost-to-go and weighted-average stage only, from given cost [T][K],
 * phi [K], eps [T][K][4]: writes u_out [T][4] and costs_out [K]. */
int pi_debug_reduce(pi_ctx *ctx, const float *cost, const float *phi, const float *eps,
                    const float *u_nominal, int K, int T, float lambda, float *u_out,
                    float *costs_out);

/* Failure path of the device-side waits, exercised without a fault: one
 * kernel waits on an mbarrier that no thread arrives at, using the same
 * bounded wait as every kernel, with a limit of limit_ns nanoseconds
 * (1e3 .. 1e9).  The wait gives up, the kernel flags the timeout in the
 * context's device error word and returns, so the next pi_sync reports
 * PI_ERR_TIMEOUT and the context stays usable.  Asynchronous on the
 * context's stream. */
int pi_debug_wait_timeout(pi_ctx *ctx, int64_t limit_ns);

/* The launch an FP32 update of K rollouts (with the context's M and split
 * mode) would use: *plain_blocks 64-slot blocks one CTA each, then, if
 * *units_per_cta > 0, the remaining blocks as the output-split launch of
 * *ctas CTAs with that many (block, output) units each (*ctas = 0 when there
 * is no split launch).  Host only; INVALID_ARG on a tensor-core context or
 * K < 1. */
int pi_debug_split_plan(pi_ctx *ctx, int K, int *plain_blocks, int *units_per_cta, int *ctas);

/* The same plan computed on the host alone, with no context and no GPU: K
 * rollouts of M sub-rollouts, L fields per output, n_sm SMs, split mode
 * `mode` (an exchange area of n_sm blocks, as pi_create allocates).  For
 * checking the planning rules without a device.  Errors: INVALID_ARG. */
int pi_debug_split_plan_sizes(int K, int M, int L, int n_sm, int mode, int *plain_blocks, int *units_per_cta,
                              int *ctas);

/* The work of CTA `cta` of a split launch over `blocks` 64-slot blocks with
 * units_per_cta (block, output) units per CTA, as the kernel computes it (the
 * same code, run on the host): *n_seg segments (1 or 2) in evaluation order,
 * seg[5 i + 0..4] = {block (relative to the split's first), first output,
 * output past the last, owned (1: this CTA steps the block's dynamics),
 * owned ? the number of earlier CTAs holding outputs of the block : this CTA's
 * index among them}.  seg holds 10 ints.  Host only.  Errors: INVALID_ARG. */
int pi_debug_split_partition(int blocks, int units_per_cta, int cta, int *seg, int *n_seg);

/* Failure path of the output-split launch's waits between CTAs, exercised
 * without a fault: with drop = 1 the next split launches leave out their last
 * CTA, so the flags it would set are never set.  The CTAs that wait on it give
 * up after the bounded wait (2 s), tell the others through the exchange area,
 * and all return; pi_sync then reports PI_ERR_TIMEOUT and the context stays
 * usable.  With drop = 2 the split launches are treated as refused by the
 * runtime (cudaErrorCooperativeLaunchTooLarge, which is what a process gets
 * when fewer SMs are open to it than the device has, under MPS or green
 * contexts), so the fallback runs: those blocks go to the plain launch, with
 * the same results.  drop = 0 restores full launches.  Errors: INVALID_ARG
 * (drop). */
int pi_debug_split_drop_cta(pi_ctx *ctx, int drop);

/* Tensor-core GEMM core of the tensor-core form, checked on its own:
 * D [128][64] f32 = A [128][K] x B [64][K]^T with A, B fp16 (IEEE binary16,
 * row-major, device), K a multiple of 16 in [16, 160].  One CTA; operands are
 * staged in shared memory in the K-major core-matrix layout and multiplied by
 * tcgen05.mma into tensor memory.  Device errors are reported by pi_sync. */
int pi_debug_tc_gemm(pi_ctx *ctx, const void *A, const void *B, int K, float *D);

#ifdef __cplusplus
}
#endif

#endif /* PI2RH_H */

// batch.cu -- many independent controllers of uneven size (K, T, L, M) updated
// together: one persistent rollout launch over a work list of (controller,
// slot block) items, one batched cost-to-go/LSE launch and one batched merge
// launch, captured once in a CUDA graph and replayed on every update.
//
// The work list is ordered by the schedule (longest item first by default, so
// the persistent CTAs finish together); the per-controller arguments live in
// a device table that each update refreshes (seeds, noise scales, lambda)
// before replaying the graph, so the graph itself never changes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "pi2rh.h"
#include "pi2rh_ctx.h"
#include "pi2rh_kernels.h"

using namespace pi2rh;

struct pi_batch {
    int device = 0;
    int n = 0;
    int form = PI_PRECISION_FP32;
    int order = PI_BATCH_ORDER_LONGEST_FIRST;
    int grid = 0;
    int split = 0;                          // tensor-core tile shape: 0 persistent, 1..4 outputs split
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;          // private stream used for capture and replay
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<pi_batch_item> items;
    // device tables
    void *d_args = nullptr;                 // RolloutArgs[n] or TcArgs[n]
    ReduceArgs *d_rargs = nullptr;
    int2 *d_ritems = nullptr, *d_sitems = nullptr, *d_mitems = nullptr;
    int *d_counter = nullptr;
    int n_ritems = 0, n_sitems = 0, n_mitems = 0;
    unsigned char *d_arena = nullptr;       // per-controller scratch
    // host copies refreshed per update
    std::vector<RolloutArgs> h_args;
    std::vector<TcArgs> h_targs;
    std::vector<ReduceArgs> h_rargs;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;
};

namespace {

int bfail(int code, const std::string &m) { return pi2rh_fail(code, m.c_str()); }

int bcuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PI_OK;
    return bfail(e == cudaErrorMemoryAllocation ? PI_ERR_OOM : PI_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define B_TRY(x)                     \
    do {                             \
        int rc_ = (x);               \
        if (rc_ != PI_OK) return rc_; \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int slots_per_block(int form) { return pi2rh_is_tc(form) ? TC_SLOTS : RF_SLOTS; }

// Relative cost of one rollout block of controller i (stage or tile count per step x steps).
double block_work(const pi_batch *b, int i)
{
    const pi_ctx *c = b->items[i].ctx;
    const double per_step = pi2rh_is_tc(b->form) ? (double)c->tiles_per_out : (double)c->spo;
    return per_step * b->items[i].T;
}

void build_rollout_items(pi_batch *b, std::vector<int2> &out)
{
    out.clear();
    const int spb = slots_per_block(b->form);
    for (int i = 0; i < b->n; ++i) {
        const long long slots = (long long)b->items[i].K * b->items[i].ctx->opts.M;
        const int nb = (int)((slots + spb - 1) / spb);
        for (int j = 0; j < nb; ++j) out.push_back(make_int2(i, j));
    }
    if (b->order == PI_BATCH_ORDER_LONGEST_FIRST) {
        std::stable_sort(out.begin(), out.end(),
                         [&](const int2 &x, const int2 &y) { return block_work(b, x.x) > block_work(b, y.x); });
    } else if (b->order == PI_BATCH_ORDER_ROUND_ROBIN) {
        // one block of each controller in turn
        std::vector<std::vector<int2>> per(b->n);
        for (const int2 &it : out) per[it.x].push_back(it);
        out.clear();
        for (size_t r = 0;; ++r) {
            bool any = false;
            for (int i = 0; i < b->n; ++i)
                if (r < per[i].size()) {
                    out.push_back(per[i][r]);
                    any = true;
                }
            if (!any) break;
        }
    }
}

int capture(pi_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    B_TRY(bcuda(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed), "begin capture"));
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) {
        if (pi2rh_is_tc(b->form)) {
            TcBatchArgs tb{static_cast<const TcArgs *>(b->d_args), b->d_ritems, b->n_ritems, b->d_counter,
                           pi2rh_tc_qprod(b->form)};
            e = b->split > 0 ? launch_rollout_tc_group(tb, b->split, b->stream)
                             : launch_rollout_tc_batch(tb, b->grid, b->stream);
        } else {
            BatchArgs fb{static_cast<const RolloutArgs *>(b->d_args), b->d_ritems, b->n_ritems, b->d_counter,
                         b->items[0].ctx->d_err};
            e = b->split > 0 ? launch_rollout_fp32_group(fb, b->stream) : launch_rollout_fp32_batch(fb, b->grid, b->stream);
        }
    }
    if (e == cudaSuccess) e = launch_scan_lse_batch(b->d_rargs, b->d_sitems, b->n_sitems, b->stream);
    if (e == cudaSuccess) e = launch_lse_merge_batch(b->d_rargs, b->d_mitems, b->n_mitems, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bcuda(e, "batch launch during capture");
    }
    B_TRY(bcuda(e2, "end capture"));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    return bcuda(e, "graph instantiate");
}

int upload_items(pi_batch *b)
{
    std::vector<int2> ritems;
    build_rollout_items(b, ritems);
    b->n_ritems = (int)ritems.size();
    return bcuda(cudaMemcpy(b->d_ritems, ritems.data(), ritems.size() * sizeof(int2), cudaMemcpyHostToDevice),
                 "upload work list");
}

void free_batch(pi_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    void *ptrs[] = {b->d_args, b->d_rargs, b->d_ritems, b->d_sitems, b->d_mitems, b->d_counter, b->d_arena};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
}

}  // namespace

extern "C" {

int pi_batch_create(const pi_batch_item *items, int n, int precision, pi_batch **out)
{
    if (!out) return bfail(PI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!items || n < 1) return bfail(PI_ERR_INVALID_ARG, "a batch needs at least one item");
    if (precision != PI_PRECISION_FP32 && !pi2rh_is_tc(precision))
        return bfail(PI_ERR_UNSUPPORTED, "unknown precision");
    const int dev = items[0].ctx ? items[0].ctx->device : 0;
    for (int i = 0; i < n; ++i) {
        const pi_batch_item &it = items[i];
        if (!it.ctx || !it.x0 || !it.u_nominal || !it.u_out || !it.costs_out)
            return bfail(PI_ERR_INVALID_ARG, "item " + std::to_string(i) + ": NULL context or buffer");
        if (it.K < 1 || it.T < 1 || (long long)it.K * it.ctx->opts.M > (1LL << 31) - 1)
            return bfail(PI_ERR_INVALID_ARG, "item " + std::to_string(i) + ": bad K or T");
        if (it.ctx->device != dev) return bfail(PI_ERR_INVALID_ARG, "all contexts must share one device");
        if (pi2rh_is_tc(precision) && (!it.ctx->d_wtiles || it.ctx->opts.precision != precision))
            return bfail(PI_ERR_INVALID_ARG, "item " + std::to_string(i) +
                                                 ": a tensor-core batch needs contexts created with the batch's precision");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return bfail(PI_ERR_CUDA, "cudaSetDevice");
    pi_batch *b = new pi_batch();
    b->device = dev;
    b->n = n;
    b->form = precision;
    b->items.assign(items, items + n);
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = sms;
    auto bail = [&](int rc) {
        free_batch(b);
        delete b;
        if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        return rc;
    };
    int rc;
    // scratch arena: per controller cost [T][K], eps [T][K], phi [K], partials [nblk][T][6]
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const size_t K = items[i].K, T = items[i].T, nblk = (K + RS_KC - 1) / RS_KC;
        off[i] = total;
        total += align256(K * T * 4) + align256(K * T * 16) + align256(K * 4) + align256(nblk * T * 48);
    }
    if ((rc = bcuda(cudaMalloc(&b->d_arena, total), "batch scratch"))) return bail(rc);
    if ((rc = bcuda(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "batch stream"))) return bail(rc);
    if ((rc = bcuda(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "event"))) return bail(rc);
    if ((rc = bcuda(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming), "event"))) return bail(rc);
    b->h_args.resize(n);
    b->h_targs.resize(n);
    b->h_rargs.resize(n);
    std::vector<int2> sitems, mitems;
    for (int i = 0; i < n; ++i) {
        const pi_batch_item &it = items[i];
        const pi_ctx *c = it.ctx;
        unsigned char *base = b->d_arena + off[i];
        const size_t K = it.K, T = it.T;
        float *cost = reinterpret_cast<float *>(base);
        float4 *eps = reinterpret_cast<float4 *>(base + align256(K * T * 4));
        float *phi = reinterpret_cast<float *>(base + align256(K * T * 4) + align256(K * T * 16));
        double *part = reinterpret_cast<double *>(base + align256(K * T * 4) + align256(K * T * 16) + align256(K * 4));
        RolloutArgs &a = b->h_args[i];
        a = ctx_rollout_args(c);
        a.K = it.K;
        a.T = it.T;
        a.x0 = it.x0;
        a.u_nom = it.u_nominal;
        a.cost_tk = cost;
        a.eps_tk = eps;
        a.phi = phi;
        TcArgs &t = b->h_targs[i];
        t = ctx_tc_args(c);
        t.K = it.K;
        t.T = it.T;
        t.x0 = it.x0;
        t.u_nom = it.u_nominal;
        t.cost_tk = cost;
        t.eps_tk = eps;
        t.phi = phi;
        ReduceArgs &r = b->h_rargs[i];
        r = ReduceArgs{cost, phi, eps, it.K, it.T, (double)c->dt, 1.0, it.costs_out, part, it.u_nominal, it.u_out};
        const int nblk = scan_blocks(it.K);
        for (int j = 0; j < nblk; ++j) sitems.push_back(make_int2(i, j));
        for (int j = 0; j < it.T; j += 8) mitems.push_back(make_int2(i, j));
    }
    b->n_sitems = (int)sitems.size();
    b->n_mitems = (int)mitems.size();
    const size_t arg_bytes = pi2rh_is_tc(precision) ? n * sizeof(TcArgs) : n * sizeof(RolloutArgs);
    size_t max_ritems = 0;
    for (int i = 0; i < n; ++i)
        max_ritems += ((size_t)items[i].K * items[i].ctx->opts.M + RF_SLOTS - 1) / RF_SLOTS;
    if ((rc = bcuda(cudaMalloc(&b->d_args, arg_bytes), "batch tables"))) return bail(rc);
    if ((rc = bcuda(cudaMalloc(&b->d_rargs, n * sizeof(ReduceArgs)), "batch tables"))) return bail(rc);
    if ((rc = bcuda(cudaMalloc(&b->d_ritems, max_ritems * sizeof(int2)), "batch tables"))) return bail(rc);
    if ((rc = bcuda(cudaMalloc(&b->d_sitems, sitems.size() * sizeof(int2)), "batch tables"))) return bail(rc);
    if ((rc = bcuda(cudaMalloc(&b->d_mitems, mitems.size() * sizeof(int2)), "batch tables"))) return bail(rc);
    if ((rc = bcuda(cudaMalloc(&b->d_counter, sizeof(int)), "batch tables"))) return bail(rc);
    if ((rc = bcuda(cudaMemcpy(b->d_sitems, sitems.data(), sitems.size() * sizeof(int2), cudaMemcpyHostToDevice),
                    "upload"))) return bail(rc);
    if ((rc = bcuda(cudaMemcpy(b->d_mitems, mitems.data(), mitems.size() * sizeof(int2), cudaMemcpyHostToDevice),
                    "upload"))) return bail(rc);
    if ((rc = upload_items(b))) return bail(rc);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    *out = b;
    return PI_OK;
}

int pi_batch_set_schedule(pi_batch *b, int order, int grid)
{
    if (!b) return bfail(PI_ERR_INVALID_ARG, "batch is NULL");
    if (order < PI_BATCH_ORDER_AS_GIVEN || order > PI_BATCH_ORDER_ROUND_ROBIN || grid < 0)
        return bfail(PI_ERR_INVALID_ARG, "bad schedule");
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->order = order;
    b->grid = grid == 0 ? sms : grid;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    int rc = upload_items(b);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return rc;
}

int pi_batch_set_tile(pi_batch *b, int split)
{
    if (!b) return bfail(PI_ERR_INVALID_ARG, "batch is NULL");
    if (split < 0 || split > 4)
        return bfail(PI_ERR_INVALID_ARG, "split must be 0..4");
    if (split > 1 && !pi2rh_is_tc(b->form))
        return bfail(PI_ERR_INVALID_ARG, "FP32 batches take tile shape 0 or 1 (outputs are not split)");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->split = split;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return PI_OK;
}

int pi_batch_set_stream(pi_batch *b, void *stream)
{
    if (!b) return bfail(PI_ERR_INVALID_ARG, "batch is NULL");
    b->user_stream = (cudaStream_t)stream;
    return PI_OK;
}

int pi_batch_update(pi_batch *b, const float *lambda, const float *sigma_u, const uint64_t *seed)
{
    if (!b) return bfail(PI_ERR_INVALID_ARG, "batch is NULL");
    if (!lambda || !sigma_u || !seed) return bfail(PI_ERR_INVALID_ARG, "NULL parameter array");
    for (int i = 0; i < b->n; ++i) {
        if (!(lambda[i] > 0.0f) || !std::isfinite(lambda[i]))
            return bfail(PI_ERR_INVALID_ARG, "lambda[" + std::to_string(i) + "] must be finite and > 0");
        for (int j = 0; j < 4; ++j)
            if (!std::isfinite(sigma_u[4 * i + j]) || sigma_u[4 * i + j] < 0.0f)
                return bfail(PI_ERR_INVALID_ARG, "sigma_u of item " + std::to_string(i) + " must be >= 0");
    }
    NvtxRange nv("pi_batch_update");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device && cudaSetDevice(b->device) != cudaSuccess) return bfail(PI_ERR_CUDA, "cudaSetDevice");
    for (int i = 0; i < b->n; ++i) {
        for (int j = 0; j < 4; ++j) {
            const float sq = sqrtf(sigma_u[4 * i + j]);
            b->h_args[i].sqrt_sigma_u[j] = sq;
            b->h_targs[i].sqrt_sigma_u[j] = sq;
        }
        b->h_args[i].seed = seed[i];
        b->h_targs[i].seed = seed[i];
        b->h_rargs[i].inv_lam_log2e = 1.4426950408889634074 / (double)lambda[i];
    }
    int rc = PI_OK;
    // order after the caller's stream, refresh the tables, replay, order the caller after us
    if (!rc) rc = bcuda(cudaEventRecord(b->ev_in, b->user_stream), "event record");
    if (!rc) rc = bcuda(cudaStreamWaitEvent(b->stream, b->ev_in, 0), "stream wait");
    const void *src = pi2rh_is_tc(b->form) ? (const void *)b->h_targs.data() : (const void *)b->h_args.data();
    const size_t bytes = pi2rh_is_tc(b->form) ? b->n * sizeof(TcArgs) : b->n * sizeof(RolloutArgs);
    if (!rc) rc = bcuda(cudaMemcpyAsync(b->d_args, src, bytes, cudaMemcpyHostToDevice, b->stream), "upload arguments");
    if (!rc)
        rc = bcuda(cudaMemcpyAsync(b->d_rargs, b->h_rargs.data(), b->n * sizeof(ReduceArgs), cudaMemcpyHostToDevice,
                                   b->stream),
                   "upload arguments");
    if (!rc && !b->exec) rc = capture(b);
    if (!rc) rc = bcuda(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    if (!rc) rc = bcuda(cudaEventRecord(b->ev_out, b->stream), "event record");
    if (!rc) rc = bcuda(cudaStreamWaitEvent(b->user_stream, b->ev_out, 0), "stream wait");
    if (!rc) b->launches += 3;
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return rc;
}

int pi_batch_sync(pi_batch *b)
{
    if (!b) return bfail(PI_ERR_INVALID_ARG, "batch is NULL");
    int rc = bcuda(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (rc) return rc;
    for (int i = 0; i < b->n; ++i) {
        rc = pi_sync(b->items[i].ctx);
        if (rc) return rc;
    }
    return PI_OK;
}

uint64_t pi_batch_launch_count(const pi_batch *b) { return b ? b->launches : 0; }

void pi_batch_destroy(pi_batch *b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    delete b;
}

}  // extern "C"

// serve.cu -- serving engine: continuous batching of receding-horizon control
// updates (Sec. 3.1, PI^2-RH) of many simulated vehicles over one shared LWPR
// model and cost.
//
// Threads: callers only queue requests and read completions; one scheduler
// thread per server owns every CUDA call on the launch lanes.  One scheduler
// pass
//   1. retires lanes: when a lane's result event has fired, the group's
//      results (already in pinned host memory) become completion records;
//      when its done event has fired, the group's pool blocks are released
//      and its agents become free again;
//   2. admits queued requests in arrival order into a group while a lane is
//      free: a request whose agent is busy (or already in the group) is
//      skipped without holding back later ones; a request whose scratch does
//      not fit the pool ends the pass (first come, first served on memory);
//   3. launches the group on the free lane: table upload, seed/state prologue,
//      one batched rollout launch over all (request, slot block) items in
//      longest-first order, the batched cost-to-go and merge
//      launches, the copy of the plans to the host, and the receding-horizon
//      advance of every agent of the group (plant step on the LWPR mean,
//      shifted warm start, counter + 1).
// Groups on different lanes overlap on the device: the CTAs of a later
// group's kernels take the SMs that an earlier group's CTAs leave.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pi2rh.h"
#include "pi2rh_ctx.h"
#include "pi2rh_kernels.h"

using namespace pi2rh;

namespace {

constexpr uint64_t SEED_STEP = 0x9E3779B97F4A7C15ull;   // Weyl increment between an agent's updates
constexpr int POLL_US = 20;                             // scheduler poll period while groups are on the GPU
constexpr int64_t REPLAY_STALL_NS = 60LL * 1000 * 1000 * 1000;

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

int sfail(int code, const std::string &m) { return pi2rh_fail(code, m.c_str()); }

int scuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PI_OK;
    return sfail(e == cudaErrorMemoryAllocation ? PI_ERR_OOM : PI_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

// First-fit allocator over [0, capacity) in 256-byte units; freed blocks are
// merged with their free neighbours.
class Pool {
  public:
    static constexpr size_t NONE = SIZE_MAX;
    explicit Pool(size_t cap = 0) { reset(cap); }
    void reset(size_t cap)
    {
        cap_ = cap & ~(size_t)255;
        free_.clear();
        if (cap_) free_[0] = cap_;
        used_ = peak_ = 0;
    }
    size_t alloc(size_t n)
    {
        n = al256(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            used_ += n;
            peak_ = std::max(peak_, used_);
            return off;
        }
        return NONE;
    }
    void release(size_t off, size_t n)
    {
        n = al256(n ? n : 1);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t capacity() const { return cap_; }
    size_t peak() const { return peak_; }
    int extents() const { return (int)free_.size(); }

  private:
    size_t cap_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length
};

// Device view of one request of a group.
struct ServeItem {
    int agent;
    int T;
    const float *u_out;   // [T][4] plan computed by the group
    int has_x0;           // 1: x0_in[i] replaces the agent's state before the update
};

// Scratch of one request inside the pool: cost [T][K], eps [T][K] (float4),
// phi [K], LSE partials [nblk][T][6] (f64), then u_out [T][4] and costs [K]
// back to back (one copy to the host).
struct ReqLayout {
    size_t cost, eps, phi, part, uout, total;
};

ReqLayout req_layout(int K, int T)
{
    const size_t k = K, t = T, nblk = scan_blocks(K);
    ReqLayout l{};
    l.cost = 0;
    l.eps = l.cost + al256(k * t * 4);
    l.phi = l.eps + al256(k * t * 16);
    l.part = l.phi + al256(k * 4);
    l.uout = l.part + al256(nblk * t * 48);
    l.total = l.uout + al256(t * 16 + k * 4);
    return l;
}

struct Req {
    uint64_t ticket = 0;
    pi_serve_request q{};
    float x0[NX] = {};
    bool has_x0 = false;
    int64_t t_submit = 0, t_launch = 0;
    size_t off = Pool::NONE, bytes = 0;
    int group_size = 0;
};

// ---------------------------------------------------------------------------
// Serving kernels (launch-sized: one CTA per request of a group).
// ---------------------------------------------------------------------------

// Seed of each request from its agent's device-resident counter, and the
// optional measured state written over the agent's state.
__global__ void serve_prep(unsigned char *args, int arg_stride, int seed_off, const ServeItem *items,
                           const float *x0_in, float *x0, const uint64_t *agent_seed, const uint64_t *ctr)
{
    const int i = blockIdx.x, c = threadIdx.x;
    const ServeItem it = items[i];
    if (c == 0)
        *reinterpret_cast<uint64_t *>(args + (size_t)i * arg_stride + seed_off) =
            agent_seed[it.agent] + ctr[it.agent] * SEED_STEP;
    if (it.has_x0 && c < NX) x0[(size_t)it.agent * NX + c] = x0_in[(size_t)i * NX + c];
}

// Plant-step input z = [x0, u_out_0] of every request.
__global__ void serve_build_z(const ServeItem *items, const float *x0, float *z)
{
    const int i = blockIdx.x, c = threadIdx.x;
    const ServeItem it = items[i];
    if (c < NX) z[(size_t)i * NZ + c] = x0[(size_t)it.agent * NX + c];
    else if (c < NZ) z[(size_t)i * NZ + c] = it.u_out[c - NX];
}

// Receding-horizon advance of every agent of the group: x0 += dt * f_mean(z),
// plan[t] = u_out[min(t + 1, T - 1)] for t < T_max, counter + 1.
__global__ void serve_apply(const ServeItem *items, const float *y, float dt, float *x0, float *warm, int T_max,
                            uint64_t *ctr)
{
    const int i = blockIdx.x;
    const ServeItem it = items[i];
    float *w = warm + (size_t)it.agent * T_max * NU;
    for (int j = threadIdx.x; j < T_max * NU; j += blockDim.x) {
        const int t = j / NU, c = j % NU;
        const int src = t + 1 < it.T ? t + 1 : it.T - 1;
        w[j] = it.u_out[src * NU + c];
    }
    if (threadIdx.x < NX) {
        float *xa = x0 + (size_t)it.agent * NX;
        xa[threadIdx.x] = fmaf(dt, y[(size_t)i * NY + threadIdx.x], xa[threadIdx.x]);
    }
    if (threadIdx.x == 0) ctr[it.agent] += 1;
}

// Per-lane device and pinned-host table layout (byte offsets).
struct Layout {
    size_t args, rargs, items, x0, ritems, sitems, mitems, upload_end;   // uploaded from the pinned mirror
    size_t ctl, z, y, var, total;                                         // device only
    int arg_stride;
    size_t res_stride;   // floats per request in the pinned result block
    size_t res_bytes;    // whole pinned result block (plus two error words)
};

struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_result = nullptr, ev_done = nullptr;
    unsigned char *d = nullptr;   // device tables
    unsigned char *h = nullptr;   // pinned mirror of the uploaded tables
    float *h_res = nullptr;       // pinned results (+ error words at the end)
    std::vector<Req> group;
    bool busy = false, result_seen = false;
};

}  // namespace

struct pi_server {
    pi_ctx *ctx = nullptr;
    pi_server_opts o{};
    int device = 0, form = PI_PRECISION_FP32, sms = 148, M = 1;
    Layout lay{};
    int max_ritems = 0, max_sitems = 0, max_mitems = 0;
    // device-resident agent state
    float *d_x0 = nullptr, *d_warm = nullptr;
    uint64_t *d_ctr = nullptr, *d_seed = nullptr;
    unsigned char *d_pool = nullptr;
    Pool pool;
    std::vector<Lane> lanes;
    // host state (guarded by mu)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::list<Req> pending;
    std::deque<pi_serve_done> done_q;
    struct Kept {
        int T, K;
        std::vector<float> v;   // plan [T][4], then costs [K] when the server keeps costs
    };
    std::unordered_map<uint64_t, Kept> results;
    std::vector<int> agent_busy;          // request of the agent on the GPU
    std::vector<int> agent_outstanding;   // queued + on the GPU
    std::vector<uint32_t> mark;
    uint32_t pass = 0;
    uint64_t next_ticket = 0;
    int inflight_reqs = 0;
    int sticky = PI_OK;                   // a failed advance step poisons later results
    pi_server_stats st{};
    bool stop = false;
    std::thread worker;

    int lane_free() const
    {
        for (size_t i = 0; i < lanes.size(); ++i)
            if (!lanes[i].busy) return (int)i;
        return -1;
    }
    bool any_busy() const
    {
        for (const Lane &l : lanes)
            if (l.busy) return true;
        return false;
    }
    bool idle() const { return pending.empty() && !any_busy(); }

    int launch(Lane &L);
    bool retire();
    bool admit();
    void run();
    void enqueue_locked(Req &&r);
};

namespace {

int status_of(int err_word)
{
    if (!err_word) return PI_OK;
    if (err_word & (DEVERR_TIMEOUT_FULL | DEVERR_TIMEOUT_EMPTY | DEVERR_TIMEOUT_DRAIN)) return PI_ERR_TIMEOUT;
    return PI_ERR_INTERNAL;
}

}  // namespace

// Fills the lane's tables for its group and enqueues the whole group update.
int pi_server::launch(Lane &L)
{
    NvtxRange nv("pi_server group launch");
    const int n = (int)L.group.size();
    const bool tc = pi2rh_is_tc(form);
    const int spb = tc ? TC_SLOTS : RF_SLOTS;
    std::stable_sort(L.group.begin(), L.group.end(), [](const Req &a, const Req &b) { return a.q.T > b.q.T; });
    unsigned char *h = L.h, *d = L.d;
    int *d_ctl = reinterpret_cast<int *>(d + lay.ctl);   // [0] work counter, [1] error word, [2] advance error word
    int2 *hr = reinterpret_cast<int2 *>(h + lay.ritems);
    int2 *hs = reinterpret_cast<int2 *>(h + lay.sitems);
    int2 *hm = reinterpret_cast<int2 *>(h + lay.mitems);
    int nr = 0, ns = 0, nm = 0, nx = 0;
    const int64_t t_launch = now_ns();
    const float dt = ctx->dt;
    for (int i = 0; i < n; ++i) {
        Req &r = L.group[i];
        r.t_launch = t_launch;
        r.group_size = n;
        const int a = r.q.agent, K = r.q.K, T = r.q.T;
        const ReqLayout rl = req_layout(K, T);
        unsigned char *base = d_pool + r.off;
        float *cost = reinterpret_cast<float *>(base + rl.cost);
        float4 *eps = reinterpret_cast<float4 *>(base + rl.eps);
        float *phi = reinterpret_cast<float *>(base + rl.phi);
        double *part = reinterpret_cast<double *>(base + rl.part);
        float *uout = reinterpret_cast<float *>(base + rl.uout);
        const float *x0p = d_x0 + (size_t)a * NX;
        const float *unom = d_warm + (size_t)a * o.T_max * NU;
        if (tc) {
            TcArgs t = ctx_tc_args(ctx);
            t.K = K;
            t.T = T;
            for (int j = 0; j < 4; ++j) t.sqrt_sigma_u[j] = sqrtf(r.q.sigma_u[j]);
            t.seed = 0;   // set on the device by serve_prep
            t.x0 = x0p;
            t.u_nom = unom;
            t.cost_tk = cost;
            t.eps_tk = eps;
            t.phi = phi;
            t.err = d_ctl + 1;
            std::memcpy(h + lay.args + (size_t)i * sizeof(TcArgs), &t, sizeof t);
        } else {
            RolloutArgs t = ctx_rollout_args(ctx);
            t.K = K;
            t.T = T;
            for (int j = 0; j < 4; ++j) t.sqrt_sigma_u[j] = sqrtf(r.q.sigma_u[j]);
            t.seed = 0;
            t.x0 = x0p;
            t.u_nom = unom;
            t.cost_tk = cost;
            t.eps_tk = eps;
            t.phi = phi;
            t.err = d_ctl + 1;
            std::memcpy(h + lay.args + (size_t)i * sizeof(RolloutArgs), &t, sizeof t);
        }
        const ReduceArgs ra{cost, phi, eps, K, T, (double)dt, 1.4426950408889634074 / (double)r.q.lambda,
                            uout + (size_t)T * NU, part, unom, uout};
        std::memcpy(h + lay.rargs + (size_t)i * sizeof(ReduceArgs), &ra, sizeof ra);
        const ServeItem si{a, T, uout, r.has_x0 ? 1 : 0};
        std::memcpy(h + lay.items + (size_t)i * sizeof(ServeItem), &si, sizeof si);
        if (r.has_x0) std::memcpy(h + lay.x0 + (size_t)i * NX * 4, r.x0, NX * 4);
        nx = r.has_x0 ? i + 1 : nx;
        const long long slots = (long long)K * M;
        const int nb = (int)((slots + spb - 1) / spb);
        for (int j = 0; j < nb; ++j) hr[nr++] = make_int2(i, j);
        for (int j = 0; j < scan_blocks(K); ++j) hs[ns++] = make_int2(i, j);
        for (int t = 0; t < T; t += 8) hm[nm++] = make_int2(i, t);
    }
    cudaStream_t s = L.stream;
    const size_t arg_bytes = (size_t)n * (tc ? sizeof(TcArgs) : sizeof(RolloutArgs));
    cudaError_t e = cudaMemsetAsync(d_ctl, 0, 4 * sizeof(int), s);
    auto up = [&](size_t off, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d + off, h + off, bytes, cudaMemcpyHostToDevice, s);
    };
    up(lay.args, arg_bytes);
    up(lay.rargs, (size_t)n * sizeof(ReduceArgs));
    up(lay.items, (size_t)n * sizeof(ServeItem));
    up(lay.x0, (size_t)nx * NX * 4);
    up(lay.ritems, (size_t)nr * sizeof(int2));
    up(lay.sitems, (size_t)ns * sizeof(int2));
    up(lay.mitems, (size_t)nm * sizeof(int2));
    const ServeItem *d_items = reinterpret_cast<const ServeItem *>(d + lay.items);
    if (e == cudaSuccess) {
        serve_prep<<<n, 32, 0, s>>>(d + lay.args, tc ? (int)sizeof(TcArgs) : (int)sizeof(RolloutArgs),
                                    tc ? (int)offsetof(TcArgs, seed) : (int)offsetof(RolloutArgs, seed), d_items,
                                    reinterpret_cast<const float *>(d + lay.x0), d_x0, d_seed, d_ctr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (tc) {
            TcBatchArgs tb{reinterpret_cast<const TcArgs *>(d + lay.args), reinterpret_cast<const int2 *>(d + lay.ritems),
                           nr, d_ctl, pi2rh_tc_qprod(form)};
            // one item per CTA (a plain launch: the block scheduler fills SMs as
            // items finish, also across lanes); a small group as one wave of
            // clusters that split each block's outputs
            e = launch_rollout_tc_group(tb, tc_group_split(nr), s);
        } else {
            BatchArgs fb{reinterpret_cast<const RolloutArgs *>(d + lay.args), reinterpret_cast<const int2 *>(d + lay.ritems),
                         nr, d_ctl, d_ctl + 1};
            e = launch_rollout_fp32_group(fb, s);   // one item per CTA
        }
    }
    const ReduceArgs *d_rargs = reinterpret_cast<const ReduceArgs *>(d + lay.rargs);
    if (e == cudaSuccess) e = launch_scan_lse_batch(d_rargs, reinterpret_cast<const int2 *>(d + lay.sitems), ns, s);
    if (e == cudaSuccess) e = launch_lse_merge_batch(d_rargs, reinterpret_cast<const int2 *>(d + lay.mitems), nm, s);
    // plans (and costs) to the host, then the error word of the update
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const Req &r = L.group[i];
        const ReqLayout rl = req_layout(r.q.K, r.q.T);
        const size_t nf = (size_t)r.q.T * NU + (o.want_costs ? (size_t)r.q.K : 0);
        e = cudaMemcpyAsync(L.h_res + (size_t)i * lay.res_stride, d_pool + r.off + rl.uout, nf * 4,
                            cudaMemcpyDeviceToHost, s);
    }
    int *h_err = reinterpret_cast<int *>(L.h_res + (size_t)o.max_group * lay.res_stride);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_err, d_ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(L.ev_result, s);
    // receding-horizon advance of the group's agents
    float *z = reinterpret_cast<float *>(d + lay.z);
    float *y = reinterpret_cast<float *>(d + lay.y);
    float *var = reinterpret_cast<float *>(d + lay.var);
    if (e == cudaSuccess) {
        serve_build_z<<<n, 32, 0, s>>>(d_items, d_x0, z);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        RolloutArgs pa = ctx_rollout_args(ctx);
        pa.M = 1;
        pa.z_in = z;
        pa.y_out = y;
        pa.var_out = var;
        pa.n_pred = n;
        pa.err = d_ctl + 2;
        e = launch_predict_fp32(pa, s);
    }
    if (e == cudaSuccess) {
        serve_apply<<<n, 128, 0, s>>>(d_items, y, dt, d_x0, d_warm, o.T_max, d_ctr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_err + 1, d_ctl + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(L.ev_done, s);
    st.launches += 7;
    st.groups += 1;
    st.peak_group_size = std::max(st.peak_group_size, n);
    L.busy = true;
    L.result_seen = false;
    if (e != cudaSuccess) {
        sfail(PI_ERR_CUDA, std::string("serving launch: ") + cudaGetErrorString(e));
        return PI_ERR_CUDA;
    }
    return PI_OK;
}

// Turns fired lane events into completion records and released resources.
bool pi_server::retire()
{
    bool progress = false;
    for (Lane &L : lanes) {
        if (!L.busy) continue;
        int *h_err = reinterpret_cast<int *>(L.h_res + (size_t)o.max_group * lay.res_stride);
        if (!L.result_seen) {
            const cudaError_t e = cudaEventQuery(L.ev_result);
            if (e == cudaErrorNotReady) continue;
            const int64_t t = now_ns();
            const int status = e != cudaSuccess ? PI_ERR_CUDA : sticky ? sticky : status_of(h_err[0]);
            for (size_t i = 0; i < L.group.size(); ++i) {
                const Req &r = L.group[i];
                pi_serve_done dn{};
                dn.ticket = r.ticket;
                dn.agent = r.q.agent;
                dn.K = r.q.K;
                dn.T = r.q.T;
                dn.status = status;
                dn.group_size = r.group_size;
                dn.t_submit_ns = r.t_submit;
                dn.t_launch_ns = r.t_launch;
                dn.t_result_ns = t;
                if (r.q.keep_result && status == PI_OK) {
                    const size_t nf = (size_t)r.q.T * NU + (o.want_costs ? (size_t)r.q.K : 0);
                    const float *src = L.h_res + i * lay.res_stride;
                    Kept &k = results[r.ticket];
                    k.T = r.q.T;
                    k.K = r.q.K;
                    k.v.assign(src, src + nf);
                }
                done_q.push_back(dn);
            }
            st.completed += L.group.size();
            L.result_seen = true;
            progress = true;
            cv_done.notify_all();
        }
        const cudaError_t e = cudaEventQuery(L.ev_done);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess || h_err[1]) sticky = e != cudaSuccess ? PI_ERR_CUDA : status_of(h_err[1]);
        for (const Req &r : L.group) {
            pool.release(r.off, r.bytes);
            agent_busy[r.q.agent] = 0;
            agent_outstanding[r.q.agent] -= 1;
        }
        inflight_reqs -= (int)L.group.size();
        L.group.clear();
        L.busy = false;
        progress = true;
        cv_done.notify_all();
    }
    return progress;
}

// Forms and launches groups while a lane is free and something fits.
bool pi_server::admit()
{
    bool progress = false;
    for (;;) {
        const int li = lane_free();
        if (li < 0 || pending.empty()) break;
        Lane &L = lanes[li];
        ++pass;
        for (auto it = pending.begin(); it != pending.end() && (int)L.group.size() < o.max_group;) {
            const int a = it->q.agent;
            if (agent_busy[a] || mark[a] == pass) {
                mark[a] = pass;   // keep the agent's later requests behind this one
                ++it;
                continue;
            }
            const size_t off = pool.alloc(it->bytes);
            if (off == Pool::NONE) {
                st.memory_waits += 1;
                break;
            }
            it->off = off;
            mark[a] = pass;
            agent_busy[a] = 1;
            L.group.push_back(std::move(*it));
            it = pending.erase(it);
        }
        if (L.group.empty()) break;
        inflight_reqs += (int)L.group.size();
        st.peak_inflight_requests = std::max(st.peak_inflight_requests, inflight_reqs);
        st.pool_peak_bytes = pool.peak();
        if (launch(L) != PI_OK) {
            // the lane's events may never fire: finish its group here with the error
            cudaStreamSynchronize(L.stream);
            const int64_t t = now_ns();
            for (const Req &r : L.group) {
                pi_serve_done dn{};
                dn.ticket = r.ticket;
                dn.agent = r.q.agent;
                dn.K = r.q.K;
                dn.T = r.q.T;
                dn.status = PI_ERR_CUDA;
                dn.group_size = (int)L.group.size();
                dn.t_submit_ns = r.t_submit;
                dn.t_launch_ns = r.t_launch;
                dn.t_result_ns = t;
                done_q.push_back(dn);
                pool.release(r.off, r.bytes);
                agent_busy[r.q.agent] = 0;
                agent_outstanding[r.q.agent] -= 1;
            }
            st.completed += L.group.size();
            inflight_reqs -= (int)L.group.size();
            L.group.clear();
            L.busy = false;
            sticky = PI_ERR_CUDA;
            cv_done.notify_all();
        }
        progress = true;
    }
    return progress;
}

void pi_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        bool progress = retire();
        progress = admit() || progress;
        if (progress) continue;
        if (any_busy()) cv_work.wait_for(lk, std::chrono::microseconds(POLL_US));
        else cv_work.wait(lk);
    }
}

void pi_server::enqueue_locked(Req &&r)
{
    r.ticket = ++next_ticket;
    r.t_submit = now_ns();
    agent_outstanding[r.q.agent] += 1;
    st.submitted += 1;
    pending.push_back(std::move(r));
    cv_work.notify_one();
}

namespace {

struct DevGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int check_request(const pi_server *s, const pi_serve_request &q)
{
    if (q.agent < 0 || q.agent >= s->o.n_agents) return sfail(PI_ERR_INVALID_ARG, "agent out of range");
    if (q.K < 1 || q.K > s->o.K_max || q.T < 1 || q.T > s->o.T_max)
        return sfail(PI_ERR_INVALID_ARG, "K or T outside [1, K_max] / [1, T_max]");
    if (!(q.lambda > 0.0f) || !std::isfinite(q.lambda)) return sfail(PI_ERR_INVALID_ARG, "lambda must be finite and > 0");
    for (int j = 0; j < 4; ++j)
        if (!std::isfinite(q.sigma_u[j]) || q.sigma_u[j] < 0.0f)
            return sfail(PI_ERR_INVALID_ARG, "sigma_u must be finite and >= 0");
    if (req_layout(q.K, q.T).total > s->pool.capacity())
        return sfail(PI_ERR_INVALID_ARG, "the request's scratch exceeds the whole HBM pool");
    return PI_OK;
}

void free_server(pi_server *s)
{
    for (Lane &L : s->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.d) cudaFree(L.d);
        if (L.h) cudaFreeHost(L.h);
        if (L.h_res) cudaFreeHost(L.h_res);
        if (L.ev_result) cudaEventDestroy(L.ev_result);
        if (L.ev_done) cudaEventDestroy(L.ev_done);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    void *ptrs[] = {s->d_x0, s->d_warm, s->d_ctr, s->d_seed, s->d_pool};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

extern "C" {

void pi_server_default_opts(pi_server_opts *o)
{
    if (!o) return;
    *o = pi_server_opts{};
    o->n_agents = 1;
    o->K_max = 16384;
    o->T_max = 128;
    o->max_inflight = 2;
    o->max_group = 64;
    o->hbm_budget = 0;
    o->want_costs = 0;
}

int pi_server_create(pi_ctx *ctx, const pi_server_opts *opts, pi_server **out)
{
    if (!out) return sfail(PI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx || !opts) return sfail(PI_ERR_INVALID_ARG, "ctx or opts is NULL");
    const pi_server_opts &o = *opts;
    if (o.n_agents < 1 || o.n_agents > (1 << 24) || o.K_max < 1 || o.K_max > (1 << 22) || o.T_max < 1 ||
        o.T_max > 65536 || o.max_inflight < 1 || o.max_inflight > 64 || o.max_group < 1 || o.max_group > 4096)
        return sfail(PI_ERR_INVALID_ARG, "server option out of range");
    if ((long long)o.K_max * ctx->opts.M > (1LL << 31) - 1) return sfail(PI_ERR_INVALID_ARG, "K_max * M too large");
    const int form = ctx->opts.precision;
    if (pi2rh_is_tc(form) && !ctx->d_wtiles)
        return sfail(PI_ERR_INVALID_ARG, "tensor-core context without coefficient tiles");
    DevGuard dg(ctx->device);
    if (dg.err != cudaSuccess) return scuda(dg.err, "cudaSetDevice");
    std::unique_ptr<pi_server> s(new pi_server());
    s->ctx = ctx;
    s->o = o;
    s->device = ctx->device;
    s->form = form;
    s->M = ctx->opts.M;
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    auto bail = [&](int rc) {
        free_server(s.get());
        return rc;
    };
    int rc;
    // pool ("admission by free HBM")
    size_t budget = o.hbm_budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        if ((rc = scuda(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo"))) return rc;
        budget = std::min(fr / 2, (size_t)32 << 30);
    }
    budget &= ~(size_t)255;
    if (budget < 256) return sfail(PI_ERR_INVALID_ARG, "HBM budget too small");
    if ((rc = scuda(cudaMalloc(&s->d_pool, budget), "serving pool"))) return bail(rc);
    s->pool.reset(budget);
    s->st.pool_bytes = s->pool.capacity();
    // agent state
    const size_t na = o.n_agents;
    if ((rc = scuda(cudaMalloc(&s->d_x0, na * NX * 4), "agent state"))) return bail(rc);
    if ((rc = scuda(cudaMalloc(&s->d_warm, na * o.T_max * NU * 4), "agent state"))) return bail(rc);
    if ((rc = scuda(cudaMalloc(&s->d_ctr, na * 8), "agent state"))) return bail(rc);
    if ((rc = scuda(cudaMalloc(&s->d_seed, na * 8), "agent state"))) return bail(rc);
    if ((rc = scuda(cudaMemset(s->d_x0, 0, na * NX * 4), "agent state"))) return bail(rc);
    if ((rc = scuda(cudaMemset(s->d_warm, 0, na * o.T_max * NU * 4), "agent state"))) return bail(rc);
    if ((rc = scuda(cudaMemset(s->d_ctr, 0, na * 8), "agent state"))) return bail(rc);
    {
        std::vector<uint64_t> seeds(na);
        for (size_t i = 0; i < na; ++i) seeds[i] = i;
        if ((rc = scuda(cudaMemcpy(s->d_seed, seeds.data(), na * 8, cudaMemcpyHostToDevice), "agent state")))
            return bail(rc);
    }
    // lane tables
    const int spb = pi2rh_is_tc(form) ? TC_SLOTS : RF_SLOTS;
    const long long g = o.max_group;
    const long long rblocks = ((long long)o.K_max * s->M + spb - 1) / spb;
    s->max_ritems = (int)std::min<long long>(g * rblocks, INT_MAX / 16);
    s->max_sitems = (int)std::min<long long>(g * scan_blocks(o.K_max), INT_MAX / 16);
    s->max_mitems = (int)std::min<long long>(g * ((o.T_max + 7) / 8), INT_MAX / 16);
    Layout &L = s->lay;
    const size_t argsz = std::max(sizeof(TcArgs), sizeof(RolloutArgs));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = al256(off + bytes);
        return at;
    };
    L.args = take(g * argsz);
    L.rargs = take(g * sizeof(ReduceArgs));
    L.items = take(g * sizeof(ServeItem));
    L.x0 = take(g * NX * 4);
    L.ritems = take((size_t)s->max_ritems * sizeof(int2));
    L.sitems = take((size_t)s->max_sitems * sizeof(int2));
    L.mitems = take((size_t)s->max_mitems * sizeof(int2));
    L.upload_end = off;
    L.ctl = take(4 * sizeof(int));
    L.z = take(g * NZ * 4);
    L.y = take(g * NY * 4);
    L.var = take(g * NY * 4);
    L.total = off;
    L.res_stride = (size_t)o.T_max * NU + (o.want_costs ? (size_t)o.K_max : 0);
    L.res_bytes = ((size_t)g * L.res_stride + 4) * 4;
    s->lanes.resize(o.max_inflight);
    for (Lane &ln : s->lanes) {
        if ((rc = scuda(cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking), "lane stream"))) return bail(rc);
        if ((rc = scuda(cudaEventCreateWithFlags(&ln.ev_result, cudaEventDisableTiming), "lane event"))) return bail(rc);
        if ((rc = scuda(cudaEventCreateWithFlags(&ln.ev_done, cudaEventDisableTiming), "lane event"))) return bail(rc);
        if ((rc = scuda(cudaMalloc(&ln.d, L.total), "lane tables"))) return bail(rc);
        if ((rc = scuda(cudaMallocHost(&ln.h, L.upload_end), "lane tables (pinned)"))) return bail(rc);
        if ((rc = scuda(cudaMallocHost(&ln.h_res, L.res_bytes), "lane results (pinned)"))) return bail(rc);
    }
    s->agent_busy.assign(na, 0);
    s->agent_outstanding.assign(na, 0);
    s->mark.assign(na, 0);
    try {
        s->worker = std::thread([srv = s.get()] { srv->run(); });
    } catch (const std::exception &ex) {
        free_server(s.get());
        return sfail(PI_ERR_INTERNAL, std::string("cannot start the scheduler thread: ") + ex.what());
    }
    *out = s.release();
    return PI_OK;
}

int pi_server_set_agent(pi_server *s, int agent, const float *x0, const float *u_warm, uint64_t seed)
{
    if (!s || !x0) return sfail(PI_ERR_INVALID_ARG, "server or x0 is NULL");
    if (agent < 0 || agent >= s->o.n_agents) return sfail(PI_ERR_INVALID_ARG, "agent out of range");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->agent_outstanding[agent]) return sfail(PI_ERR_BUSY, "agent has a request queued or in flight");
    DevGuard dg(s->device);
    if (dg.err != cudaSuccess) return scuda(dg.err, "cudaSetDevice");
    const size_t wn = (size_t)s->o.T_max * NU;
    int rc;
    if ((rc = scuda(cudaMemcpy(s->d_x0 + (size_t)agent * NX, x0, NX * 4, cudaMemcpyHostToDevice), "set agent"))) return rc;
    if (u_warm) {
        if ((rc = scuda(cudaMemcpy(s->d_warm + agent * wn, u_warm, wn * 4, cudaMemcpyHostToDevice), "set agent")))
            return rc;
    } else if ((rc = scuda(cudaMemset(s->d_warm + agent * wn, 0, wn * 4), "set agent"))) {
        return rc;
    }
    const uint64_t zero = 0;
    if ((rc = scuda(cudaMemcpy(s->d_ctr + agent, &zero, 8, cudaMemcpyHostToDevice), "set agent"))) return rc;
    return scuda(cudaMemcpy(s->d_seed + agent, &seed, 8, cudaMemcpyHostToDevice), "set agent");
}

int pi_server_submit(pi_server *s, const pi_serve_request *req, uint64_t *ticket)
{
    if (!s || !req) return sfail(PI_ERR_INVALID_ARG, "server or request is NULL");
    int rc = check_request(s, *req);
    if (rc) return rc;
    Req r;
    r.q = *req;
    r.q.x0 = nullptr;
    if (req->x0) {
        std::memcpy(r.x0, req->x0, sizeof r.x0);
        r.has_x0 = true;
    }
    r.bytes = req_layout(req->K, req->T).total;
    std::lock_guard<std::mutex> lk(s->mu);
    s->enqueue_locked(std::move(r));
    if (ticket) *ticket = s->next_ticket;
    return PI_OK;
}

int pi_server_cancel(pi_server *s, uint64_t ticket)
{
    if (!s) return sfail(PI_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        if (it->ticket != ticket) continue;
        pi_serve_done dn{};
        dn.ticket = it->ticket;
        dn.agent = it->q.agent;
        dn.K = it->q.K;
        dn.T = it->q.T;
        dn.status = PI_ERR_CANCELLED;
        dn.t_submit_ns = it->t_submit;
        dn.t_result_ns = now_ns();
        s->agent_outstanding[it->q.agent] -= 1;
        s->pending.erase(it);
        s->done_q.push_back(dn);
        s->st.completed += 1;
        s->cv_done.notify_all();
        return PI_OK;
    }
    if (ticket == 0 || ticket > s->next_ticket) return sfail(PI_ERR_INVALID_ARG, "unknown ticket");
    return sfail(PI_ERR_BUSY, "the request is on the GPU or finished");
}

int pi_server_poll(pi_server *s, pi_serve_done *out, int max, int64_t timeout_us, int *n_out)
{
    if (!s || !n_out || max < 0 || (max > 0 && !out)) return sfail(PI_ERR_INVALID_ARG, "bad argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done_q.empty() && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->done_q.empty(); });
    int n = 0;
    while (n < max && !s->done_q.empty()) {
        out[n++] = s->done_q.front();
        s->done_q.pop_front();
    }
    *n_out = n;
    return PI_OK;
}

int pi_server_result(pi_server *s, uint64_t ticket, float *u_out, float *costs)
{
    if (!s || !u_out) return sfail(PI_ERR_INVALID_ARG, "server or u_out is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return sfail(PI_ERR_INVALID_ARG, "no kept result for this ticket");
    const pi_server::Kept &k = it->second;
    std::memcpy(u_out, k.v.data(), (size_t)k.T * NU * 4);
    if (costs && s->o.want_costs) std::memcpy(costs, k.v.data() + (size_t)k.T * NU, (size_t)k.K * 4);
    s->results.erase(it);
    return PI_OK;
}

int pi_server_drain(pi_server *s, int64_t timeout_ms)
{
    if (!s) return sfail(PI_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(std::max<int64_t>(timeout_ms, 0)),
                                        [&] { return s->idle(); });
    return ok ? PI_OK : sfail(PI_ERR_TIMEOUT, "requests still queued or on the GPU");
}

int pi_server_replay(pi_server *s, const pi_serve_arrival *arr, int n, const pi_serve_request *proto,
                     pi_serve_done *done, int *n_done, int *n_dropped)
{
    if (!s || !proto || !n_done || !n_dropped || n < 0 || (n > 0 && (!arr || !done)))
        return sfail(PI_ERR_INVALID_ARG, "bad argument");
    *n_done = *n_dropped = 0;
    for (int i = 0; i < n; ++i) {
        pi_serve_request q = *proto;
        q.agent = arr[i].agent;
        q.K = arr[i].K;
        q.T = arr[i].T;
        int rc = check_request(s, q);
        if (rc) return rc;
        if (arr[i].t_ns < 0 || (i > 0 && arr[i].t_ns < arr[i - 1].t_ns))
            return sfail(PI_ERR_INVALID_ARG, "arrival times must be >= 0 and sorted");
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->idle() || !s->done_q.empty())
        return sfail(PI_ERR_BUSY, "replay needs an idle server with no unread completions");
    std::vector<char> waiting(s->o.n_agents, 0);
    int idx = 0, n_out = 0, nd = 0, ndrop = 0;
    const int64_t t0 = now_ns();
    int64_t last_progress = t0;
    for (;;) {
        const int64_t now = now_ns();
        while (idx < n && t0 + arr[idx].t_ns <= now) {
            const int a = arr[idx].agent;
            if (waiting[a]) {
                ++ndrop;
            } else {
                Req r;
                r.q = *proto;
                r.q.agent = a;
                r.q.K = arr[idx].K;
                r.q.T = arr[idx].T;
                r.q.x0 = nullptr;
                r.q.keep_result = 0;
                r.bytes = req_layout(r.q.K, r.q.T).total;
                s->enqueue_locked(std::move(r));
                waiting[a] = 1;
                ++n_out;
            }
            ++idx;
        }
        while (!s->done_q.empty()) {
            const pi_serve_done d = s->done_q.front();
            s->done_q.pop_front();
            if (nd < n) done[nd++] = d;
            waiting[d.agent] = 0;
            --n_out;
            last_progress = now;
        }
        if (idx >= n && n_out == 0) break;
        if (n_out > 0 && now - last_progress > REPLAY_STALL_NS) {
            *n_done = nd;
            *n_dropped = ndrop;
            return sfail(PI_ERR_TIMEOUT, "no request completed for 60 s");
        }
        const int64_t next = idx < n ? t0 + arr[idx].t_ns : now + 50'000'000;
        const auto tp = std::chrono::steady_clock::time_point(std::chrono::nanoseconds(next));
        s->cv_done.wait_until(lk, tp);
    }
    *n_done = nd;
    *n_dropped = ndrop;
    return PI_OK;
}

int pi_server_state_save(pi_server *s, float *x0, float *u_warm, uint64_t *counter, uint64_t *seed)
{
    if (!s || !x0 || !u_warm || !counter || !seed) return sfail(PI_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->idle()) return sfail(PI_ERR_BUSY, "server has requests queued or in flight");
    DevGuard dg(s->device);
    if (dg.err != cudaSuccess) return scuda(dg.err, "cudaSetDevice");
    const size_t na = s->o.n_agents;
    int rc;
    if ((rc = scuda(cudaMemcpy(x0, s->d_x0, na * NX * 4, cudaMemcpyDeviceToHost), "state save"))) return rc;
    if ((rc = scuda(cudaMemcpy(u_warm, s->d_warm, na * s->o.T_max * NU * 4, cudaMemcpyDeviceToHost), "state save")))
        return rc;
    if ((rc = scuda(cudaMemcpy(counter, s->d_ctr, na * 8, cudaMemcpyDeviceToHost), "state save"))) return rc;
    return scuda(cudaMemcpy(seed, s->d_seed, na * 8, cudaMemcpyDeviceToHost), "state save");
}

int pi_server_state_load(pi_server *s, const float *x0, const float *u_warm, const uint64_t *counter,
                         const uint64_t *seed)
{
    if (!s || !x0 || !u_warm || !counter || !seed) return sfail(PI_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->idle()) return sfail(PI_ERR_BUSY, "server has requests queued or in flight");
    DevGuard dg(s->device);
    if (dg.err != cudaSuccess) return scuda(dg.err, "cudaSetDevice");
    const size_t na = s->o.n_agents;
    int rc;
    if ((rc = scuda(cudaMemcpy(s->d_x0, x0, na * NX * 4, cudaMemcpyHostToDevice), "state load"))) return rc;
    if ((rc = scuda(cudaMemcpy(s->d_warm, u_warm, na * s->o.T_max * NU * 4, cudaMemcpyHostToDevice), "state load")))
        return rc;
    if ((rc = scuda(cudaMemcpy(s->d_ctr, counter, na * 8, cudaMemcpyHostToDevice), "state load"))) return rc;
    return scuda(cudaMemcpy(s->d_seed, seed, na * 8, cudaMemcpyHostToDevice), "state load");
}

int pi_server_get_stats(const pi_server *s, pi_server_stats *out)
{
    if (!s || !out) return sfail(PI_ERR_INVALID_ARG, "NULL argument");
    pi_server *m = const_cast<pi_server *>(s);
    std::lock_guard<std::mutex> lk(m->mu);
    *out = m->st;
    out->pool_peak_bytes = m->pool.peak();
    return PI_OK;
}

void pi_server_destroy(pi_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    DevGuard dg(s->device);
    free_server(s);
    delete s;
}

int pi_debug_struct_layout(size_t *out, int max, int *n)
{
    if (!out || !n || max < 0) return sfail(PI_ERR_INVALID_ARG, "bad argument");
#define PI_L(T, ...) sizeof(T), __VA_ARGS__
    const size_t v[] = {
        PI_L(pi_lwpr_params, offsetof(pi_lwpr_params, n_in), offsetof(pi_lwpr_params, n_out),
             offsetof(pi_lwpr_params, L), offsetof(pi_lwpr_params, dt), offsetof(pi_lwpr_params, c),
             offsetof(pi_lwpr_params, D), offsetof(pi_lwpr_params, beta), offsetof(pi_lwpr_params, b),
             offsetof(pi_lwpr_params, sigma)),
        PI_L(pi_cost_params, offsetof(pi_cost_params, goal), offsetof(pi_cost_params, Q_pos),
             offsetof(pi_cost_params, Q_vel), offsetof(pi_cost_params, Q_ang), offsetof(pi_cost_params, w_obs),
             offsetof(pi_cost_params, obs_sharp), offsetof(pi_cost_params, radius), offsetof(pi_cost_params, w_crash),
             offsetof(pi_cost_params, w_var), offsetof(pi_cost_params, w_T), offsetof(pi_cost_params, obs_kind),
             offsetof(pi_cost_params, n_obs), offsetof(pi_cost_params, obs_xy)),
        PI_L(pi_opts, offsetof(pi_opts, precision), offsetof(pi_opts, model_noise), offsetof(pi_opts, M),
             offsetof(pi_opts, device)),
        PI_L(pi_batch_item, offsetof(pi_batch_item, ctx), offsetof(pi_batch_item, K), offsetof(pi_batch_item, T),
             offsetof(pi_batch_item, x0), offsetof(pi_batch_item, u_nominal), offsetof(pi_batch_item, u_out),
             offsetof(pi_batch_item, costs_out)),
        PI_L(pi_server_opts, offsetof(pi_server_opts, n_agents), offsetof(pi_server_opts, K_max),
             offsetof(pi_server_opts, T_max), offsetof(pi_server_opts, max_inflight),
             offsetof(pi_server_opts, max_group), offsetof(pi_server_opts, hbm_budget),
             offsetof(pi_server_opts, want_costs)),
        PI_L(pi_serve_request, offsetof(pi_serve_request, agent), offsetof(pi_serve_request, K),
             offsetof(pi_serve_request, T), offsetof(pi_serve_request, lambda), offsetof(pi_serve_request, sigma_u),
             offsetof(pi_serve_request, x0), offsetof(pi_serve_request, keep_result)),
        PI_L(pi_serve_done, offsetof(pi_serve_done, ticket), offsetof(pi_serve_done, agent),
             offsetof(pi_serve_done, K), offsetof(pi_serve_done, T), offsetof(pi_serve_done, status),
             offsetof(pi_serve_done, group_size), offsetof(pi_serve_done, t_submit_ns),
             offsetof(pi_serve_done, t_launch_ns), offsetof(pi_serve_done, t_result_ns)),
        PI_L(pi_serve_arrival, offsetof(pi_serve_arrival, t_ns), offsetof(pi_serve_arrival, agent),
             offsetof(pi_serve_arrival, K), offsetof(pi_serve_arrival, T)),
        PI_L(pi_server_stats, offsetof(pi_server_stats, submitted), offsetof(pi_server_stats, completed),
             offsetof(pi_server_stats, groups), offsetof(pi_server_stats, launches),
             offsetof(pi_server_stats, memory_waits), offsetof(pi_server_stats, pool_bytes),
             offsetof(pi_server_stats, pool_peak_bytes), offsetof(pi_server_stats, peak_inflight_requests),
             offsetof(pi_server_stats, peak_group_size)),
    };
#undef PI_L
    const int cnt = (int)(sizeof v / sizeof v[0]);
    if (max < cnt) return sfail(PI_ERR_INVALID_ARG, "out is too small");
    for (int i = 0; i < cnt; ++i) out[i] = v[i];
    *n = cnt;
    return PI_OK;
}

int pi_debug_pool(size_t capacity, const int *op, const size_t *size, int n, int64_t *offset, int *free_extents)
{
    if (n < 0 || (n > 0 && (!op || !size || !offset)) || !free_extents)
        return sfail(PI_ERR_INVALID_ARG, "bad argument");
    Pool p(capacity);
    for (int i = 0; i < n; ++i) {
        if (op[i] == 1) {
            const size_t o = p.alloc(size[i]);
            offset[i] = o == Pool::NONE ? -1 : (int64_t)o;
        } else if (op[i] == 0) {
            const size_t j = size[i];
            if (j >= (size_t)i || op[j] != 1 || offset[j] < 0)
                return sfail(PI_ERR_INVALID_ARG, "free of an operation that is not an earlier successful allocation");
            p.release((size_t)offset[j], size[j]);
            offset[i] = offset[j];
            offset[j] = -2;   // freed (a second free of it is rejected)
        } else {
            return sfail(PI_ERR_INVALID_ARG, "op must be 0 or 1");
        }
    }
    *free_extents = p.extents();
    return PI_OK;
}

}  // extern "C"

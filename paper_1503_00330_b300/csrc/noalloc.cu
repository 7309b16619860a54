// noalloc.cu -- pi_update_noalloc: the same control update as pi_update, for
// callers that must not allocate device memory while they run.
//
// Who needs it: a controller whose real-time loop forbids allocation after
// start-up (cudaMalloc / cudaMallocAsync can block for an unbounded time,
// may synchronize the device, and can fail mid-flight), and a host program
// that hands all GPU memory to its own pool and does not let libraries
// allocate behind its back.  Such a caller creates its pi_ctx during set-up
// and then calls this entry point in its loop.
//
// It runs the rollout kernel of the context's form (FP32 or tensor cores; an
// FP32 context's output-split launch uses the exchange area that pi_create
// allocated), then the same scan and merge kernels as pi_update, so its
// results are those of pi_update bit for bit.  Instead of the context's growable scratch, this path keeps the per-update
// scratch (cost [T][K], eps [T][K][4], phi [K], log-sum-exp partials) in one
// file-scope device array of fixed size, NOALLOC_BYTES (about 21 MiB), which
// every GPU that loads the library holds until the process exits.  The
// array's name is only a host-side stand-in for the device symbol, so the
// host code below asks the runtime for its device address with
// cudaGetSymbolAddress, once per device, with that device current, and passes
// that address to the kernels.  With CUDA's lazy module loading (the default),
// that first lookup is also when the runtime loads this file's module on the
// device and commits the array's memory, so the first call on each device
// belongs in the caller's set-up, before its real-time loop and before any
// stream capture.
#include <cmath>
#include <mutex>
#include <string>

#include "pi2rh.h"
#include "pi2rh_ctx.h"
#include "pi2rh_kernels.h"

namespace {

constexpr size_t NA_MAX_KT = PI2RH_NOALLOC_MAX_KT;
constexpr size_t NA_MAX_K = PI2RH_NOALLOC_MAX_K;
constexpr size_t NA_MAX_T = PI2RH_NOALLOC_MAX_T;
// Layout of the array: eps, then cost, then phi, then the partials
// (at most K*T/RS_KC + T rows of 6 doubles).  All offsets are multiples of 256.
constexpr size_t NA_EPS_OFF = 0;
constexpr size_t NA_COST_OFF = NA_EPS_OFF + NA_MAX_KT * sizeof(float4);
constexpr size_t NA_PHI_OFF = NA_COST_OFF + NA_MAX_KT * sizeof(float);
constexpr size_t NA_PART_OFF = NA_PHI_OFF + NA_MAX_K * sizeof(float);
constexpr size_t NA_PART_ROWS = NA_MAX_KT / pi2rh::RS_KC + NA_MAX_T;
constexpr size_t NOALLOC_BYTES = NA_PART_OFF + NA_PART_ROWS * 6 * sizeof(double);
static_assert(NA_COST_OFF % 256 == 0 && NA_PHI_OFF % 256 == 0 && NA_PART_OFF % 256 == 0, "alignment");

constexpr int NA_MAX_DEVICES = 128;
std::mutex g_na_mutex;
void *g_na_ptr[NA_MAX_DEVICES] = {};

}  // namespace

// The scratch itself.  Shared by every call on a device; it keeps the last
// call's contents.  Nothing in it needs to start at zero: each update writes
// every element it later reads (eps, cost and phi by the rollout kernel, the
// partials by the scan kernel) before reading it.
static __device__ __align__(256) unsigned char pi2rh_noalloc_scratch[NOALLOC_BYTES];

namespace {

// Device address of the scratch array on `dev` (the current device).  Looked
// up on the first call for that device and cached.
int noalloc_scratch(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= NA_MAX_DEVICES) return pi2rh_fail(PI_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, pi2rh_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            std::string m = std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                            cudaGetErrorString(e);
            return pi2rh_fail(PI_ERR_CUDA, m.c_str());
        }
        g_na_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_na_ptr[dev]);
    return PI_OK;
}

int na_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PI_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return pi2rh_fail(PI_ERR_CUDA, m.c_str());
}

}  // namespace

extern "C" int pi_update_noalloc(pi_ctx *c, const float *x0, const float *u_nom, int K, int T, float lambda,
                                 const float *sigma_u, uint64_t seed, float *u_out, float *costs_out)
{
    using namespace pi2rh;
    if (!c) return pi2rh_fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (!x0 || !u_nom || !u_out || !costs_out || !sigma_u) return pi2rh_fail(PI_ERR_INVALID_ARG, "a buffer is NULL");
    if (K < 1 || T < 1) return pi2rh_fail(PI_ERR_INVALID_ARG, "K and T must be >= 1");
    if ((size_t)K > NA_MAX_K || (size_t)T > NA_MAX_T || (size_t)K * (size_t)T > NA_MAX_KT)
        return pi2rh_fail(PI_ERR_INVALID_ARG,
                          "pi_update_noalloc: size beyond its fixed scratch (needs K <= 65536, T <= 4096 and "
                          "K*T <= 1048576); use pi_update for larger problems");
    if (!(lambda > 0.0f) || !std::isfinite(lambda)) return pi2rh_fail(PI_ERR_INVALID_ARG, "lambda must be finite and > 0");
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(sigma_u[i]) || sigma_u[i] < 0.0f)
            return pi2rh_fail(PI_ERR_INVALID_ARG, "sigma_u must be finite and >= 0");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != c->device) {
        int rc = na_cuda(cudaSetDevice(c->device), "cudaSetDevice");
        if (rc) return rc;
    }
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(c->device, &base);
    if (rc == PI_OK) {
        float4 *eps = reinterpret_cast<float4 *>(base + NA_EPS_OFF);
        float *cost = reinterpret_cast<float *>(base + NA_COST_OFF);
        float *phi = reinterpret_cast<float *>(base + NA_PHI_OFF);
        double *part = reinterpret_cast<double *>(base + NA_PART_OFF);

        const bool tc = pi2rh_is_tc(c->opts.precision);
        cudaEvent_t *ev = timing_slot(c);
        if (ev) rc = na_cuda(cudaEventRecord(ev[0], c->stream), "event record");
        if (rc == PI_OK && tc) {
            TcArgs t = ctx_tc_args(c);
            t.K = K;
            t.T = T;
            for (int i = 0; i < 4; ++i) t.sqrt_sigma_u[i] = sqrtf(sigma_u[i]);
            t.seed = seed;
            t.x0 = x0;
            t.u_nom = u_nom;
            t.cost_tk = cost;
            t.eps_tk = eps;
            t.phi = phi;
            rc = na_cuda(launch_rollout_tc(t, c->stream), "tensor-core rollout kernel launch");
        } else if (rc == PI_OK) {
            RolloutArgs a = ctx_rollout_args(c);
            a.K = K;
            a.T = T;
            for (int i = 0; i < 4; ++i) a.sqrt_sigma_u[i] = sqrtf(sigma_u[i]);
            a.seed = seed;
            a.x0 = x0;
            a.u_nom = u_nom;
            a.cost_tk = cost;
            a.eps_tk = eps;
            a.phi = phi;
            rc = na_cuda(ctx_split_args(c, a), "split exchange area clear");
            int n = 0;
            if (rc == PI_OK) rc = na_cuda(launch_rollout_fp32(a, c->stream, &n), "rollout kernel launch");
            if (rc == PI_OK) c->launches += (uint64_t)(n - 1);   // counted as one below
        }
        if (rc == PI_OK && ev) rc = na_cuda(cudaEventRecord(ev[1], c->stream), "event record");
        const double inv_lam_log2e = 1.4426950408889634074 / (double)lambda;
        if (rc == PI_OK)
            rc = na_cuda(launch_scan_lse(cost, phi, eps, K, T, c->dt, inv_lam_log2e, costs_out, part, c->stream),
                         "scan kernel launch");
        if (rc == PI_OK && ev) rc = na_cuda(cudaEventRecord(ev[2], c->stream), "event record");
        if (rc == PI_OK)
            rc = na_cuda(launch_lse_merge(part, scan_blocks(K), T, inv_lam_log2e, u_nom, u_out, c->stream),
                         "merge kernel launch");
        if (rc == PI_OK && ev) rc = na_cuda(cudaEventRecord(ev[3], c->stream), "event record");
        if (rc == PI_OK && ev) ++c->n_timed;
        if (rc == PI_OK) c->launches += 3;
    }
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return rc;
}

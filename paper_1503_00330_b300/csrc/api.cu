// api.cu -- the extern "C" boundary of the library (declared in pi2rh.h):
// context creation (model validation and packing), scratch management,
// launches of the update pipeline, the host-buffer path, error reporting and
// host-side fault injection (PI_FAULT=alloc|launch|timeout).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "pi2rh.h"
#include "pi2rh_ctx.h"
#include "pi2rh_kernels.h"
#include "tc_ptx.cuh"

using namespace pi2rh;


namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(PI_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(PI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PI_CUDA(call, what)                                    \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));   \
    } while (0)

#define PI_TRY(call)                 \
    do {                             \
        int rc_ = (call);            \
        if (rc_ != PI_OK) return rc_; \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Host-side fault injection: PI_FAULT=alloc|launch|timeout makes the update
// entry points return the matching error before touching the GPU.
int injected_fault()
{
    const char *f = getenv("PI_FAULT");
    if (!f || !*f) return PI_OK;
    if (!strcmp(f, "alloc")) return fail(PI_ERR_OOM, "injected fault: allocation");
    if (!strcmp(f, "launch")) return fail(PI_ERR_CUDA, "injected fault: launch");
    if (!strcmp(f, "timeout")) return fail(PI_ERR_TIMEOUT, "injected fault: device wait timeout");
    return PI_OK;
}

bool finite_all(const float *p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

template <class T>
int grow(T **ptr, size_t *cap, size_t need, cudaStream_t s, const char *what)
{
    if (need <= *cap) return PI_OK;
    size_t n = need < 2 * *cap ? 2 * *cap : need;
    if (*ptr) PI_CUDA(cudaFreeAsync(*ptr, s), what);
    *ptr = nullptr;
    *cap = 0;
    PI_CUDA(cudaMallocAsync((void **)ptr, n * sizeof(T), s), what);
    *cap = n;
    return PI_OK;
}

int ensure_scratch(pi_ctx *c, int K, int T)
{
    const size_t kt = (size_t)K * T;
    PI_TRY(grow(&c->d_cost, &c->cap_cost, kt, c->stream, "scratch cost"));
    PI_TRY(grow(&c->d_eps, &c->cap_eps, kt, c->stream, "scratch eps"));
    PI_TRY(grow(&c->d_phi, &c->cap_phi, (size_t)K, c->stream, "scratch phi"));
    PI_TRY(grow(&c->d_part, &c->cap_part, (size_t)scan_blocks(K) * T * 6, c->stream, "scratch partials"));
    return PI_OK;
}

int check_sizes(int K, int T, int M)
{
    if (K < 1 || T < 1) return fail(PI_ERR_INVALID_ARG, "K and T must be >= 1 (K=%d, T=%d)", K, T);
    if ((long long)K * M > (1LL << 31) - 1 || (long long)K * T > (1LL << 40))
        return fail(PI_ERR_INVALID_ARG, "problem too large (K=%d, T=%d, M=%d)", K, T, M);
    return PI_OK;
}

int check_update_args(const float *lambda_p, float lambda, const float *sigma_u)
{
    (void)lambda_p;
    if (!(lambda > 0.0f) || !std::isfinite(lambda))
        return fail(PI_ERR_INVALID_ARG, "lambda must be finite and > 0 (got %g)", (double)lambda);
    if (!sigma_u) return fail(PI_ERR_INVALID_ARG, "sigma_u is NULL");
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(sigma_u[i]) || sigma_u[i] < 0.0f)
            return fail(PI_ERR_INVALID_ARG, "sigma_u[%d] must be finite and >= 0", i);
    return PI_OK;
}

RolloutArgs base_args(const pi_ctx *c) { return ctx_rollout_args(c); }

TcArgs tc_args(const pi_ctx *c) { return ctx_tc_args(c); }

int launch_rollouts(pi_ctx *c, const float *x0, const float *u_nom, int K, int T,
                    const float *sigma_u, uint64_t seed, float *cost, float4 *eps, float *phi)
{
    NvtxRange nv("pi2rh rollout");
    if (pi2rh_is_tc(c->opts.precision)) {
        TcArgs t = tc_args(c);
        t.K = K;
        t.T = T;
        for (int i = 0; i < 4; ++i) t.sqrt_sigma_u[i] = sqrtf(sigma_u[i]);
        t.seed = seed;
        t.x0 = x0;
        t.u_nom = u_nom;
        t.cost_tk = cost;
        t.eps_tk = eps;
        t.phi = phi;
        {
            cudaError_t e = launch_rollout_tc(t, c->stream);
            if (e != cudaSuccess) {
                std::string w = std::string("tensor-core rollout kernel launch (") + tc_launch_diag() + ")";
                return cuda_fail(e, w.c_str());
            }
        }
        c->launches++;
        return PI_OK;
    }
    RolloutArgs a = base_args(c);
    a.K = K;
    a.T = T;
    for (int i = 0; i < 4; ++i) a.sqrt_sigma_u[i] = sqrtf(sigma_u[i]);
    a.seed = seed;
    a.x0 = x0;
    a.u_nom = u_nom;
    a.cost_tk = cost;
    a.eps_tk = eps;
    a.phi = phi;
    PI_CUDA(ctx_split_args(c, a), "split exchange area clear");
    int n = 0;
    PI_CUDA(launch_rollout_fp32(a, c->stream, &n), "rollout kernel launch");
    c->launches += (uint64_t)n;
    return PI_OK;
}

// ev_mid (may be null) is recorded between the scan and the merge launches.
int launch_reduce(pi_ctx *c, const float *cost, const float *phi, const float4 *eps,
                  const float *u_nom, int K, int T, float lambda, float *u_out, float *costs_out,
                  cudaEvent_t ev_mid = nullptr)
{
    NvtxRange nv("pi2rh cost-to-go + weighted average");
    const double inv_lam_log2e = 1.4426950408889634074 / (double)lambda;
    PI_CUDA(launch_scan_lse(cost, phi, eps, K, T, c->dt, inv_lam_log2e, costs_out, c->d_part,
                            c->stream),
            "scan kernel launch");
    c->launches++;
    if (ev_mid) PI_CUDA(cudaEventRecord(ev_mid, c->stream), "event record");
    PI_CUDA(launch_lse_merge(c->d_part, scan_blocks(K), T, inv_lam_log2e, u_nom, u_out, c->stream),
            "merge kernel launch");
    c->launches++;
    return PI_OK;
}

void free_ctx_memory(pi_ctx *c)
{
    void *ptrs[] = {c->d_rec, c->d_obs, c->d_err, c->d_cost, c->d_eps, c->d_phi, c->d_part,
                    c->d_x0, c->d_unom, c->d_uout, c->d_costs, c->d_rh, c->d_wtiles, c->d_wconst, c->d_split};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, c->stream);
    cudaStreamSynchronize(c->stream);
    for (auto &set : c->ev)
        for (cudaEvent_t &e : set)
            if (e) cudaEventDestroy(e);
}

}  // namespace

namespace {

// Packs the model for the tensor-core form: per output and tile of 128
// fields, 11 chunks of 8 KB of fp16 coefficient blocks (128 rows x 16 K,
// K-major core-matrix layout, as the MMAs read them):
//   chunk 0 = [S hi of K step 0 | Y hi],  chunk 1 = [S lo of K step 0 | Y lo]
//     (K step 0 and the Y GEMM share the A operand z, so each pair of blocks
//     is one 256-row B operand of an N=256 MMA);
//   chunk j + 1 = [S hi | S lo] of K step j, j = 1..9;
// with cs_j the weight of the constant feature 152 (see rollout_tc.cu for
// the algebra), and the fp32 per-field constants cy_j and sigma_j^2.  The
// constant feature is 1 + 2^-14 as hi + lo, so its weight's lo part is
// cs_lo - 2^-14 cs_hi; a padding field of a ragged last tile has the weight
// -inf (hi; lo 0) and all other weights 0, so its exponent is exactly -inf and
// its softmax weight 0.
void pack_tc(const pi_lwpr_params *lw, int tiles, std::vector<unsigned char> &wt, std::vector<float> &wc)
{
    const int L = lw->L, TF = TC_TILE_FIELDS;
    const double kap = 0.72134752044448170368;   // log2(e) / 2
    wt.assign((size_t)NY * tiles * TC_TILE_BYTES, 0);
    wc.assign((size_t)NY * tiles * 2 * TF, 0.0f);
    // byte offsets (within a tile) of the hi and lo halves of coefficient
    // (field row i, feature k) of the S GEMM, and of coefficient k of the Y GEMM
    auto s_off = [](int i, int k, size_t &hi, size_t &lo) {
        const uint32_t o = kmajor_offset(i, k % 16, 16);
        if (k < 16) {
            hi = o;
            lo = (size_t)TC_CHUNK_BYTES + o;
        } else {
            hi = (size_t)(k / 16 + 1) * TC_CHUNK_BYTES + o;
            lo = hi + TC_HALF_CHUNK;
        }
    };
    auto y_off = [](int i, int k, size_t &hi, size_t &lo) {
        hi = (size_t)TC_HALF_CHUNK + kmajor_offset(i, k, 16);
        lo = (size_t)TC_CHUNK_BYTES + hi;
    };
    auto put = [](unsigned char *tile, size_t hi_off, size_t lo_off, double v) {
        const __half hi = __float2half_rn((float)v);
        const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
        *reinterpret_cast<__half *>(tile + hi_off) = hi;
        *reinterpret_cast<__half *>(tile + lo_off) = lo;
    };
    for (int o = 0; o < NY; ++o)
        for (int tt = 0; tt < tiles; ++tt) {
            unsigned char *tile = wt.data() + ((size_t)o * tiles + tt) * TC_TILE_BYTES;
            float *cst = wc.data() + ((size_t)o * tiles + tt) * 2 * TF;
            for (int i = 0; i < TF; ++i) {
                const int j = tt * TF + i;
                size_t ho, lo_o;
                if (j >= L) {
                    // padding field: exponent -inf, zero weight
                    s_off(i, TC_CONST_FEATURE, ho, lo_o);
                    *reinterpret_cast<__half *>(tile + ho) = __ushort_as_half((unsigned short)0xFC00u);
                    continue;
                }
                const size_t f = (size_t)o * L + j;
                const float *c = lw->c + f * NZ;
                const float *D = lw->D + f * NZ * NZ;
                const float *beta = lw->beta + f * NZ;
                double Dsc[NZ], cDc = 0.0, bc = 0.0;
                for (int a2 = 0; a2 < NZ; ++a2) {
                    double acc = 0.0;
                    for (int b2 = 0; b2 < NZ; ++b2)
                        acc += 0.5 * ((double)D[a2 * NZ + b2] + (double)D[b2 * NZ + a2]) * (double)c[b2];
                    Dsc[a2] = acc;
                    cDc += (double)c[a2] * acc;
                    bc += (double)beta[a2] * (double)c[a2];
                }
                for (int k = 0; k < TC_KF; ++k) {
                    s_off(i, k, ho, lo_o);
                    double v = 0.0;
                    if (k < 16) {
                        v = 2.0 * kap * Dsc[k];
                    } else if (k < 152) {
                        const int ra = tc_feat_row(k), cb = tc_feat_col(k);
                        v = ra == cb ? -kap * (double)D[ra * NZ + ra]
                                     : -kap * ((double)D[ra * NZ + cb] + (double)D[cb * NZ + ra]);
                    } else if (k == TC_CONST_FEATURE) {
                        // cs_j against the constant feature 1 + 2^-14 (hi + lo):
                        // hi*hi + hi*lo + lo*hi = cs_hi + (cs_lo - 2^-14 cs_hi) + 2^-14 cs_hi
                        const double cs = -kap * cDc;
                        const __half hi = __float2half_rn((float)cs);
                        const double hd = (double)__half2float(hi);
                        const __half lo = __float2half_rn((float)(cs - hd - 0x1p-14 * hd));
                        *reinterpret_cast<__half *>(tile + ho) = hi;
                        *reinterpret_cast<__half *>(tile + lo_o) = lo;
                        continue;
                    }
                    put(tile, ho, lo_o, v);
                }
                for (int k = 0; k < 16; ++k) {
                    y_off(i, k, ho, lo_o);
                    put(tile, ho, lo_o, (double)beta[k]);
                }
                cst[i] = (float)((double)lw->b[f] - bc);
                const double sg = (double)lw->sigma[f];
                cst[TF + i] = (float)(sg * sg);
            }
        }
}

}  // namespace

int pi2rh_fail(int code, const char *msg)
{
    return fail(code, "%s", msg);
}

extern "C" {

void pi_default_opts(pi_opts *o)
{
    if (!o) return;
    o->precision = PI_PRECISION_FP32;
    o->model_noise = PI_NOISE_SAMPLED;
    o->M = 1;
    o->device = 0;
}

const char *pi_last_error(void) { return g_err.c_str(); }

uint64_t pi_launch_count(const pi_ctx *c) { return c ? c->launches : 0; }

int pi_create(const pi_lwpr_params *lw, const pi_cost_params *cp, const pi_opts *opts_in, pi_ctx **out)
{
    if (!out) return fail(PI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!lw || !cp) return fail(PI_ERR_INVALID_ARG, "lwpr or cost params are NULL");
    pi_opts opts;
    pi_default_opts(&opts);
    if (opts_in) opts = *opts_in;
    if (lw->n_in != NZ || lw->n_out != NY)
        return fail(PI_ERR_INVALID_ARG, "n_in must be %d and n_out %d (got %d, %d)", NZ, NY, lw->n_in,
                    lw->n_out);
    if (lw->L < 1 || lw->L > (1 << 20)) return fail(PI_ERR_INVALID_ARG, "L out of range (%d)", lw->L);
    if (!(lw->dt > 0.0f) || !std::isfinite(lw->dt)) return fail(PI_ERR_INVALID_ARG, "dt must be > 0");
    if (!lw->c || !lw->D || !lw->beta || !lw->b || !lw->sigma)
        return fail(PI_ERR_INVALID_ARG, "an LWPR array is NULL");
    if (opts.precision != PI_PRECISION_FP32 && !pi2rh_is_tc(opts.precision))
        return fail(PI_ERR_UNSUPPORTED, "precision %d is not available", opts.precision);
    if (opts.model_noise != PI_NOISE_SAMPLED && opts.model_noise != PI_NOISE_MEAN_ONLY)
        return fail(PI_ERR_INVALID_ARG, "model_noise must be 0 or 1");
    if (opts.M < 1 || opts.M > PI2RH_MAX_M || (opts.M & (opts.M - 1)))
        return fail(PI_ERR_INVALID_ARG, "M must be a power of two in [1, %d] (got %d)", PI2RH_MAX_M, opts.M);
    if (cp->n_obs < 0 || cp->n_obs > PI2RH_MAX_OBS)
        return fail(PI_ERR_INVALID_ARG, "n_obs must be in [0, %d]", PI2RH_MAX_OBS);
    if (cp->n_obs > 0 && !cp->obs_xy) return fail(PI_ERR_INVALID_ARG, "obs_xy is NULL");
    if (cp->obs_kind != PI_OBS_INDICATOR && cp->obs_kind != PI_OBS_GAUSSIAN)
        return fail(PI_ERR_INVALID_ARG, "obs_kind must be 0 or 1");
    const int L = lw->L;
    const size_t nf = (size_t)NY * L;
    if (!finite_all(lw->c, nf * NZ) || !finite_all(lw->D, nf * NZ * NZ) ||
        !finite_all(lw->beta, nf * NZ) || !finite_all(lw->b, nf) || !finite_all(lw->sigma, nf))
        return fail(PI_ERR_INVALID_ARG, "LWPR parameters must be finite");
    const float scal[] = {cp->goal[0], cp->goal[1], cp->goal[2], cp->Q_pos[0], cp->Q_pos[1],
                          cp->Q_pos[2], cp->Q_vel, cp->Q_ang, cp->w_obs, cp->obs_sharp,
                          cp->radius, cp->w_crash, cp->w_var, cp->w_T};
    if (!finite_all(scal, sizeof scal / sizeof scal[0]) ||
        (cp->n_obs > 0 && !finite_all(cp->obs_xy, (size_t)2 * cp->n_obs)))
        return fail(PI_ERR_INVALID_ARG, "cost parameters must be finite");

    // Pack field pairs (see the record layout in pi2rh_device.cuh).
    const int P = (L + 1) / 2;
    std::vector<float2> rec((size_t)NY * P * REC_LEN, make_float2(0.f, 0.f));
    const double kap = 0.72134752044448170368;   // log2(e) / 2
    for (int o = 0; o < NY; ++o) {
        for (int j = 0; j < L; ++j) {
            float2 *r = &rec[((size_t)o * P + j / 2) * REC_LEN];
            const int h = j & 1;
            auto put = [&](int e, float v) {
                if (h) r[e].y = v; else r[e].x = v;
            };
            const size_t f = (size_t)o * L + j;
            const float *c = lw->c + f * NZ;
            const float *D = lw->D + f * NZ * NZ;
            for (int a = 0; a < NZ; ++a) put(REC_NEGC + a, -c[a]);
            for (int i = 0; i < NZ; ++i)
                for (int jj = i; jj < NZ; ++jj) {
                    double v = (i == jj) ? -kap * (double)D[i * NZ + i]
                                         : -kap * ((double)D[i * NZ + jj] + (double)D[jj * NZ + i]);
                    put(REC_A + tri_index(i, jj), (float)v);
                }
            for (int a = 0; a < NZ; ++a) put(REC_BETA + a, lw->beta[f * NZ + a]);
            put(REC_B, lw->b[f]);
            const double s = (double)lw->sigma[f];
            put(REC_VAR, (float)(s * s));
            put(REC_BIAS, 0.0f);
        }
        if (L & 1) rec[((size_t)o * P + P - 1) * REC_LEN + REC_BIAS].y = -INFINITY;
    }

    pi_ctx *c = new pi_ctx();
    c->device = opts.device;
    c->opts = opts;
    c->L = L;
    c->P = P;
    c->spo = (P + RF_PAIRS_PER_STAGE - 1) / RF_PAIRS_PER_STAGE;
    c->dt = lw->dt;
    DeviceGuard dg(opts.device);
    if (dg.err != cudaSuccess) {
        delete c;
        return cuda_fail(dg.err, "cudaSetDevice");
    }
    auto bail = [&](cudaError_t e, const char *what) {
        free_ctx_memory(c);
        delete c;
        return cuda_fail(e, what);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_rec, rec.size() * sizeof(float2))) != cudaSuccess) return bail(e, "model alloc");
    if ((e = cudaMemcpy(c->d_rec, rec.data(), rec.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "model copy");
    const int nob = cp->n_obs > 0 ? cp->n_obs : 1;
    if ((e = cudaMalloc(&c->d_obs, nob * sizeof(float2))) != cudaSuccess) return bail(e, "obstacle alloc");
    if (cp->n_obs > 0 &&
        (e = cudaMemcpy(c->d_obs, cp->obs_xy, cp->n_obs * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "obstacle copy");
    if ((e = cudaMalloc(&c->d_err, sizeof(int))) != cudaSuccess) return bail(e, "error word alloc");
    if ((e = cudaMemset(c->d_err, 0, sizeof(int))) != cudaSuccess) return bail(e, "error word clear");
    if (!pi2rh_is_tc(opts.precision)) {
        // exchange area of the output-split rollout launch: one block per SM at most
        int nsm = 0;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, opts.device)) != cudaSuccess)
            return bail(e, "SM count");
        int coop = 0;
        if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, opts.device)) != cudaSuccess)
            return bail(e, "cooperative-launch attribute");
        if (coop && nsm > 0) {
            c->split_max_blocks = nsm;
            const size_t nb = split_bytes(nsm);
            if ((e = cudaMalloc(&c->d_split, nb)) != cudaSuccess) return bail(e, "split exchange alloc");
            if ((e = cudaMemset(c->d_split, 0, nb)) != cudaSuccess) return bail(e, "split exchange clear");
        }
    }
    if (pi2rh_is_tc(opts.precision)) {
        std::vector<unsigned char> wt;
        std::vector<float> wc;
        c->tiles_per_out = (L + TC_TILE_FIELDS - 1) / TC_TILE_FIELDS;
        pack_tc(lw, c->tiles_per_out, wt, wc);
        if ((e = cudaMalloc(&c->d_wtiles, wt.size())) != cudaSuccess) return bail(e, "tile alloc");
        if ((e = cudaMemcpy(c->d_wtiles, wt.data(), wt.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "tile copy");
        if ((e = cudaMalloc(&c->d_wconst, wc.size() * sizeof(float))) != cudaSuccess) return bail(e, "const alloc");
        if ((e = cudaMemcpy(c->d_wconst, wc.data(), wc.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "const copy");
    }
    CostDev &C = c->cost;
    for (int d = 0; d < 3; ++d) {
        C.goal[d] = cp->goal[d];
        C.Q_pos[d] = cp->Q_pos[d];
    }
    C.Q_vel = cp->Q_vel;
    C.Q_ang = cp->Q_ang;
    C.w_obs = cp->w_obs;
    C.obs_sharp = cp->obs_sharp;
    C.radius = cp->radius;
    C.w_crash = cp->w_crash;
    C.w_var = cp->w_var;
    C.w_T = cp->w_T;
    C.obs_kind = cp->obs_kind;
    C.n_obs = cp->n_obs;
    C.obs = c->d_obs;
    *out = c;
    return PI_OK;
}

int pi_set_output_split(pi_ctx *c, int mode)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (mode != PI_SPLIT_OFF && mode != PI_SPLIT_AUTO && mode != PI_SPLIT_ALWAYS)
        return fail(PI_ERR_INVALID_ARG, "split mode must be PI_SPLIT_OFF, PI_SPLIT_AUTO or PI_SPLIT_ALWAYS");
    c->split_mode = mode;
    return PI_OK;
}

int pi_debug_split_plan(pi_ctx *c, int K, int *plain_blocks, int *units_per_cta, int *ctas)
{
    if (!c || !plain_blocks || !units_per_cta || !ctas) return fail(PI_ERR_INVALID_ARG, "NULL argument");
    if (pi2rh_is_tc(c->opts.precision)) return fail(PI_ERR_INVALID_ARG, "the output split is an FP32-form launch");
    if (K < 1) return fail(PI_ERR_INVALID_ARG, "K must be >= 1");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    RolloutArgs a = base_args(c);
    a.K = K;
    a.split = c->d_split;
    a.split_max_blocks = c->split_max_blocks;
    a.split_mode = c->split_mode;
    const Fp32Launch L = fp32_launch_plan(a, c->stream);
    *plain_blocks = L.plain_blocks;
    *units_per_cta = L.upc;
    *ctas = L.upc > 0 ? L.split_ctas : 0;
    return PI_OK;
}

int pi_debug_split_plan_sizes(int K, int M, int L, int n_sm, int mode, int *plain_blocks, int *units_per_cta,
                              int *ctas)
{
    if (!plain_blocks || !units_per_cta || !ctas) return fail(PI_ERR_INVALID_ARG, "NULL argument");
    if (K < 1 || M < 1 || L < 1 || n_sm < 1) return fail(PI_ERR_INVALID_ARG, "K, M, L and n_sm must be >= 1");
    if (mode != PI_SPLIT_OFF && mode != PI_SPLIT_AUTO && mode != PI_SPLIT_ALWAYS)
        return fail(PI_ERR_INVALID_ARG, "unknown split mode");
    const long long blocks = ((long long)K * M + RF_SLOTS - 1) / RF_SLOTS;
    const Fp32Launch Lp = fp32_plan_blocks(blocks, n_sm, (L + 1) / 2, mode, n_sm);
    *plain_blocks = Lp.plain_blocks;
    *units_per_cta = Lp.upc;
    *ctas = Lp.upc > 0 ? Lp.split_ctas : 0;
    return PI_OK;
}

int pi_debug_split_partition(int blocks, int units_per_cta, int cta, int *seg, int *n_seg)
{
    if (!seg || !n_seg) return fail(PI_ERR_INVALID_ARG, "NULL argument");
    const int n = fp32_split_partition(blocks, units_per_cta, cta, seg);
    if (n == 0) return fail(PI_ERR_INVALID_ARG, "no such CTA in that split (blocks >= 1, 1 <= units < 12)");
    *n_seg = n;
    return PI_OK;
}

int pi_debug_split_drop_cta(pi_ctx *c, int drop)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (drop < 0 || drop > 2) return fail(PI_ERR_INVALID_ARG, "drop must be 0, 1 or 2");
    c->split_drop = drop;
    return PI_OK;
}

int pi_set_stream(pi_ctx *c, void *stream)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    // Scratch is stream-ordered: finish the old stream's work before switching.
    PI_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    c->stream = (cudaStream_t)stream;
    return PI_OK;
}

int pi_reserve(pi_ctx *c, int K, int T)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    PI_TRY(check_sizes(K, T, c->opts.M));
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    return ensure_scratch(c, K, T);
}

int pi_update(pi_ctx *c, const float *x0, const float *u_nom, int K, int T, float lambda,
              const float *sigma_u, uint64_t seed, float *u_out, float *costs_out)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (!x0 || !u_nom || !u_out || !costs_out) return fail(PI_ERR_INVALID_ARG, "a buffer is NULL");
    PI_TRY(check_sizes(K, T, c->opts.M));
    PI_TRY(check_update_args(nullptr, lambda, sigma_u));
    PI_TRY(injected_fault());
    NvtxRange nv("pi_update");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    PI_TRY(ensure_scratch(c, K, T));
    cudaEvent_t *ev = timing_slot(c);
    if (ev) PI_CUDA(cudaEventRecord(ev[0], c->stream), "event record");
    PI_TRY(launch_rollouts(c, x0, u_nom, K, T, sigma_u, seed, c->d_cost, c->d_eps, c->d_phi));
    if (ev) PI_CUDA(cudaEventRecord(ev[1], c->stream), "event record");
    PI_TRY(launch_reduce(c, c->d_cost, c->d_phi, c->d_eps, u_nom, K, T, lambda, u_out, costs_out,
                         ev ? ev[2] : nullptr));
    if (ev) {
        PI_CUDA(cudaEventRecord(ev[3], c->stream), "event record");
        ++c->n_timed;
    }
    return PI_OK;
}

int pi_rh_advance(pi_ctx *c, float *x0, const float *u_out, int T, float *u_next)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (!x0 || !u_out || !u_next || T < 1) return fail(PI_ERR_INVALID_ARG, "bad argument");
    if (u_next < u_out + (size_t)T * NU && u_out < u_next + (size_t)T * NU)
        return fail(PI_ERR_INVALID_ARG, "u_nom_next must not overlap u_out");
    NvtxRange nv("pi_rh_advance");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    if (!c->d_rh) PI_CUDA(cudaMallocAsync((void **)&c->d_rh, 40 * sizeof(float), c->stream), "rh scratch");
    PI_CUDA(launch_rh_build_z(x0, u_out, c->d_rh, c->stream), "rh kernel launch");
    RolloutArgs a = base_args(c);
    a.M = 1;
    a.z_in = c->d_rh;
    a.y_out = c->d_rh + 16;
    a.var_out = c->d_rh + 28;
    a.n_pred = 1;
    PI_CUDA(launch_predict_fp32(a, c->stream), "predict kernel launch");
    PI_CUDA(launch_rh_apply(x0, c->d_rh + 16, c->dt, u_out, T, u_next, c->stream), "rh kernel launch");
    c->launches += 3;
    return PI_OK;
}

int pi_set_timing(pi_ctx *c, int enable)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    if (enable && !c->ev[0][0])
        for (auto &set : c->ev)
            for (cudaEvent_t &e : set) PI_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    c->timing = enable != 0;
    return PI_OK;
}

int pi_stage_times_at(pi_ctx *c, int back, float *ms)
{
    if (!c || !ms) return fail(PI_ERR_INVALID_ARG, "bad argument");
    if (!c->ev[0][0]) return fail(PI_ERR_INVALID_ARG, "timing is not enabled");
    const uint64_t avail = c->n_timed < (uint64_t)PI2RH_TIMING_RING ? c->n_timed : (uint64_t)PI2RH_TIMING_RING;
    if (back < 0 || (uint64_t)back >= avail)
        return fail(PI_ERR_INVALID_ARG, "no timed update %d calls back (%llu kept)", back, (unsigned long long)avail);
    cudaEvent_t *ev = c->ev[(c->n_timed - 1 - (uint64_t)back) % PI2RH_TIMING_RING];
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    PI_CUDA(cudaEventSynchronize(ev[3]), "cudaEventSynchronize");
    PI_CUDA(cudaEventElapsedTime(&ms[0], ev[0], ev[1]), "cudaEventElapsedTime");
    PI_CUDA(cudaEventElapsedTime(&ms[1], ev[1], ev[2]), "cudaEventElapsedTime");
    PI_CUDA(cudaEventElapsedTime(&ms[2], ev[2], ev[3]), "cudaEventElapsedTime");
    return PI_OK;
}

int pi_stage_times(pi_ctx *c, float *ms) { return pi_stage_times_at(c, 0, ms); }

int pi_sync(pi_ctx *c)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    PI_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    int err = 0;
    PI_CUDA(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word read");
    if (err) {
        PI_CUDA(cudaMemset(c->d_err, 0, sizeof(int)), "error word clear");
        if (err & (DEVERR_TIMEOUT_FULL | DEVERR_TIMEOUT_EMPTY | DEVERR_TIMEOUT_DRAIN | DEVERR_TIMEOUT_PEER))
            return fail(PI_ERR_TIMEOUT, "a bounded device-side wait expired (flags 0x%x)", err);
        return fail(PI_ERR_INTERNAL, "device-side check failed (flags 0x%x)", err);
    }
    return PI_OK;
}

int pi_update_host(pi_ctx *c, const float *x0, const float *u_nom, int K, int T, float lambda,
                   const float *sigma_u, uint64_t seed, float *u_out, float *costs_out)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (!x0 || !u_nom || !u_out || !costs_out) return fail(PI_ERR_INVALID_ARG, "a buffer is NULL");
    PI_TRY(check_sizes(K, T, c->opts.M));
    PI_TRY(check_update_args(nullptr, lambda, sigma_u));
    PI_TRY(injected_fault());
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    PI_TRY(grow(&c->d_x0, &c->cap_x0, (size_t)NX, c->stream, "staging x0"));
    PI_TRY(grow(&c->d_unom, &c->cap_unom, (size_t)T * NU, c->stream, "staging u_nom"));
    PI_TRY(grow(&c->d_uout, &c->cap_uout, (size_t)T * NU, c->stream, "staging u_out"));
    PI_TRY(grow(&c->d_costs, &c->cap_costs, (size_t)K, c->stream, "staging costs"));
    PI_CUDA(cudaMemcpyAsync(c->d_x0, x0, NX * sizeof(float), cudaMemcpyHostToDevice, c->stream), "copy x0");
    PI_CUDA(cudaMemcpyAsync(c->d_unom, u_nom, (size_t)T * NU * sizeof(float), cudaMemcpyHostToDevice, c->stream),
            "copy u_nom");
    PI_TRY(pi_update(c, c->d_x0, c->d_unom, K, T, lambda, sigma_u, seed, c->d_uout, c->d_costs));
    PI_CUDA(cudaMemcpyAsync(u_out, c->d_uout, (size_t)T * NU * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
            "copy u_out");
    PI_CUDA(cudaMemcpyAsync(costs_out, c->d_costs, (size_t)K * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
            "copy costs");
    return pi_sync(c);
}

void pi_destroy(pi_ctx *c)
{
    if (!c) return;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    free_ctx_memory(c);
    delete c;
}

int pi_debug_noise(uint64_t seed, int K, int T, int m, uint32_t *raw, void *stream)
{
    PI_TRY(check_sizes(K, T, 1));
    if (!raw || m < 0) return fail(PI_ERR_INVALID_ARG, "bad argument");
    PI_CUDA(launch_noise_raw(seed, K, T, m, raw, (cudaStream_t)stream), "noise kernel launch");
    return PI_OK;
}

int pi_debug_normals(uint64_t seed, int K, int T, int m, float *ctrl, float *model, void *stream)
{
    PI_TRY(check_sizes(K, T, 1));
    if (!ctrl || !model || m < 0) return fail(PI_ERR_INVALID_ARG, "bad argument");
    PI_CUDA(launch_noise_normals(seed, K, T, m, ctrl, model, (cudaStream_t)stream), "normals kernel launch");
    return PI_OK;
}

int pi_debug_lwpr(pi_ctx *c, const float *z, int n, float *y, float *var)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (n < 1 || !z || !y || !var) return fail(PI_ERR_INVALID_ARG, "bad argument");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    if (pi2rh_is_tc(c->opts.precision)) {
        TcArgs t = tc_args(c);
        t.M = 1;
        t.z_in = z;
        t.y_out = y;
        t.var_out = var;
        t.n_pred = n;
        {
            cudaError_t e = launch_predict_tc(t, c->stream);
            if (e != cudaSuccess) {
                std::string w = std::string("tensor-core predict kernel launch (") + tc_launch_diag() + ")";
                return cuda_fail(e, w.c_str());
            }
        }
        c->launches++;
        return PI_OK;
    }
    RolloutArgs a = base_args(c);
    a.M = 1;
    a.z_in = z;
    a.y_out = y;
    a.var_out = var;
    a.n_pred = n;
    PI_CUDA(launch_predict_fp32(a, c->stream), "predict kernel launch");
    c->launches++;
    return PI_OK;
}

int pi_debug_rollout(pi_ctx *c, const float *x0, const float *u_nom, int K, int T,
                     const float *sigma_u, uint64_t seed, float *cost, float *eps, float *phi)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (!x0 || !u_nom || !cost || !eps || !phi) return fail(PI_ERR_INVALID_ARG, "a buffer is NULL");
    PI_TRY(check_sizes(K, T, c->opts.M));
    PI_TRY(check_update_args(nullptr, 1.0f, sigma_u));
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    return launch_rollouts(c, x0, u_nom, K, T, sigma_u, seed, cost, reinterpret_cast<float4 *>(eps), phi);
}

int pi_debug_reduce(pi_ctx *c, const float *cost, const float *phi, const float *eps,
                    const float *u_nom, int K, int T, float lambda, float *u_out, float *costs_out)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (!cost || !phi || !eps || !u_nom || !u_out || !costs_out)
        return fail(PI_ERR_INVALID_ARG, "a buffer is NULL");
    PI_TRY(check_sizes(K, T, 1));
    const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
    PI_TRY(check_update_args(nullptr, lambda, zero4));
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    PI_TRY(grow(&c->d_part, &c->cap_part, (size_t)scan_blocks(K) * T * 6, c->stream, "scratch partials"));
    return launch_reduce(c, cost, phi, reinterpret_cast<const float4 *>(eps), u_nom, K, T, lambda, u_out,
                         costs_out);
}

int pi_debug_wait_timeout(pi_ctx *c, int64_t limit_ns)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (limit_ns < 1000 || limit_ns > 1000000000) return fail(PI_ERR_INVALID_ARG, "limit_ns outside [1e3, 1e9]");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    PI_CUDA(launch_wait_timeout(c->d_err, (unsigned long long)limit_ns, c->stream), "wait kernel launch");
    c->launches += 1;
    return PI_OK;
}

int pi_debug_tc_gemm(pi_ctx *c, const void *A, const void *B, int K, float *D)
{
    if (!c) return fail(PI_ERR_INVALID_ARG, "ctx is NULL");
    if (!A || !B || !D || K < 16 || K > 160 || K % 16) return fail(PI_ERR_INVALID_ARG, "bad argument");
    DeviceGuard dg(c->device);
    PI_CUDA(dg.err, "cudaSetDevice");
    PI_CUDA(launch_tc_gemm_check(A, B, K, D, c->d_err, c->stream), "tc gemm launch");
    c->launches++;
    return PI_OK;
}

}  // extern "C"

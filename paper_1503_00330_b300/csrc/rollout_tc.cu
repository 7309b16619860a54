// rollout_tc.cu -- tensor-core form of the fused rollout kernel.
//
// The receptive-field exponents and local predictions (Sec. 2, Eq. 1) of all
// 12 L fields are evaluated for 128 rollout slots at a time as two GEMMs on
// the 5th-generation tensor cores:
//   s_j = -(1/2) log2(e) (z - c_j)^T D_j (z - c_j)
//       = phi(z) . w_j + cs_j,   phi(z) = [z_a (16), z_a z_b (a <= b, 136), 0 (8)]
//   y_j = b_j + beta_j . (z - c_j) = z . beta_j + cy_j
// with w_j = [2k (D_s c_j)_a, -k D'_ab, 0], k = log2(e)/2, D_s = (D + D^T)/2,
// D'_aa = D_aa, D'_ab = D_ab + D_ba; the constants cs_j = -k c_j^T D_s c_j and
// cy_j = b_j - beta_j . c_j are added in FP32 in the epilogue.
//
// Precision: operands are split into fp16 hi + lo parts and each product is
// formed as hi*hi + hi*lo + lo*hi (three tcgen05.mma kind::f16 per K step,
// fp32 accumulation in tensor memory); the dropped lo*lo term is ~2^-22
// relative, so the exponents carry FP32-level accuracy.
//
// Roles (one CTA per SM, 128 slots, 320 threads):
//   warp 0 lane 0: producer -- 1-D bulk copies (TMA) of the pre-packed
//                  coefficient tiles (64 fields, 45,056 B) into a 2-stage ring,
//                  and of the per-field constants (cs, cy, sigma^2) into a
//                  4-deep constant ring;
//   warp 1 lane 0: MMA issuer -- 33 MMAs per tile (S: 10 K steps x 3, Y: 1 x 3)
//                  into one of two TMEM accumulator buffers;
//   warps 2-9:     epilogue -- tcgen05.ld of S and Y, online base-2 softmax
//                  per output (chunks of 16 fields, one rescale per chunk),
//                  merge of the two column halves, then the dynamics step
//                  (cost, Euler step, Philox noise) and the feature tile of
//                  the next step.
// Every wait is bounded; on expiry the kernel flags the device error word,
// drains its copies and MMAs, frees its tensor memory and returns.
#include <cstdio>

#include <cuda_fp16.h>

#include "pi2rh_kernels.h"
#include "tc_ptx.cuh"

namespace pi2rh {

namespace {

constexpr int BM = TC_SLOTS;            // rollout slots per CTA (MMA M)
constexpr int TNF = TC_TILE_FIELDS;     // fields per tile (MMA N)
constexpr int KF = TC_KF;               // feature columns of phi (S GEMM K)
constexpr int KY = 16;                  // Y GEMM K (z only)
constexpr int NSTAGE = 2;
constexpr int NCONST = 4;
constexpr int NEPI = 8;                 // epilogue warps
constexpr int NTHREADS = (2 + NEPI) * 32;
constexpr int NE = NEPI * 32;
constexpr int MAX_OBS = 256;

constexpr int PHI_BYTES = BM * KF * 2;                 // one fp16 feature tile
constexpr int OFF_PHI_HI = 0;
constexpr int OFF_PHI_LO = OFF_PHI_HI + PHI_BYTES;
constexpr int OFF_STAGE = OFF_PHI_LO + PHI_BYTES;
constexpr int OFF_CONST = OFF_STAGE + NSTAGE * TC_TILE_BYTES;
constexpr int OFF_PART = OFF_CONST + NCONST * TC_CONST_BYTES;   // [2][5][BM]
constexpr int OFF_Z = OFF_PART + 2 * 5 * BM * 4;                // [NZ][BM]
constexpr int OFF_X = OFF_Z + NZ * BM * 4;                      // [NX][BM]
constexpr int OFF_Y = OFF_X + NX * BM * 4;                      // [NY][BM]
constexpr int OFF_V = OFF_Y + NY * BM * 4;
constexpr int OFF_YREF = OFF_V + NY * BM * 4;
constexpr int OFF_Q = OFF_YREF + NY * BM * 4;                   // [BM]
constexpr int OFF_OBS = OFF_Q + BM * 4;
constexpr int OFF_BAR = OFF_OBS + MAX_OBS * 8;
// barriers: stage_full[2], stage_empty[2], acc_full[2], acc_empty[2],
//           const_full[4], const_empty[4], phi_ready
constexpr int NBARS = 2 * NSTAGE + 4 + 2 * NCONST + 1;
constexpr int OFF_TSLOT = OFF_BAR + NBARS * 8;
constexpr int OFF_ABORT = OFF_TSLOT + 8;
constexpr int SMEM_BYTES = OFF_ABORT + 16;
static_assert(OFF_STAGE % 128 == 0 && OFF_CONST % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

constexpr uint32_t TMEM_COLS = 256;     // 2 buffers x (S 64 + Y 64)

// Feature k of phi: k < 16 -> z_k * 1; 16 <= k < 152 -> z_a z_b; k >= 152 -> 0.
__host__ __device__ constexpr int feat_a(int k) { return k < 16 ? k : tc_feat_row(k); }
__host__ __device__ constexpr int feat_b(int k) { return k < 16 ? 16 : tc_feat_col(k); }

struct Soft {
    float m, s0, s1, s2, s3;
};

__device__ __forceinline__ void merge_into(Soft &a, const Soft &b)
{
    const float M = fmaxf(a.m, b.m);
    const float Ms = M == -INFINITY ? 0.0f : M;
    const float ca = ex2(a.m - Ms), cb = ex2(b.m - Ms);
    a.s0 = fmaf(a.s0, ca, b.s0 * cb);
    a.s1 = fmaf(a.s1, ca, b.s1 * cb);
    a.s2 = fmaf(a.s2, ca, b.s2 * cb);
    a.s3 = fmaf(a.s3, ca, b.s3 * cb);
    a.m = M;
}

__device__ __forceinline__ uint32_t pack_h2(__half lo, __half hi)
{
    return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}

template <int K>
__device__ __forceinline__ float feature(const float (&zext)[17])
{
    if constexpr (K < 152) {
        constexpr int fa = feat_a(K), fb = feat_b(K);
        return zext[fa] * zext[fb];
    } else {
        return 0.0f;
    }
}

template <int K>
__device__ __forceinline__ void split_pair(const float (&zext)[17], uint32_t &hw, uint32_t &lw)
{
    const float f0 = feature<K>(zext), f1 = feature<K + 1>(zext);
    const __half h0 = __float2half_rn(f0), h1 = __float2half_rn(f1);
    hw = pack_h2(h0, h1);
    lw = pack_h2(__float2half_rn(f0 - __half2float(h0)), __float2half_rn(f1 - __half2float(h1)));
}

// Writes the hi/lo fp16 feature rows of slot r from z (zext[16] == 1), one
// 16-byte core-matrix row (8 features) at a time.
template <int K8 = 0>
__device__ __forceinline__ void build_features(unsigned char *smem, int r, const float (&zext)[17])
{
    if constexpr (K8 < KF / 8) {
        uint32_t hw[4], lw[4];
        split_pair<K8 * 8 + 0>(zext, hw[0], lw[0]);
        split_pair<K8 * 8 + 2>(zext, hw[1], lw[1]);
        split_pair<K8 * 8 + 4>(zext, hw[2], lw[2]);
        split_pair<K8 * 8 + 6>(zext, hw[3], lw[3]);
        const uint32_t off = kmajor_offset(r, K8 * 8, KF);
        *reinterpret_cast<uint4 *>(smem + OFF_PHI_HI + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(smem + OFF_PHI_LO + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        build_features<K8 + 1>(smem, r, zext);
    }
}

template <bool PREDICT>
__global__ void __launch_bounds__(NTHREADS, 1) rollout_tc_kernel(const __grid_constant__ TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    float *part = reinterpret_cast<float *>(smem + OFF_PART);
    float *zbuf = reinterpret_cast<float *>(smem + OFF_Z);
    float *xbuf = reinterpret_cast<float *>(smem + OFF_X);
    float *ybuf = reinterpret_cast<float *>(smem + OFF_Y);
    float *vbuf = reinterpret_cast<float *>(smem + OFF_V);
    float *yrbuf = reinterpret_cast<float *>(smem + OFF_YREF);
    float *qbuf = reinterpret_cast<float *>(smem + OFF_Q);
    float2 *obs_s = reinterpret_cast<float2 *>(smem + OFF_OBS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
    uint64_t *stage_full = bars, *stage_empty = bars + 2, *acc_full = bars + 4, *acc_empty = bars + 6;
    uint64_t *const_full = bars + 8, *const_empty = bars + 12, *phi_ready = bars + 16;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + OFF_TSLOT);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + OFF_ABORT);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = a.tiles_per_out;
    const int G = NY * ntiles;                                  // tiles per step
    const int nsteps = PREDICT ? 2 : a.T;
    const long long total = (long long)G * nsteps;
    const int M = PREDICT ? 1 : a.M;

    if (warp == 1) {
        tmem_alloc(tslot, TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&stage_full[i], 1);
            mbar_init(&stage_empty[i], 1);
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], NEPI);
        }
        for (int i = 0; i < NCONST; ++i) {
            mbar_init(&const_full[i], 1);
            mbar_init(&const_empty[i], NEPI);
        }
        mbar_init(phi_ready, NEPI);
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int i = tid; i < a.cost.n_obs; i += NTHREADS) obs_s[i] = a.cost.obs[i];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // -------------------------------------------------------------- producer
        if (lane == 0) {
            long long issued = 0;
            for (long long g = 0; g < total; ++g) {
                const int s = (int)(g & 1), c = (int)(g & 3);
                bool ok = true;
                if (g >= 2) ok = mbar_wait_bounded(&stage_empty[s], (uint32_t)(((g >> 1) - 1) & 1), abort_flag);
                if (ok && g >= 4) ok = mbar_wait_bounded(&const_empty[c], (uint32_t)(((g >> 2) - 1) & 1), abort_flag);
                if (!ok) {
                    if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                    *abort_flag = 1;
                    break;
                }
                const long long tile = g % G;                   // (output, tile) in order
                mbar_arrive_expect_tx(&stage_full[s], TC_TILE_BYTES);
                bulk_g2s(smem + OFF_STAGE + s * TC_TILE_BYTES, a.wtiles + tile * TC_TILE_BYTES, TC_TILE_BYTES,
                         &stage_full[s]);
                mbar_arrive_expect_tx(&const_full[c], TC_CONST_BYTES);
                bulk_g2s(smem + OFF_CONST + c * TC_CONST_BYTES, a.wconst + tile * TC_CONST_BYTES, TC_CONST_BYTES,
                         &const_full[c]);
                issued = g + 1;
            }
            for (long long g = (issued > 4 ? issued - 4 : 0); g < issued; ++g) {
                if (g >= issued - 2 && !mbar_wait_drain(&stage_full[g & 1], (uint32_t)((g >> 1) & 1)))
                    atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
                if (!mbar_wait_drain(&const_full[g & 3], (uint32_t)((g >> 2) & 1)))
                    atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // -------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16_f32(BM, TNF);
            const uint32_t phi_hi = smem_u32(smem + OFF_PHI_HI), phi_lo = smem_u32(smem + OFF_PHI_LO);
            long long g = 0;
            bool ok = true;
            for (int t = 0; t < nsteps && ok; ++t) {
                ok = mbar_wait_bounded(phi_ready, (uint32_t)(t & 1), abort_flag);
                tc_fence_after();
                for (int j = 0; j < G && ok; ++j, ++g) {
                    const int s = (int)(g & 1), buf = (int)(g & 1);
                    ok = mbar_wait_bounded(&stage_full[s], (uint32_t)((g >> 1) & 1), abort_flag);
                    if (ok && g >= 2) ok = mbar_wait_bounded(&acc_empty[buf], (uint32_t)(((g >> 1) - 1) & 1), abort_flag);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + OFF_STAGE + s * TC_TILE_BYTES);
                    const uint32_t dS = tbase + buf * 128, dY = tbase + buf * 128 + 64;
                    const uint32_t sbo_a = 16 * KF, sbo_s = 16 * KF, sbo_y = 16 * KY;
#pragma unroll 1
                    for (int ks = 0; ks < KF / 16; ++ks) {
                        const uint64_t ah = smem_desc_kmajor(phi_hi + ks * 256, 128, sbo_a);
                        const uint64_t al = smem_desc_kmajor(phi_lo + ks * 256, 128, sbo_a);
                        const uint64_t bh = smem_desc_kmajor(st + TC_OFF_SHI + ks * 256, 128, sbo_s);
                        const uint64_t bl = smem_desc_kmajor(st + TC_OFF_SLO + ks * 256, 128, sbo_s);
                        mma_f16(dS, ah, bh, idesc, ks > 0);
                        mma_f16(dS, ah, bl, idesc, true);
                        mma_f16(dS, al, bh, idesc, true);
                    }
                    {
                        const uint64_t ah = smem_desc_kmajor(phi_hi, 128, sbo_a);
                        const uint64_t al = smem_desc_kmajor(phi_lo, 128, sbo_a);
                        const uint64_t bh = smem_desc_kmajor(st + TC_OFF_YHI, 128, sbo_y);
                        const uint64_t bl = smem_desc_kmajor(st + TC_OFF_YLO, 128, sbo_y);
                        mma_f16(dY, ah, bh, idesc, false);
                        mma_f16(dY, ah, bl, idesc, true);
                        mma_f16(dY, al, bh, idesc, true);
                    }
                    mma_commit(&stage_empty[s]);
                    mma_commit(&acc_full[buf]);
                }
            }
            if (!ok) {
                if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
                *abort_flag = 1;
            }
            // all MMAs issued must complete before the tensor memory is freed
            if (g > 0 && !mbar_wait_drain(&acc_full[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1)))
                atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------------- epilogue
        const int ew = warp - 2;
        const int q = warp & 3, h = ew >> 2;                 // lane quarter, column half
        const int r = 32 * q + lane;                         // slot row of this thread
        const bool owner = h == 0;
        const long long gslot = (long long)blockIdx.x * BM + r;
        const int k = (int)(gslot / M), m = (int)(gslot % M);
        const bool writer = owner && !PREDICT && k < a.K && m == 0;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;

        // initial feature tile
        if (owner) {
            float zext[17];
            if (PREDICT) {
                const bool okp = gslot < a.n_pred;
#pragma unroll
                for (int c = 0; c < NZ; ++c) zext[c] = okp ? a.z_in[(size_t)gslot * NZ + c] : 0.0f;
            } else {
                const float4 n = box_muller4(noise_block(a.seed, (uint32_t)k, 0u, 0u, 0u));
                const float eps[4] = {a.sqrt_sigma_u[0] * n.x, a.sqrt_sigma_u[1] * n.y, a.sqrt_sigma_u[2] * n.z,
                                      a.sqrt_sigma_u[3] * n.w};
#pragma unroll
                for (int c = 0; c < NX; ++c) {
                    zext[c] = a.x0[c];
                    xbuf[c * BM + r] = zext[c];
                }
#pragma unroll
                for (int c = 0; c < NU; ++c) zext[NX + c] = a.u_nom[c] + eps[c];
                if (writer) a.eps_tk[k] = make_float4(eps[0], eps[1], eps[2], eps[3]);
            }
            zext[16] = 1.0f;
#pragma unroll
            for (int c = 0; c < NZ; ++c) zbuf[c * BM + r] = zext[c];
#pragma unroll
            for (int o = 0; o < NY; ++o) yrbuf[o * BM + r] = 0.0f;
            build_features(smem, r, zext);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(phi_ready);
        // both column halves read the owners' y_ref (and x) of step 0
        named_bar_sync(1, NE);

        long long g = 0;
        bool aborted = false;
        for (int t = 0; t < nsteps; ++t) {
            for (int o = 0; o < NY; ++o) {
                const float yref = yrbuf[o * BM + r];
                Soft st{-INFINITY, 0.f, 0.f, 0.f, 0.f};
                for (int j = 0; j < ntiles; ++j, ++g) {
                    const int buf = (int)(g & 1), c = (int)(g & 3);
                    if (!aborted && !mbar_wait_bounded(&acc_full[buf], (uint32_t)((g >> 1) & 1), abort_flag))
                        aborted = true;
                    aborted = __any_sync(0xffffffffu, aborted);   // the TMEM loads below are warp-collective
                    tc_fence_after();
                    if (!aborted && !mbar_wait_bounded(&const_full[c], (uint32_t)((g >> 2) & 1), abort_flag))
                        aborted = true;
                    aborted = __any_sync(0xffffffffu, aborted);
                    const float *cs = reinterpret_cast<const float *>(smem + OFF_CONST + c * TC_CONST_BYTES) + h * 32;
                    const float *cy = cs + TNF;
                    const float *cv = cs + 2 * TNF;
                    const uint32_t base = tbase + lane_off + buf * 128 + h * 32;
#pragma unroll
                    for (int ch = 0; ch < 2; ++ch) {
                        float sv[16], yv[16];
                        if (!aborted) tmem_ld16x2_wait(base + 16 * ch, base + 64 + 16 * ch, sv, yv);
                        if (ch == 1) {
                            // both halves of the accumulator read: hand the buffer back
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&acc_empty[buf]);
                        }
                        if (!aborted) {
                            float sm = -INFINITY;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                sv[i] += cs[16 * ch + i];
                                sm = fmaxf(sm, sv[i]);
                            }
                            const float mn = fmaxf(st.m, sm);
                            const float mns = mn == -INFINITY ? 0.0f : mn;
                            const float sc = ex2(st.m - mns);
                            float s0 = st.s0 * sc, s1 = st.s1 * sc, s2 = st.s2 * sc, s3 = st.s3 * sc;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const float w = ex2(sv[i] - mns);
                                const float e = yv[i] + (cy[16 * ch + i] - yref);
                                const float we = w * e;
                                s0 += w;
                                s1 += we;
                                s2 = fmaf(we, e, s2);
                                s3 = fmaf(w, cv[16 * ch + i], s3);
                            }
                            st = Soft{mn, s0, s1, s2, s3};
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&const_empty[c]);
                }
                // merge the two column halves of this output
                float *pb = part + (o & 1) * 5 * BM;
                if (!owner) {
                    pb[0 * BM + r] = st.m;
                    pb[1 * BM + r] = st.s0;
                    pb[2 * BM + r] = st.s1;
                    pb[3 * BM + r] = st.s2;
                    pb[4 * BM + r] = st.s3;
                }
                named_bar_sync(1, NE);
                if (owner) {
                    const Soft other{pb[0 * BM + r], pb[1 * BM + r], pb[2 * BM + r], pb[3 * BM + r], pb[4 * BM + r]};
                    merge_into(st, other);
                    const float inv = 1.0f / st.s0;
                    const float me = st.s1 * inv;
                    ybuf[o * BM + r] = yref + me;
                    vbuf[o * BM + r] = fmaxf(fmaf(-me, me, st.s2 * inv), 0.0f) + st.s3 * inv;
                }
            }

            // ---------------------------------------------------------- dynamics
            if (owner) {
                float y[NY], var[NY], zext[17];
#pragma unroll
                for (int o = 0; o < NY; ++o) {
                    y[o] = ybuf[o * BM + r];
                    var[o] = vbuf[o * BM + r];
                }
                if (PREDICT) {
                    if (t == 0) {
#pragma unroll
                        for (int o = 0; o < NY; ++o) yrbuf[o * BM + r] = y[o];
                    } else if (gslot < a.n_pred) {
#pragma unroll
                        for (int o = 0; o < NY; ++o) {
                            a.y_out[(size_t)gslot * NY + o] = y[o];
                            a.var_out[(size_t)gslot * NY + o] = var[o];
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NZ; ++c) zext[c] = zbuf[c * BM + r];
                } else {
                    float x[NX];
#pragma unroll
                    for (int c = 0; c < NX; ++c) x[c] = xbuf[c * BM + r];
                    qbuf[r] = running_cost(a.cost, obs_s, x, var);
                    float n[NY];
                    if (a.model_noise) {
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            const float4 nb = box_muller4(
                                noise_block(a.seed, (uint32_t)k, (uint32_t)t, (uint32_t)(b + 1), (uint32_t)m));
                            n[4 * b] = nb.x;
                            n[4 * b + 1] = nb.y;
                            n[4 * b + 2] = nb.z;
                            n[4 * b + 3] = nb.w;
                        }
                    } else {
#pragma unroll
                        for (int o = 0; o < NY; ++o) n[o] = 0.0f;
                    }
#pragma unroll
                    for (int c = 0; c < NX; ++c) {
                        const float xdot = fmaf(sqrtf(var[c]), n[c], y[c]);
                        x[c] = fmaf(a.dt, xdot, x[c]);
                        xbuf[c * BM + r] = x[c];
                        zext[c] = x[c];
                        yrbuf[c * BM + r] = y[c];
                    }
                    named_bar_sync(2, BM);
                    if (writer) {
                        float qs = 0.0f;
                        for (int i = 0; i < M; ++i) qs += qbuf[r + i];
                        a.cost_tk[(size_t)t * a.K + k] = qs / (float)M;
                    }
                    if (t + 1 < a.T) {
                        const float4 nn =
                            box_muller4(noise_block(a.seed, (uint32_t)k, (uint32_t)(t + 1), 0u, 0u));
                        const float eps[4] = {a.sqrt_sigma_u[0] * nn.x, a.sqrt_sigma_u[1] * nn.y,
                                              a.sqrt_sigma_u[2] * nn.z, a.sqrt_sigma_u[3] * nn.w};
#pragma unroll
                        for (int c = 0; c < NU; ++c) zext[NX + c] = a.u_nom[(size_t)(t + 1) * NU + c] + eps[c];
                        if (writer)
                            a.eps_tk[(size_t)(t + 1) * a.K + k] = make_float4(eps[0], eps[1], eps[2], eps[3]);
                    } else {
#pragma unroll
                        for (int c = 0; c < NU; ++c) zext[NX + c] = 0.0f;
                        named_bar_sync(2, BM);
                        qbuf[r] = terminal_cost(a.cost, x);
                        named_bar_sync(2, BM);
                        if (writer) {
                            float ps = 0.0f;
                            for (int i = 0; i < M; ++i) ps += qbuf[r + i];
                            a.phi[k] = ps / (float)M;
                        }
                    }
                }
                zext[16] = 1.0f;
                if (t + 1 < nsteps) build_features(smem, r, zext);
            }
            const bool any_abort = bar_sync_or(3, NE, aborted || *abort_flag != 0);
            if (any_abort) break;
            if (t + 1 < nsteps) {
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(phi_ready);
            }
        }
        if (aborted || *abort_flag) {
            if (lane == 0 && !*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
            *abort_flag = 1;
        }
    }

    // all roles done: free the tensor memory
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, TMEM_COLS);
    }
}

bool g_tc_attr[2] = {false, false};
char g_tc_diag[256] = "";

template <bool PREDICT>
cudaError_t launch_tc_impl(const TcArgs &a, cudaStream_t s, long long slots)
{
    if (a.cost.n_obs > MAX_OBS || a.tiles_per_out <= 0) return cudaErrorInvalidValue;
    if (!g_tc_attr[PREDICT]) {
        cudaError_t e = cudaFuncSetAttribute(rollout_tc_kernel<PREDICT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, rollout_tc_kernel<PREDICT>);
        if (e != cudaSuccess) return e;
        snprintf(g_tc_diag, sizeof g_tc_diag,
                 "regs %d, maxThreadsPerBlock %d, dynamic smem %d (max %d), static smem %zu, local %zu",
                 fa.numRegs, fa.maxThreadsPerBlock, SMEM_BYTES, fa.maxDynamicSharedSizeBytes, fa.sharedSizeBytes,
                 fa.localSizeBytes);
        if (fa.maxThreadsPerBlock < NTHREADS) return cudaErrorLaunchOutOfResources;
        g_tc_attr[PREDICT] = true;
    }
    const long long blocks = (slots + BM - 1) / BM;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    rollout_tc_kernel<PREDICT><<<(unsigned)blocks, NTHREADS, SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

const char *tc_launch_diag() { return g_tc_diag; }

cudaError_t launch_rollout_tc(const TcArgs &a, cudaStream_t s)
{
    if (a.M < 1 || a.M > BM || (a.M & (a.M - 1)) != 0) return cudaErrorInvalidValue;
    return launch_tc_impl<false>(a, s, (long long)a.K * a.M);
}

cudaError_t launch_predict_tc(const TcArgs &a, cudaStream_t s)
{
    return launch_tc_impl<true>(a, s, (long long)a.n_pred);
}

}  // namespace pi2rh

// rollout_tc.cu -- tensor-core form of the fused rollout kernel.
//
// The receptive-field exponents and local predictions (Sec. 2, Eq. 1) of all
// 12 L fields are evaluated for 128 rollout slots at a time as two GEMMs on
// the 5th-generation tensor cores:
//   s_j = -(1/2) log2(e) (z - c_j)^T D_j (z - c_j) = phi(z) . w_j,
//         phi(z) = [z_a (16), z_a z_b (a <= b, 136), 1, 0 (7)]
//   y_j = b_j + beta_j . (z - c_j) = z . beta_j + cy_j
// with w_j = [2k (D_s c_j)_a, -k D'_ab, cs_j, 0], k = log2(e)/2,
// D_s = (D + D^T)/2, D'_aa = D_aa, D'_ab = D_ab + D_ba and the constant
// cs_j = -k c_j^T D_s c_j (the weight of the constant feature); the constant
// cy_j = b_j - beta_j . c_j is added in FP32 in the epilogue.  A padding field
// of a ragged last tile has the weight -inf on the constant feature and 0
// elsewhere, so its exponent is -inf and its softmax weight 0.
//
// Precision: operands are split into fp16 hi + lo parts and each product is
// formed as hi*hi + hi*lo + lo*hi (three tcgen05.mma kind::f16 per K step,
// fp32 accumulation in tensor memory); the dropped lo*lo term is ~2^-22
// relative, so the exponents carry FP32-level accuracy.  The constant feature
// is split as 1 + 2^-14 (its weight's lo part compensates), so that the
// lo*hi product of a padding field is 2^-14 * -inf, never 0 * -inf.
//
// Roles (one CTA per SM, 128 slots, 320 threads):
//   warp 0:        producer (one elected lane issues) -- 1-D bulk copies
//                  (TMA) of the pre-packed coefficient chunks (8 KB each,
//                  11 per tile of 128 fields) in NGRP groups per tile
//                  (one copy and one barrier pair each) into a ring that
//                  holds one tile, and of the per-field
//                  constants (cy, sigma^2) into a 4-deep constant ring;
//   warp 1:        MMA issuer (the whole warp runs the loop, one elected
//                  lane issues) -- per tile of 128 fields, 30 MMAs (M=128,
//                  K=16, 3 split products per K step: K step 0 of S and the
//                  Y GEMM as one N=256 MMA, K steps 1-9 with N=128) into one
//                  of two TMEM accumulator buffers, releasing each chunk
//                  group as soon as its MMAs complete;
//   warps 2-9:     epilogue -- tcgen05.ld of S and Y, online base-2 softmax
//                  per output on packed FP32x2 operations (chunks of 16
//                  fields, one rescale per chunk; running sums of w, w e and
//                  w (e^2 + sigma^2)), merge of the two column halves, then
//                  the dynamics step (cost, Euler step, Philox noise) and
//                  the feature tile of the next step.
// Launch forms: one CTA per 128-slot block; clusters of 2-4 CTAs that split a
// block's 12 outputs when the blocks alone would leave SMs idle (means and
// variances exchanged through distributed shared memory); a persistent
// work-list form and a one-wave group form for batches.
// Every wait is bounded; on expiry the kernel flags the device error word,
// drains its copies and MMAs, frees its tensor memory and returns.
#include <array>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include <cuda_fp16.h>

#include "pi2rh_kernels.h"
#include "tc_ptx.cuh"

namespace pi2rh {

namespace {

constexpr int BM = TC_SLOTS;            // rollout slots per CTA (MMA M)
constexpr int TNF = TC_TILE_FIELDS;     // fields per tile (MMA N)
constexpr int KF = TC_KF;               // feature columns of phi (S GEMM K)
constexpr int NCH = TC_CHUNKS_PER_TILE; // chunks per tile
// The chunk ring holds one tile, in NGRP copy groups of consecutive chunks
// (group x = chunks GRP_BEGIN[x] .. GRP_BEGIN[x + 1] - 1, in the ring slots of
// the same index); each group is one bulk copy and one full/empty barrier
// pair, so every slot, descriptor offset and barrier of the MMA issuer's
// per-tile sequence is a compile-time constant.  A group is refilled for the
// next tile as soon as this tile's MMAs that read it are done, so the copy
// has the other groups' MMAs to land in.
constexpr int NSLOT = NCH;              // chunk slots in the ring (one tile)
// Two groups, chunks 0-5 and 6-10 (three groups of 4/4/3 and four of 3/3/3/2
// chunks measured the same: the refill of a group lands in time either way)
constexpr int NGRP = 2;
__host__ __device__ constexpr int grp_begin(int x) { return x == 0 ? 0 : x == 1 ? 6 : NCH; }
static_assert(grp_begin(1) >= 2 && grp_begin(NGRP) == NCH, "group 0 holds the N = 256 chunk pair");
constexpr int NCONST = 4;
constexpr int NEPI = 8;                 // epilogue warps
constexpr int NTHREADS = (2 + NEPI) * 32;
constexpr int NE = NEPI * 32;
constexpr int MAX_OBS = 256;
constexpr int HALF = TNF / 2;           // columns per epilogue warp

constexpr int PHI_BYTES = BM * KF * 2;                 // one fp16 feature tile
constexpr int OFF_PHI_HI = 0;
constexpr int OFF_PHI_LO = OFF_PHI_HI + PHI_BYTES;
constexpr int OFF_RING = OFF_PHI_LO + PHI_BYTES;
constexpr int OFF_CONST = OFF_RING + NSLOT * TC_CHUNK_BYTES;
constexpr int NSUM = 4;                 // softmax state: max, sums of w, w e, w (e^2 + sigma^2)
constexpr int OFF_PART = OFF_CONST + NCONST * TC_CONST_BYTES;   // [2][NSUM][BM]
constexpr int OFF_Z = OFF_PART + 2 * NSUM * BM * 4;             // [NZ][BM]
constexpr int OFF_X = OFF_Z + NZ * BM * 4;                      // [NX][BM]
constexpr int OFF_Y = OFF_X + NX * BM * 4;                      // [NY][BM]
constexpr int OFF_V = OFF_Y + NY * BM * 4;
constexpr int OFF_YREF = OFF_V + NY * BM * 4;
constexpr int OFF_Q = OFF_YREF + NY * BM * 4;                   // [BM]
constexpr int OFF_N = OFF_Q + BM * 4;                           // [NY + NU][BM] normals of the step
constexpr int OFF_SD = OFF_N + (NY + NU) * BM * 4;              // [NY][BM] sqrt of the variances
constexpr int OFF_OBS = OFF_SD + NY * BM * 4;
constexpr int OFF_BAR = OFF_OBS + MAX_OBS * 8;
// barriers: full[NGRP], empty[NGRP], acc_full[2], acc_empty[2],
//           const_full[4], const_empty[4], phi_ready, xfull, xfree, drain
constexpr int NBARS = 2 * NGRP + 4 + 2 * NCONST + 4;
constexpr int OFF_TSLOT = OFF_BAR + NBARS * 8;
constexpr int OFF_ABORT = OFF_TSLOT + 8;
constexpr int SMEM_BYTES = OFF_ABORT + 16;
static_assert(OFF_RING % 128 == 0 && OFF_CONST % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
static_assert(OFF_SD % 16 == 0, "alignment");
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

constexpr uint32_t TMEM_COLS = 512;     // 2 buffers x (S 128 + Y 128)

// Feature k of phi: k < 16 -> z_k * 1; 16 <= k < 152 -> z_a z_b; 152 -> 1
// (split as 1 + 2^-14 by split_pair); k > 152 -> 0.
__host__ __device__ constexpr int feat_a(int k) { return k < 16 ? k : tc_feat_row(k); }
__host__ __device__ constexpr int feat_b(int k) { return k < 16 ? 16 : tc_feat_col(k); }

// Online softmax state of one output for one slot: the running maximum m of
// the exponents and, relative to 2^m, the sums of w, w e and w (e^2 +
// sigma^2), e = y_j - y_ref.
struct Soft {
    float m, s0, s1, s2;
};

__device__ __forceinline__ void merge_into(Soft &a, const Soft &b)
{
    const float M = fmaxf(a.m, b.m);
    const float Ms = M == -INFINITY ? 0.0f : M;
    const float ca = ex2(a.m - Ms), cb = ex2(b.m - Ms);
    a.s0 = fmaf(a.s0, ca, b.s0 * cb);
    a.s1 = fmaf(a.s1, ca, b.s1 * cb);
    a.s2 = fmaf(a.s2, ca, b.s2 * cb);
    a.m = M;
}

__device__ __forceinline__ float max3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Folds the 16 fields of one chunk (exponents sv, local predictions without
// their constant yv) into the softmax state, two fields per packed FP32x2
// operation (even and odd columns accumulate separately and are added at the
// end).
__device__ __forceinline__ void soft_chunk(Soft &st, const float (&sv)[16], const float (&yv)[16],
                                           const float2 *cy2, const float2 *cv2, float yref)
{
    float2 sp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) sp[i] = make_float2(sv[2 * i], sv[2 * i + 1]);
    const float m0 = max3(sp[0].x, sp[0].y, sp[1].x), m1 = max3(sp[1].y, sp[2].x, sp[2].y);
    const float m2 = max3(sp[3].x, sp[3].y, sp[4].x), m3 = max3(sp[4].y, sp[5].x, sp[5].y);
    const float m4 = max3(sp[6].x, sp[6].y, sp[7].x);
    const float mn = max3(max3(m0, m1, m2), max3(m3, m4, sp[7].y), st.m);
    const float mns = mn == -INFINITY ? 0.0f : mn;
    const float sc = ex2(st.m - mns);
    const float2 nm = make_float2(-mns, -mns), ny = make_float2(-yref, -yref);
    float2 s0 = make_float2(st.s0 * sc, 0.0f), s1 = make_float2(st.s1 * sc, 0.0f);
    float2 s2 = make_float2(st.s2 * sc, 0.0f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 d = __fadd2_rn(sp[i], nm);
        const float2 w = make_float2(ex2(d.x), ex2(d.y));
        const float2 e = __fadd2_rn(make_float2(yv[2 * i], yv[2 * i + 1]), __fadd2_rn(cy2[i], ny));
        s0 = __fadd2_rn(s0, w);
        s1 = __ffma2_rn(w, e, s1);
        s2 = __ffma2_rn(w, __ffma2_rn(e, e, cv2[i]), s2);
    }
    st = Soft{mn, s0.x + s0.y, s1.x + s1.y, s2.x + s2.y};
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
    } else if constexpr (K == TC_CONST_FEATURE) {
        return 1.0f;
    } else {
        return 0.0f;
    }
}

// Features K and K+1 as fp16 hi and lo pairs (hi = f rounded to fp16, lo = the
// exact FP32 remainder f - hi rounded to fp16), two at a time on packed
// conversions.  The constant feature's lo part is 2^-14 (see the header).
template <int K>
__device__ __forceinline__ void split_pair(const float (&zext)[17], uint32_t &hw, uint32_t &lw)
{
    const float2 f = make_float2(feature<K>(zext), feature<K + 1>(zext));
    const __half2 h = __floats2half2_rn(f.x, f.y);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(f.x - hf.x, f.y - hf.y);
    hw = *reinterpret_cast<const uint32_t *>(&h);
    if constexpr (K == TC_CONST_FEATURE)
        lw = pack_h2(__ushort_as_half((unsigned short)0x0400u), __high2half(l));   // 2^-14
    else
        lw = *reinterpret_cast<const uint32_t *>(&l);
}

// Writes the hi/lo fp16 feature rows of slot r from z (zext[16] == 1), one
// 16-byte core-matrix row (8 features) at a time: rows K8 .. K8END - 1.
template <int K8 = 0, int K8END = KF / 8>
__device__ __forceinline__ void build_features(unsigned char *smem, int r, const float (&zext)[17])
{
    if constexpr (K8 < K8END) {
        uint32_t hw[4], lw[4];
        split_pair<K8 * 8 + 0>(zext, hw[0], lw[0]);
        split_pair<K8 * 8 + 2>(zext, hw[1], lw[1]);
        split_pair<K8 * 8 + 4>(zext, hw[2], lw[2]);
        split_pair<K8 * 8 + 6>(zext, hw[3], lw[3]);
        const uint32_t off = kmajor_offset(r, K8 * 8, KF);
        *reinterpret_cast<uint4 *>(smem + OFF_PHI_HI + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(smem + OFF_PHI_LO + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        build_features<K8 + 1, K8END>(smem, r, zext);
    }
}

struct TcSmem {
    unsigned char *base;
    float *part, *zbuf, *xbuf, *ybuf, *vbuf, *yrbuf, *qbuf, *nbuf, *sdbuf;
    float2 *obs_s;
    uint64_t *full, *empty, *acc_full, *acc_empty, *const_full, *const_empty, *phi_ready;
    uint64_t *xfull, *xfree;   // output exchange between the CTAs of a cluster (split form)
    uint64_t *drain;           // the issuer's last commit after a timeout
    uint32_t *tslot;
    volatile int *abort_flag;
};

__device__ __forceinline__ TcSmem tc_smem(unsigned char *smem)
{
    TcSmem S;
    S.base = smem;
    S.part = reinterpret_cast<float *>(smem + OFF_PART);
    S.zbuf = reinterpret_cast<float *>(smem + OFF_Z);
    S.xbuf = reinterpret_cast<float *>(smem + OFF_X);
    S.ybuf = reinterpret_cast<float *>(smem + OFF_Y);
    S.vbuf = reinterpret_cast<float *>(smem + OFF_V);
    S.yrbuf = reinterpret_cast<float *>(smem + OFF_YREF);
    S.qbuf = reinterpret_cast<float *>(smem + OFF_Q);
    S.nbuf = reinterpret_cast<float *>(smem + OFF_N);
    S.sdbuf = reinterpret_cast<float *>(smem + OFF_SD);
    S.obs_s = reinterpret_cast<float2 *>(smem + OFF_OBS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
    S.full = bars;
    S.empty = bars + NGRP;
    S.acc_full = bars + 2 * NGRP;
    S.acc_empty = S.acc_full + 2;
    S.const_full = S.acc_empty + 2;
    S.const_empty = S.const_full + NCONST;
    S.phi_ready = S.const_empty + NCONST;
    S.xfull = S.phi_ready + 1;
    S.xfree = S.phi_ready + 2;
    S.drain = S.phi_ready + 3;
    S.tslot = reinterpret_cast<uint32_t *>(smem + OFF_TSLOT);
    S.abort_flag = reinterpret_cast<volatile int *>(smem + OFF_ABORT);
    return S;
}

// One-time set-up: TMEM allocation (warp 1) and barrier initialization
// (thread 0).  ncl = CTAs in the cluster (1 unless the outputs are split).
__device__ __forceinline__ void tc_setup(const TcSmem &S, uint32_t ncl)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 1) {
        tmem_alloc(S.tslot, TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < NGRP; ++i) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.acc_full[i], 1);
            mbar_init(&S.acc_empty[i], NEPI);
        }
        for (int i = 0; i < NCONST; ++i) {
            mbar_init(&S.const_full[i], 1);
            mbar_init(&S.const_empty[i], NEPI);
        }
        mbar_init(S.phi_ready, NEPI);
        // every owner thread of every other CTA arrives once per step
        const uint32_t xc = ncl > 1 ? (ncl - 1) * BM : 1;
        mbar_init(S.xfull, xc);
        mbar_init(S.xfree, xc);
        mbar_init(S.drain, 1);
        *S.abort_flag = 0;
        fence_mbar_init();
    }
}

// Persistent per-role positions (carried across work items): g counts the
// tiles whose copies (producer) or MMAs (issuer) have been issued; ts counts
// the issuer's steps (feature tiles).  The tile counter fixes every ring
// position and barrier phase: tile g uses constant slot g & 3, chunk groups
// A and B at phase g & 1, accumulator buffer g & 1.
struct TcProducer {
    long long g = 0;              // tiles started
    long long n[NGRP] = {};       // copies of each group issued
};
struct TcIssuer {
    long long g = 0, ts = 0;
    bool drained = false;   // committed to the drain barrier after a timeout
};

// Producer (all of warp 0; one elected lane issues the copies) for one work
// item -- the tiles of outputs o_begin .. o_begin + n_out - 1, every step --;
// false after a timeout.  Per tile: its constants into the 4-deep constant
// ring, then each copy group once the MMAs of the previous tile that read the
// group's slots are done.  A tile's chunks are contiguous in global memory, so
// each group is one copy.
template <bool PREDICT>
__device__ bool tc_producer_item(const TcArgs &a, const TcSmem &S, TcProducer &P, int o_begin, int n_out)
{
    unsigned char *smem = S.base;
    uint64_t *full = S.full, *empty = S.empty, *const_full = S.const_full, *const_empty = S.const_empty;
    volatile int *abort_flag = S.abort_flag;
    const int G = n_out * a.tiles_per_out;
    const long long tile0 = (long long)o_begin * a.tiles_per_out;
    const int nsteps = PREDICT ? 2 : a.T;
    bool ok = true;
    for (int t = 0; t < nsteps && ok; ++t) {
        for (int jt = 0; jt < G; ++jt) {
            const long long gt = P.g;
            const long long tile = tile0 + jt;
            const unsigned char *src = a.wtiles + tile * TC_TILE_BYTES;
            const int c = (int)(gt & 3);
            if (gt >= 4)
                ok = __all_sync(0xffffffffu,
                                mbar_wait_bounded(&const_empty[c], (uint32_t)(((gt >> 2) - 1) & 1), abort_flag));
            if (!ok) break;
            if (elect_one()) {
                mbar_arrive_expect_tx(&const_full[c], TC_CONST_BYTES);
                bulk_g2s(smem + OFF_CONST + c * TC_CONST_BYTES, a.wconst + tile * TC_CONST_BYTES, TC_CONST_BYTES,
                         &const_full[c]);
            }
            __syncwarp();
            P.g = gt + 1;
            const uint32_t prev = (uint32_t)((gt - 1) & 1);   // phase of the previous tile's groups
#pragma unroll
            for (int x = 0; x < NGRP; ++x) {
                if (gt >= 1) ok = __all_sync(0xffffffffu, mbar_wait_bounded(&empty[x], prev, abort_flag));
                if (!ok) break;
                const int c0 = grp_begin(x), nc = grp_begin(x + 1) - grp_begin(x);
                if (elect_one()) {
                    mbar_arrive_expect_tx(&full[x], (uint32_t)(nc * TC_CHUNK_BYTES));
                    bulk_g2s(smem + OFF_RING + c0 * TC_CHUNK_BYTES, src + c0 * TC_CHUNK_BYTES,
                             (uint32_t)(nc * TC_CHUNK_BYTES), &full[x]);
                }
                __syncwarp();
                P.n[x] = gt + 1;
            }
            if (!ok) break;
        }
    }
    return ok;
}

// The MMAs of chunks J..J1-1 of a tile (all in the ring slots of the same
// index): chunk 1 issues the N = 256 triple of K step 0 of S (columns 0-127)
// and the Y GEMM (128-255), whose B operand is chunks 0 and 1 (hi and lo,
// 256 rows each); chunk j >= 2 issues the N = 128 triple of K step j - 1, or
// with QP = 2 on the quadratic-feature K steps 1-8 the pair A_hi B_hi +
// A_hi B_lo.
template <int J, int J1, int QP>
__device__ __forceinline__ void tc_issue_chunks(uint32_t dS, uint64_t a_hi, uint64_t a_lo, uint64_t b0,
                                                uint32_t idesc, uint32_t idesc_wide)
{
    if constexpr (J < J1) {
        constexpr uint64_t CH = TC_CHUNK_BYTES >> 4;
        if constexpr (J == 1) {
            mma3_elect(dS, a_hi, a_lo, b0, b0 + CH, idesc_wide, 0u);
        } else if constexpr (J >= 2) {
            constexpr uint64_t ka = (uint64_t)((J - 1) * 16);
            constexpr uint64_t bl = J * CH + (uint64_t)(TC_HALF_CHUNK >> 4);
            if constexpr (QP == 2 && J <= TC_QUAD_LAST_CHUNK)
                mma2_elect(dS, a_hi + ka, b0 + J * CH, b0 + bl, idesc);
            else
                mma3_elect(dS, a_hi + ka, a_lo + ka, b0 + J * CH, b0 + bl, idesc, 1u);
        }
        tc_issue_chunks<J + 1, J1, QP>(dS, a_hi, a_lo, b0, idesc, idesc_wide);
    }
}

// The copy groups of one tile from group X on: wait for the group's chunks,
// issue their MMAs, release the group's slots (the commit arrives when those
// MMAs are done); false after a timeout.
template <int X, int QP>
__device__ __forceinline__ bool tc_issue_groups(const TcSmem &S, uint32_t dS, uint64_t a_hi, uint64_t a_lo,
                                                uint64_t b0, uint32_t idesc, uint32_t idesc_wide, uint32_t ph)
{
    if constexpr (X < NGRP) {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&S.full[X], ph, S.abort_flag))) return false;
        tc_fence_after();
        tc_issue_chunks<grp_begin(X), grp_begin(X + 1), QP>(dS, a_hi, a_lo, b0, idesc, idesc_wide);
        commit_elect(&S.empty[X]);
        return tc_issue_groups<X + 1, QP>(S, dS, a_hi, a_lo, b0, idesc, idesc_wide, ph);
    }
    return true;
}

// MMA issuer (all of warp 1) for one work item; false after a timeout.  The
// whole warp runs the loop, so every counter and descriptor is warp-uniform,
// and the lane elect.sync picks issues the MMAs and commits.  (The issuing
// warp shares its scheduler with two epilogue warps, so every instruction of
// this loop costs issue slots on the critical path: the per-tile sequence
// below has no per-chunk bookkeeping.)  Per tile: wait for a free accumulator,
// then for each copy group its MMAs (tc_issue_groups), then signal the
// accumulator.
template <bool PREDICT, int QP>
__device__ bool tc_issuer_item(const TcArgs &a, const TcSmem &S, uint32_t tbase, TcIssuer &I, int n_out)
{
    unsigned char *smem = S.base;
    uint64_t *full = S.full, *empty = S.empty, *acc_full = S.acc_full, *acc_empty = S.acc_empty;
    uint64_t *phi_ready = S.phi_ready;
    volatile int *abort_flag = S.abort_flag;
    const int G = n_out * a.tiles_per_out;
    const int nsteps = PREDICT ? 2 : a.T;
    const uint32_t idesc = idesc_f16_f32(BM, TNF), idesc_wide = idesc_f16_f32(BM, 2 * TNF);
    // descriptors: A = feature tile K step j (rows 2560 B apart; step j at
    // +256 B), B = a chunk half (128 rows x 16 K, rows 256 B apart; 256 rows
    // for the whole first two chunks); chunk and half offsets are added to the
    // 14-bit start field (>> 4; the addresses stay < 256 KB).
    const uint64_t a_hi = smem_desc_kmajor(smem_u32(smem + OFF_PHI_HI), 128, 16 * KF);
    const uint64_t a_lo = smem_desc_kmajor(smem_u32(smem + OFF_PHI_LO), 128, 16 * KF);
    const uint64_t b0 = smem_desc_kmajor(smem_u32(smem + OFF_RING), 128, 256);
    long long g = I.g;
    bool ok = true;
    for (int t = 0; t < nsteps && ok; ++t) {
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(phi_ready, (uint32_t)(I.ts & 1), abort_flag));
        ++I.ts;
        tc_fence_after();
        for (int jt = 0; jt < G && ok; ++jt, ++g) {
            const int buf = (int)(g & 1);
            const uint32_t ph = (uint32_t)(g & 1);
            if (g >= 2)
                ok = __all_sync(0xffffffffu,
                                mbar_wait_bounded(&acc_empty[buf], (uint32_t)(((g >> 1) - 1) & 1), abort_flag));
            if (!ok) break;
            const uint32_t dS = tbase + buf * 256;   // S: columns 0-127, Y: 128-255
            ok = tc_issue_groups<0, QP>(S, dS, a_hi, a_lo, b0, idesc, idesc_wide, ph);
            if (!ok) break;
            commit_elect(&acc_full[buf]);
        }
    }
    // after a timeout, one commit on the drain barrier (which nothing else
    // completes) covers every MMA issued; the drain waits for it
    if (!ok) {
        commit_elect(S.drain);
        I.drained = true;
    }
    I.g = g;
    return ok;
}

// Epilogue warps (2-9) for one work item: the 128 slots starting at
// slot_base, outputs o_begin .. o_begin + n_out - 1.  With ncl > 1 CTAs in
// the cluster (split form, rollouts only), every CTA evaluates its own share
// of the outputs, sends each one's means and variances to the other CTAs'
// y / var buffers (distributed shared memory) right after its merge, behind
// the next output's tiles, and at the end of the step steps the dynamics of
// all 128 slots itself -- the same arithmetic on the same values in every
// CTA; only rank 0 writes the outputs.  Per step, xfull completes when the
// other CTAs' values have landed and xfree when they have read this CTA's
// previous ones, so a CTA is never more than one step ahead of another.
template <bool PREDICT, int NSPLIT>
__device__ void tc_epilogue_item(const TcArgs &a, const TcSmem &S, uint32_t tbase, long long slot_base, long long &g,
                                 bool &aborted, uint32_t rank)
{
    constexpr int n_out = NY / NSPLIT;
    constexpr uint32_t ncl = NSPLIT;
    const int o_begin = (int)rank * n_out;
    unsigned char *smem = S.base;
    float *part = S.part, *zbuf = S.zbuf, *xbuf = S.xbuf, *ybuf = S.ybuf, *vbuf = S.vbuf, *yrbuf = S.yrbuf,
          *qbuf = S.qbuf, *nbuf = S.nbuf, *sdbuf = S.sdbuf;
    float2 *obs_s = S.obs_s;
    uint64_t *acc_full = S.acc_full, *acc_empty = S.acc_empty, *const_full = S.const_full,
             *const_empty = S.const_empty, *phi_ready = S.phi_ready;
    volatile int *abort_flag = S.abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    (void)tid;
    const int ntiles = a.tiles_per_out;
    const int nsteps = PREDICT ? 2 : a.T;
    const int M = PREDICT ? 1 : a.M;
    const int ew = warp - 2;
    const int q = warp & 3, h = ew >> 2;                 // lane quarter, column half
    const int r = 32 * q + lane;                         // slot row of this thread
    const bool owner = h == 0;
    const long long gslot = slot_base + r;
    const int k = (int)(gslot / M), m = (int)(gslot % M);
    const bool writer = owner && rank == 0 && !PREDICT && k < a.K && m == 0;
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

    for (int t = 0; t < nsteps; ++t) {
        // The normals of this step (model noise) and the next step's controls
        // do not depend on the state: the other column half draws them while
        // every epilogue warp waits for the step's first tile, off the serial
        // dynamics step at the end of the step.  The owners read them there,
        // after barrier 4; the end-of-step barrier 3 orders these writes after
        // the previous step's reads.
        if (!PREDICT && !owner) {
            if (a.model_noise) {
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float4 nb =
                        box_muller4(noise_block(a.seed, (uint32_t)k, (uint32_t)t, (uint32_t)(b + 1), (uint32_t)m));
                    nbuf[(4 * b + 0) * BM + r] = nb.x;
                    nbuf[(4 * b + 1) * BM + r] = nb.y;
                    nbuf[(4 * b + 2) * BM + r] = nb.z;
                    nbuf[(4 * b + 3) * BM + r] = nb.w;
                }
            }
            if (t + 1 < a.T) {
                // the next step's controls u = u_nom + eps (and eps itself to the output)
                const float4 nn = box_muller4(noise_block(a.seed, (uint32_t)k, (uint32_t)(t + 1), 0u, 0u));
                const float eps[4] = {a.sqrt_sigma_u[0] * nn.x, a.sqrt_sigma_u[1] * nn.y, a.sqrt_sigma_u[2] * nn.z,
                                      a.sqrt_sigma_u[3] * nn.w};
#pragma unroll
                for (int c = 0; c < NU; ++c) nbuf[(NY + c) * BM + r] = a.u_nom[(size_t)(t + 1) * NU + c] + eps[c];
                if (rank == 0 && k < a.K && m == 0)
                    a.eps_tk[(size_t)(t + 1) * a.K + k] = make_float4(eps[0], eps[1], eps[2], eps[3]);
            }
            named_bar_arrive(4, NE);
        }
        // split form: the other CTAs have read this CTA's values of the last
        // step before any of this step's are sent (after each merge below)
        if (!PREDICT && ncl > 1 && owner && t > 0 && !aborted &&
            !mbar_wait_cluster_bounded(S.xfree, (uint32_t)((t - 1) & 1), abort_flag))
            aborted = true;
        for (int o = o_begin; o < o_begin + n_out; ++o) {
            const float yref = yrbuf[o * BM + r];
            Soft st{-INFINITY, 0.f, 0.f, 0.f};
            for (int j = 0; j < ntiles; ++j, ++g) {
                const int buf = (int)(g & 1), c = (int)(g & 3);
                if (!aborted && !mbar_wait_bounded(&acc_full[buf], (uint32_t)((g >> 1) & 1), abort_flag))
                    aborted = true;
                aborted = __any_sync(0xffffffffu, aborted);   // the TMEM loads below are warp-collective
                tc_fence_after();
                if (!aborted && !mbar_wait_bounded(&const_full[c], (uint32_t)((g >> 2) & 1), abort_flag))
                    aborted = true;
                aborted = __any_sync(0xffffffffu, aborted);
                const float *cy = reinterpret_cast<const float *>(smem + OFF_CONST + c * TC_CONST_BYTES) + h * HALF;
                const float *cv = cy + TNF;
                const uint32_t base = tbase + lane_off + buf * 256 + h * HALF;
#pragma unroll
                for (int ch = 0; ch < HALF / 16; ++ch) {
                    float sv[16], yv[16];
                    if (!aborted) tmem_ld16x2_wait(base + 16 * ch, base + 128 + 16 * ch, sv, yv);
                    if (ch == HALF / 16 - 1) {
                        // every column of this half read: hand the buffer back
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&acc_empty[buf]);
                    }
                    if (!aborted) {
                        const float2 *cy2 = reinterpret_cast<const float2 *>(cy + 16 * ch);
                        const float2 *cv2 = reinterpret_cast<const float2 *>(cv + 16 * ch);
                        soft_chunk(st, sv, yv, cy2, cv2, yref);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&const_empty[c]);
            }
            // merge the two column halves of this output
            float *pp = part + (o & 1) * NSUM * BM;
            if (!owner) {
                pp[0 * BM + r] = st.m;
                pp[1 * BM + r] = st.s0;
                pp[2 * BM + r] = st.s1;
                pp[3 * BM + r] = st.s2;
            }
            named_bar_sync(1, NE);
            if (owner) {
                const Soft other{pp[0 * BM + r], pp[1 * BM + r], pp[2 * BM + r], pp[3 * BM + r]};
                merge_into(st, other);
                // mean y_ref + E[e]; variance E[e^2 + sigma^2] - E[e]^2
                const float inv = 1.0f / st.s0;
                const float me = st.s1 * inv;
                const float yo = yref + me, vo = fmaxf(fmaf(-me, me, st.s2 * inv), 0.0f);
                // the standard deviation of the sampled step, here rather than in the serial step
                const float so = sqrtf(vo);
                ybuf[o * BM + r] = yo;
                vbuf[o * BM + r] = vo;
                sdbuf[o * BM + r] = so;
                if (!PREDICT && ncl > 1 && !aborted)   // send now, behind the next output's tiles
                    for (uint32_t pr = 0; pr < ncl; ++pr) {
                        if (pr == rank) continue;
                        st_cluster_f32(mapa_shared(ybuf, pr) + (uint32_t)((o * BM + r) * 4), yo);
                        st_cluster_f32(mapa_shared(vbuf, pr) + (uint32_t)((o * BM + r) * 4), vo);
                        st_cluster_f32(mapa_shared(sdbuf, pr) + (uint32_t)((o * BM + r) * 4), so);
                    }
            }
        }

        // ------------------------------------------ exchange (split form only)
        if (!PREDICT && ncl > 1 && owner) {
            // every output's values were sent after its merge; the arrivals
            // (release) publish them, then this CTA waits for the others'
            if (!aborted)
                for (uint32_t pr = 0; pr < ncl; ++pr)
                    if (pr != rank) mbar_arrive_remote(mapa_shared(S.xfull, pr));
            if (!aborted && !mbar_wait_cluster_bounded(S.xfull, (uint32_t)(t & 1), abort_flag)) aborted = true;
        }

        // ---------------------------------------------------------- dynamics
        if (owner) {
            float y[NY], var[NY], zext[17];
#pragma unroll
            for (int o = 0; o < NY; ++o) {
                y[o] = ybuf[o * BM + r];
                var[o] = vbuf[o * BM + r];
            }
            if (!PREDICT && ncl > 1 && !aborted)
                for (uint32_t pr = 0; pr < ncl; ++pr)
                    if (pr != rank) mbar_arrive_remote(mapa_shared(S.xfree, pr));
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
                // the Euler step first: the next step's features (and with them
                // the tensor core) wait for it, the running cost does not
                float n[NY];
                named_bar_sync(4, NE);   // the other half's normals of this step are in nbuf
                if (a.model_noise) {
#pragma unroll
                    for (int o = 0; o < NY; ++o) n[o] = nbuf[o * BM + r];
                } else {
#pragma unroll
                    for (int o = 0; o < NY; ++o) n[o] = 0.0f;
                }
#pragma unroll
                for (int c = 0; c < NX; ++c) {
                    const float xdot = fmaf(sdbuf[c * BM + r], n[c], y[c]);
                    zext[c] = fmaf(a.dt, xdot, xbuf[c * BM + r]);
                }
                if (t + 1 < a.T) {
#pragma unroll
                    for (int c = 0; c < NU; ++c) zext[NX + c] = nbuf[(NY + c) * BM + r];
                } else {
#pragma unroll
                    for (int c = 0; c < NU; ++c) zext[NX + c] = 0.0f;
                }
            }
            zext[16] = 1.0f;
            if (PREDICT) {
                if (t + 1 < nsteps) build_features(smem, r, zext);
            } else {
                if (t + 1 < nsteps) {
                    // publish z, build this half of the feature rows, release them to the issuer
#pragma unroll
                    for (int c = 0; c < NZ; ++c) zbuf[c * BM + r] = zext[c];
                    named_bar_arrive(5, NE);
                    build_features<0, KF / 16>(smem, r, zext);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(phi_ready);
                }
                // off the tensor core's path: the running cost at (x_t, z_t) from the state still
                // in xbuf, then the new state, this step's means as the next reference, the costs
                float x[NX];
#pragma unroll
                for (int c = 0; c < NX; ++c) x[c] = xbuf[c * BM + r];
                qbuf[r] = running_cost(a.cost, obs_s, x, var);
#pragma unroll
                for (int c = 0; c < NX; ++c) {
                    xbuf[c * BM + r] = zext[c];
                    yrbuf[c * BM + r] = y[c];
                }
                named_bar_sync(2, BM);
                if (writer) {
                    float qs = 0.0f;
                    for (int i = 0; i < M; ++i) qs += qbuf[r + i];
                    a.cost_tk[(size_t)t * a.K + k] = qs / (float)M;
                }
                if (t + 1 >= a.T) {
                    named_bar_sync(2, BM);
#pragma unroll
                    for (int c = 0; c < NX; ++c) x[c] = zext[c];
                    qbuf[r] = terminal_cost(a.cost, x);
                    named_bar_sync(2, BM);
                    if (writer) {
                        float ps = 0.0f;
                        for (int i = 0; i < M; ++i) ps += qbuf[r + i];
                        a.phi[k] = ps / (float)M;
                    }
                }
            }
        } else if (!PREDICT && t + 1 < nsteps) {
            named_bar_sync(5, NE);
            float zext[17];
#pragma unroll
            for (int c = 0; c < NZ; ++c) zext[c] = zbuf[c * BM + r];
            zext[16] = 1.0f;
            build_features<KF / 16, KF / 8>(smem, r, zext);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(phi_ready);
        }
        const bool any_abort = bar_sync_or(3, NE, aborted || *abort_flag != 0);
        if (any_abort) break;
        if (PREDICT && t + 1 < nsteps) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(phi_ready);
        }
    }
}

__device__ __forceinline__ void tc_drain(const TcArgs &a, const TcSmem &S, const TcProducer &P, const TcIssuer &I,
                                         bool issuer_ok)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) {
        // keep the CTA alive until every copy issued has landed: the last
        // phase of each group barrier, and of the last constant slots
        for (int x = 0; x < NGRP; ++x)
            if (P.n[x] > 0 && !mbar_wait_drain(&S.full[x], (uint32_t)((P.n[x] - 1) & 1)))
                atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
        for (long long g = (P.g > NCONST ? P.g - NCONST : 0); g < P.g; ++g)
            if (!mbar_wait_drain(&S.const_full[g & 3], (uint32_t)((g >> 2) & 1))) atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
    }
    if (warp == 1 && lane == 0) {
        // every MMA issued must complete before the tensor memory is freed:
        // normally the last tile's accumulator commit covers them all, after a
        // timeout the issuer's commit on the drain barrier does
        if (issuer_ok && I.g > 0 &&
            !mbar_wait_drain(&S.acc_full[(I.g - 1) & 1], (uint32_t)(((I.g - 1) >> 1) & 1)))
            atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
        if (I.drained && !mbar_wait_drain(S.drain, 0u)) atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
    }
}

__device__ __forceinline__ void tc_flag_abort(const TcArgs &a, const TcSmem &S, int code)
{
    if (!*S.abort_flag) atomicOr(a.err, code);
    *S.abort_flag = 1;
}

// One CTA's whole life for the 128-slot block at slot_base: set-up, the
// three roles, drain, tensor-memory release.  With NSPLIT > 1 the CTA is one
// of the NSPLIT CTAs of a cluster that share the block and split its outputs.
template <bool PREDICT, int NSPLIT, int QP>
__device__ __forceinline__ void tc_cta(const TcArgs &a, long long slot_base, unsigned char *smem)
{
    static_assert(NSPLIT == 1 || !PREDICT, "prediction mode is not split");
    const TcSmem S = tc_smem(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t ncl = NSPLIT;
    const uint32_t rank = NSPLIT > 1 ? cluster_rank() : 0u;
    constexpr int n_out = NY / NSPLIT;
    const int o_begin = (int)rank * n_out;
    tc_setup(S, ncl);
    for (int i = tid; i < a.cost.n_obs; i += NTHREADS) S.obs_s[i] = a.cost.obs[i];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (ncl > 1) cluster_sync_all();   // every CTA's barriers exist before any remote arrival
    const uint32_t tbase = *S.tslot;
    TcProducer P;
    TcIssuer I;
    bool issuer_ok = true;
    if (warp == 0) {
        const bool pok = tc_producer_item<PREDICT>(a, S, P, o_begin, n_out);
        if (!pok && lane == 0) tc_flag_abort(a, S, DEVERR_TIMEOUT_EMPTY);
        __syncwarp();
    } else if (warp == 1) {
        issuer_ok = tc_issuer_item<PREDICT, QP>(a, S, tbase, I, n_out);
        if (!issuer_ok && lane == 0) tc_flag_abort(a, S, DEVERR_TIMEOUT_FULL);
        __syncwarp();
    } else {
        long long g = 0;
        bool aborted = false;
        tc_epilogue_item<PREDICT, NSPLIT>(a, S, tbase, slot_base, g, aborted, rank);
        if (aborted) tc_flag_abort(a, S, DEVERR_TIMEOUT_FULL);
    }
    tc_drain(a, S, P, I, issuer_ok);
    // all roles done: free the tensor memory
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, TMEM_COLS);
    }
    if (ncl > 1) cluster_sync_all();   // no CTA leaves while another may still write into it
}

// Single-controller kernel.  NSPLIT = 1: one CTA per 128-slot block.
// NSPLIT = 2, 3, 4 (rollouts only): launched in clusters of NSPLIT CTAs that
// share one slot block and split its 12 outputs (see tc_epilogue_item).
template <bool PREDICT, int NSPLIT, int QP>
__global__ void __launch_bounds__(NTHREADS, 1) rollout_tc_kernel(const __grid_constant__ TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_cta<PREDICT, NSPLIT, QP>(a, (long long)(blockIdx.x / NSPLIT) * BM, smem);
}

// Group form: one (controller, 128-slot block) item per CTA (NSPLIT = 1) or
// per cluster of NSPLIT CTAs, all items in one wave; the arguments come from
// the device table.  Used when a batch's items alone would leave SMs idle.
template <int NSPLIT, int QP>
__global__ void __launch_bounds__(NTHREADS, 1) rollout_tc_group_kernel(const __grid_constant__ TcBatchArgs b)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // the item's arguments are read from the device table where they are used
    // (a shared-memory copy kept more values live and spilled)
    const int2 it = b.items[blockIdx.x / NSPLIT];
    tc_cta<false, NSPLIT, QP>(b.args[it.x], (long long)it.y * BM, smem);
}

// Persistent batched form (see rollout_fp32_batch_kernel): CTAs claim
// (controller, 128-slot block) items; every ring position and the TMEM
// allocation carry over between items.
template <int QP>
__global__ void __launch_bounds__(NTHREADS, 1) rollout_tc_batch_kernel(const __grid_constant__ TcBatchArgs b)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcArgs s_args;
    __shared__ int s_item;
    const TcSmem S = tc_smem(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    tc_setup(S, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *S.tslot;
    TcProducer P;
    TcIssuer I;
    bool issuer_ok = true;
    long long g = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= b.n_items || *S.abort_flag) break;
        const int2 it = b.items[item];
        if (tid == 0) s_args = b.args[it.x];
        __syncthreads();
        const TcArgs &a = s_args;
        for (int i = tid; i < a.cost.n_obs; i += NTHREADS) S.obs_s[i] = a.cost.obs[i];
        __syncthreads();
        if (warp == 0) {
            const bool pok = tc_producer_item<false>(a, S, P, 0, NY);
            if (!pok && lane == 0) tc_flag_abort(a, S, DEVERR_TIMEOUT_EMPTY);
            __syncwarp();
        } else if (warp == 1) {
            if (issuer_ok) {
                issuer_ok = tc_issuer_item<false, QP>(a, S, tbase, I, NY);
                if (!issuer_ok && lane == 0) tc_flag_abort(a, S, DEVERR_TIMEOUT_FULL);
            }
            __syncwarp();
        } else {
            tc_epilogue_item<false, 1>(a, S, tbase, (long long)it.y * BM, g, aborted, 0);
            if (aborted) tc_flag_abort(a, S, DEVERR_TIMEOUT_FULL);
        }
        __syncthreads();
    }
    tc_drain(b.args[0], S, P, I, issuer_ok);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, TMEM_COLS);
    }
}

char g_tc_diag[256] = "";

void split_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, long long blocks, int split, cudaStream_t s)
{
    cfg.gridDim = dim3((unsigned)(blocks * split));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)split;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

// Sets the shared-memory attribute of one kernel instantiation once and
// checks that it can be launched with NTHREADS threads.
template <bool PREDICT, int NSPLIT, int QP = 3>
cudaError_t prepare_tc()
{
    static std::atomic<uint64_t> done;
    cudaError_t e = set_smem_once(done, rollout_tc_kernel<PREDICT, NSPLIT, QP>, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    static std::atomic<bool> checked{false};
    if (checked.load(std::memory_order_acquire)) return cudaSuccess;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, rollout_tc_kernel<PREDICT, NSPLIT, QP>);
    if (e != cudaSuccess) return e;
    snprintf(g_tc_diag, sizeof g_tc_diag,
             "split %d: regs %d, maxThreadsPerBlock %d, dynamic smem %d (max %d), static smem %zu, local %zu", NSPLIT,
             fa.numRegs, fa.maxThreadsPerBlock, SMEM_BYTES, fa.maxDynamicSharedSizeBytes, fa.sharedSizeBytes,
             fa.localSizeBytes);
    if (fa.maxThreadsPerBlock < NTHREADS) return cudaErrorLaunchOutOfResources;
    checked.store(true, std::memory_order_release);
    return cudaSuccess;
}

// CTAs of the single-controller kernel with clusters of NSPLIT that can be
// resident at once (0 if the cluster shape cannot be launched).  Both product
// counts use the same threads and shared memory, so the three-product
// instantiation stands for both.
template <int NSPLIT>
long long resident_ctas()
{
    if (prepare_tc<false, NSPLIT>() != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (NSPLIT == 1) return sms;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    split_config(cfg, at, sms, NSPLIT, nullptr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, rollout_tc_kernel<false, NSPLIT, 3>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (long long)clusters * NSPLIT;
}

// Relative time of `items` 128-slot items whose outputs are split over s CTAs
// when `resident` CTAs run at once: whole waves of CTAs that each carry 1/s of
// an item's work, times the split's own cost (a CTA repeats the dynamics step
// and exchanges its outputs).  The overheads are the ones measured on this
// kernel (12 outputs, L = 2048): +3 % for 2 CTAs, +13 % for 3, +19 % for 4.
double split_cost(long long items, int s, long long resident)
{
    static const double overhead[5] = {0.0, 0.0, 0.03, 0.13, 0.19};
    if (resident <= 0) return 1e300;
    const long long waves = (items * s + resident - 1) / resident;
    return (double)waves / s * (1.0 + overhead[s]);
}

// Output split of the single-controller rollout launch: the split of least
// split_cost (ties to the smaller split).  Small K spreads each block over a
// cluster so that the SMs fill up; a few waves of blocks use pairs to shorten
// the last, partly empty wave.  PI2RH_TC_SPLIT = 1..4 forces a value (the
// results are bitwise the same for every split).
// Resident CTAs of the single-controller kernel for splits 1-4 on the current
// device, from the occupancy API on the first launch there and cached (the
// queries cost tens of microseconds of host time in front of every launch
// otherwise, with the GPU idle).
std::array<long long, 5> resident_per_split()
{
    static std::mutex m;
    static std::map<int, std::array<long long, 5>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(m);
    auto it = cache.find(dev);
    if (it == cache.end())
        it = cache.emplace(dev, std::array<long long, 5>{0, resident_ctas<1>(), resident_ctas<2>(), resident_ctas<3>(),
                                                         resident_ctas<4>()}).first;
    return it->second;
}

int choose_split(long long blocks)
{
    if (const char *e = getenv("PI2RH_TC_SPLIT")) {
        const int v = atoi(e);
        if (v >= 1 && v <= 4) return v;
    }
    const std::array<long long, 5> res = resident_per_split();
    int best = 1;
    for (int sp = 2; sp <= 4; ++sp)
        if (split_cost(blocks, sp, res[sp]) < split_cost(blocks, best, res[best])) best = sp;
    return best;
}

template <int NSPLIT, int QP>
cudaError_t launch_split(const TcArgs &a, long long blocks, cudaStream_t s)
{
    cudaError_t e = prepare_tc<false, NSPLIT, QP>();
    if (e != cudaSuccess) return e;
    if (NSPLIT == 1) {
        rollout_tc_kernel<false, NSPLIT, QP><<<(unsigned)blocks, NTHREADS, SMEM_BYTES, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    split_config(cfg, at, blocks, NSPLIT, s);
    return cudaLaunchKernelEx(&cfg, rollout_tc_kernel<false, NSPLIT, QP>, a);
}

template <int NSPLIT, int QP = 3>
cudaError_t prepare_group()
{
    static std::atomic<uint64_t> done;
    return set_smem_once(done, rollout_tc_group_kernel<NSPLIT, QP>, SMEM_BYTES);
}

// Clusters of NSPLIT CTAs of the group kernel that can be resident at once on
// the current device (0 if the shape cannot be launched), queried once per
// device and cached.
template <int NSPLIT>
long long group_resident_clusters()
{
    static std::mutex m;
    static std::map<int, long long> cache;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(m);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    long long n = 0;
    if (prepare_group<NSPLIT>() == cudaSuccess) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        split_config(cfg, at, sms, NSPLIT, nullptr);
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, rollout_tc_group_kernel<NSPLIT, 3>, &cfg) == cudaSuccess)
            n = clusters;
        else
            cudaGetLastError();   // the shape cannot be launched: not an error of the caller's
    } else {
        cudaGetLastError();
    }
    cache.emplace(dev, n);
    return n;
}

template <int NSPLIT>
bool group_clusters_resident(long long items)
{
    return group_resident_clusters<NSPLIT>() >= items;
}

template <int NSPLIT, int QP>
cudaError_t launch_group(const TcBatchArgs &b, cudaStream_t s)
{
    cudaError_t e = prepare_group<NSPLIT, QP>();
    if (e != cudaSuccess) return e;
    if (NSPLIT == 1) {
        rollout_tc_group_kernel<1, QP><<<(unsigned)b.n_items, NTHREADS, SMEM_BYTES, s>>>(b);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    split_config(cfg, at, b.n_items, NSPLIT, s);
    return cudaLaunchKernelEx(&cfg, rollout_tc_group_kernel<NSPLIT, QP>, b);
}

cudaError_t check_tc_args(const TcArgs &a)
{
    return a.cost.n_obs > MAX_OBS || a.tiles_per_out <= 0 || (a.qprod != 2 && a.qprod != 3) ? cudaErrorInvalidValue
                                                                                             : cudaSuccess;
}

template <int QP>
cudaError_t launch_rollout_tc_qp(const TcArgs &a, long long blocks, cudaStream_t s)
{
    switch (choose_split(blocks)) {
    case 4: return launch_split<4, QP>(a, blocks, s);
    case 3: return launch_split<3, QP>(a, blocks, s);
    case 2: return launch_split<2, QP>(a, blocks, s);
    default: return launch_split<1, QP>(a, blocks, s);
    }
}

template <int QP>
cudaError_t launch_group_qp(const TcBatchArgs &b, int split, cudaStream_t s)
{
    switch (split) {
    case 4: return launch_group<4, QP>(b, s);
    case 3: return launch_group<3, QP>(b, s);
    case 2: return launch_group<2, QP>(b, s);
    default: return launch_group<1, QP>(b, s);
    }
}

}  // namespace

const char *tc_launch_diag() { return g_tc_diag; }

cudaError_t launch_rollout_tc(const TcArgs &a, cudaStream_t s)
{
    if (a.M < 1 || a.M > BM || (a.M & (a.M - 1)) != 0) return cudaErrorInvalidValue;
    cudaError_t e = check_tc_args(a);
    if (e != cudaSuccess) return e;
    const long long blocks = ((long long)a.K * a.M + BM - 1) / BM;
    if (blocks <= 0 || blocks > 0x7fffffffLL / 4) return cudaErrorInvalidValue;
    return a.qprod == 2 ? launch_rollout_tc_qp<2>(a, blocks, s) : launch_rollout_tc_qp<3>(a, blocks, s);
}

cudaError_t launch_predict_tc(const TcArgs &a, cudaStream_t s)
{
    cudaError_t e = check_tc_args(a);
    if (e != cudaSuccess) return e;
    const long long blocks = ((long long)a.n_pred + BM - 1) / BM;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (a.qprod == 2) {
        if ((e = prepare_tc<true, 1, 2>()) != cudaSuccess) return e;
        rollout_tc_kernel<true, 1, 2><<<(unsigned)blocks, NTHREADS, SMEM_BYTES, s>>>(a);
    } else {
        if ((e = prepare_tc<true, 1, 3>()) != cudaSuccess) return e;
        rollout_tc_kernel<true, 1, 3><<<(unsigned)blocks, NTHREADS, SMEM_BYTES, s>>>(a);
    }
    return cudaGetLastError();
}

int tc_group_split(int n_items)
{
    if (n_items <= 0) return 1;
    if (const char *e = getenv("PI2RH_TC_SPLIT")) {
        const int v = atoi(e);
        if (v >= 1 && v <= 4) return v;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((long long)n_items * 4 <= sms && group_clusters_resident<4>(n_items)) return 4;
    if ((long long)n_items * 3 <= sms && group_clusters_resident<3>(n_items)) return 3;
    if ((long long)n_items * 2 <= sms && group_clusters_resident<2>(n_items)) return 2;
    return 1;
}

cudaError_t launch_rollout_tc_group(const TcBatchArgs &b, int split, cudaStream_t s)
{
    if (b.n_items <= 0 || (b.qprod != 2 && b.qprod != 3)) return cudaErrorInvalidValue;
    return b.qprod == 2 ? launch_group_qp<2>(b, split, s) : launch_group_qp<3>(b, split, s);
}

std::atomic<uint64_t> g_tc_batch_attr[2];

cudaError_t launch_rollout_tc_batch(const TcBatchArgs &b, int grid, cudaStream_t s)
{
    if (grid <= 0 || (b.qprod != 2 && b.qprod != 3)) return cudaErrorInvalidValue;
    cudaError_t e;
    if (b.qprod == 2) {
        if ((e = set_smem_once(g_tc_batch_attr[0], rollout_tc_batch_kernel<2>, SMEM_BYTES)) != cudaSuccess) return e;
        rollout_tc_batch_kernel<2><<<grid, NTHREADS, SMEM_BYTES, s>>>(b);
    } else {
        if ((e = set_smem_once(g_tc_batch_attr[1], rollout_tc_batch_kernel<3>, SMEM_BYTES)) != cudaSuccess) return e;
        rollout_tc_batch_kernel<3><<<grid, NTHREADS, SMEM_BYTES, s>>>(b);
    }
    return cudaGetLastError();
}

}  // namespace pi2rh

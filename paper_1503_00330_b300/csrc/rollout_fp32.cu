// rollout_fp32.cu -- fused FP32 rollout kernel of one PI^2-RH update.
//
// One CTA owns RF_SLOTS = 64 rollout slots (rollout k, sub-rollout m) for all
// T steps.  Per step and per output o it evaluates every receptive field of
// the LWPR model (Sec. 2, Eq. 1) for its 64 slots:
//     d = z - c_j,  s_j = -(1/2) log2(e) d^T D_j d,  e_j = b_j + beta_j . d - y_ref
// and folds them into an online (max-shifted) base-2 softmax that carries
//     sum w, sum w e, sum w e^2, sum w sigma_j^2
// so that the mean y = y_ref + S1/S0 and the variance
//     sum_j w_j ((y - y_j)^2 + sigma_j^2) = S2/S0 - (S1/S0)^2 + S3/S0
// come out of one pass (y_ref is the slot's previous mean of that output, so
// the spread term does not cancel).  Then the slot's running cost, the sampled
// Euler step x + dt (y + sigma n) (Sec. 3.2) and the next control perturbation
// are computed, with Philox noise generated in the kernel.
//
// Data movement: the model is far larger than shared memory (12 L records of
// 1376 bytes per field pair), so it is streamed through a ring of NSTAGE
// shared-memory stages (two of 64 records, 88 KB each) by one producer warp
// issuing 1-D bulk asynchronous copies (TMA) that complete on mbarriers; each
// of the eight consumer warps takes 8 field-pair records per stage, records
// j * 8 + warp, so a warp still walks pairs warp, warp + 8, ... in order and
// pays one wait and one arrival per 8 records.  All 32 lanes of a consumer warp read the same
// record (shared-memory broadcast), and each lane evaluates it for two slots,
// so every parameter load feeds four field-slot evaluations on the packed
// FP32x2 FMA datapath.  Every wait is bounded; on expiry the kernel records a
// flag in the device error word, drains its copies and returns.
//
// Launches (launch_rollout_fp32): one CTA per 64-slot block
// (rollout_fp32_kernel) for every whole wave of blocks; the blocks of a last,
// partial wave (all of them when there are fewer blocks than SMs) can instead
// go to rollout_fp32_split_kernel, which deals their (block, output) units out
// to one co-resident CTA per SM with the same per-output arithmetic (see the
// comment above that kernel).  The batched and serving paths use the
// persistent and one-item-per-CTA forms at the end of the file.
#include "pi2rh.h"
#include "pi2rh_kernels.h"

namespace pi2rh {

namespace {

constexpr int NSTAGE = 2;
constexpr int CW = RF_CONSUMER_WARPS;          // consumer warps
constexpr int NTHREADS = (CW + 1) * 32;        // + one producer warp
constexpr int NCONS = CW * 32;                 // consumer threads
constexpr int SLOTS = RF_SLOTS;                // 2 per consumer lane
constexpr int STAGE_BYTES = RF_PAIRS_PER_STAGE * REC_BYTES;
constexpr int MAX_OBS = 256;

// Shared-memory layout (bytes from the dynamic base).
constexpr int OFF_STAGE = 0;
constexpr int OFF_PART = OFF_STAGE + NSTAGE * STAGE_BYTES;          // [2][CW][5][SLOTS] f32
constexpr int PART_BUF = CW * 5 * SLOTS;                            // floats per buffer
constexpr int OFF_Z = OFF_PART + 2 * PART_BUF * 4;                  // [NZ][SLOTS]
constexpr int OFF_X = OFF_Z + NZ * SLOTS * 4;                       // [NX][SLOTS]
constexpr int OFF_Y = OFF_X + NX * SLOTS * 4;                       // [NY][SLOTS]
constexpr int OFF_V = OFF_Y + NY * SLOTS * 4;                       // [NY][SLOTS]
constexpr int OFF_YREF = OFF_V + NY * SLOTS * 4;                    // [NY][SLOTS]
constexpr int OFF_Q = OFF_YREF + NY * SLOTS * 4;                    // [SLOTS]
constexpr int OFF_OBS = OFF_Q + SLOTS * 4;                          // [MAX_OBS] float2
constexpr int OFF_BAR = OFF_OBS + MAX_OBS * 8;                      // full[NSTAGE], empty[NSTAGE]
constexpr int OFF_ABORT = OFF_BAR + 2 * NSTAGE * 8;
constexpr int SMEM_BYTES = OFF_ABORT + 16;
static_assert(OFF_PART % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

struct Soft {
    float m, s0, s1, s2, s3;
};

__device__ __forceinline__ void soft_init(Soft &st)
{
    st.m = -INFINITY;
    st.s0 = st.s1 = st.s2 = st.s3 = 0.0f;
}

// Adds two fields (packed exponent s, centered prediction e, variance v).
__device__ __forceinline__ void soft_add2(Soft &st, float2 s, float2 e, float2 v)
{
    float mn = fmaxf(st.m, fmaxf(s.x, s.y));
    float sc = ex2(st.m - mn);
    float wa = ex2(s.x - mn), wb = ex2(s.y - mn);
    float wea = wa * e.x, web = wb * e.y;
    st.s0 = fmaf(st.s0, sc, wa + wb);
    st.s1 = fmaf(st.s1, sc, wea + web);
    st.s2 = fmaf(st.s2, sc, fmaf(wea, e.x, web * e.y));
    st.s3 = fmaf(st.s3, sc, fmaf(wa, v.x, wb * v.y));
    st.m = mn;
}

__device__ __forceinline__ float2 f2(float4 v, int hi)
{
    return hi ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
}

// Row I of the symmetric quadratic form: s += d_I (sum_{j>=I} A_Ij d_j), for
// both slots; rows are expanded at compile time so every index is constant.
// Even rows add into s, odd rows into s2 (summed once at the end), which
// halves the dependency chain across the 16 rows.
template <int I>
__device__ __forceinline__ void quad_rows(const float4 *__restrict__ r4, const float2 (&dA)[NZ],
                                          const float2 (&dB)[NZ], float2 &sA, float2 &sB, float2 &sA2, float2 &sB2)
{
    if constexpr (I < NZ) {
        constexpr int base = REC_A + tri_index(I, I);   // first entry of row I
        const float2 a0 = f2(r4[base >> 1], base & 1);
        float2 tA = __fmul2_rn(a0, dA[I]);
        float2 tB = __fmul2_rn(a0, dB[I]);
#pragma unroll
        for (int j = I + 1; j < NZ; ++j) {
            const int e = base + (j - I);
            const float2 aij = f2(r4[e >> 1], e & 1);
            tA = __ffma2_rn(aij, dA[j], tA);
            tB = __ffma2_rn(aij, dB[j], tB);
        }
        if (I & 1) {
            sA2 = __ffma2_rn(dA[I], tA, sA2);
            sB2 = __ffma2_rn(dB[I], tB, sB2);
        } else {
            sA = __ffma2_rn(dA[I], tA, sA);
            sB = __ffma2_rn(dB[I], tB, sB);
        }
        quad_rows<I + 1>(r4, dA, dB, sA, sB, sA2, sB2);
    }
}

// Evaluates one field-pair record for two slots A and B.
__device__ __forceinline__ void process_pair(const float4 *__restrict__ r4, const float2 (&zA)[NZ],
                                             const float2 (&zB)[NZ], float2 yrA, float2 yrB,
                                             Soft &stA, Soft &stB)
{
    float2 dA[NZ], dB[NZ];
#pragma unroll
    for (int a = 0; a < NZ; a += 2) {
        float4 nc = r4[(REC_NEGC + a) >> 1];
        dA[a] = __fadd2_rn(zA[a], f2(nc, 0));
        dA[a + 1] = __fadd2_rn(zA[a + 1], f2(nc, 1));
        dB[a] = __fadd2_rn(zB[a], f2(nc, 0));
        dB[a + 1] = __fadd2_rn(zB[a + 1], f2(nc, 1));
    }
    float4 tail = r4[REC_B >> 1];        // {b.x, b.y, var.x, var.y}
    float4 tail2 = r4[REC_BIAS >> 1];    // {bias.x, bias.y, 0, 0}
    float2 sA = f2(tail2, 0), sB = sA;
    float2 sA2 = make_float2(0.f, 0.f), sB2 = sA2;
    quad_rows<0>(r4, dA, dB, sA, sB, sA2, sB2);
    sA = __fadd2_rn(sA, sA2);
    sB = __fadd2_rn(sB, sB2);
    float2 b = f2(tail, 0);
    float2 eA = __fadd2_rn(b, yrA), eB = __fadd2_rn(b, yrB);   // yr holds -y_ref
#pragma unroll
    for (int a = 0; a < NZ; a += 2) {
        float4 be = r4[(REC_BETA + a) >> 1];
        eA = __ffma2_rn(f2(be, 0), dA[a], eA);
        eA = __ffma2_rn(f2(be, 1), dA[a + 1], eA);
        eB = __ffma2_rn(f2(be, 0), dB[a], eB);
        eB = __ffma2_rn(f2(be, 1), dB[a + 1], eB);
    }
    float2 v = f2(tail, 1);
    soft_add2(stA, sA, eA, v);
    soft_add2(stB, sB, eB, v);
}

// Merges the CW per-warp partials of one output for one slot.
__device__ __forceinline__ void merge_partials(const float *pb, int slot, float yref, float &y,
                                               float &var)
{
    float M = -INFINITY;
#pragma unroll
    for (int w = 0; w < CW; ++w) M = fmaxf(M, pb[(w * 5 + 0) * SLOTS + slot]);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int w = 0; w < CW; ++w) {
        float sc = ex2(pb[(w * 5 + 0) * SLOTS + slot] - M);
        s0 = fmaf(pb[(w * 5 + 1) * SLOTS + slot], sc, s0);
        s1 = fmaf(pb[(w * 5 + 2) * SLOTS + slot], sc, s1);
        s2 = fmaf(pb[(w * 5 + 3) * SLOTS + slot], sc, s2);
        s3 = fmaf(pb[(w * 5 + 4) * SLOTS + slot], sc, s3);
    }
    float inv = 1.0f / s0;
    float mean_e = s1 * inv;
    y = yref + mean_e;
    var = fmaxf(fmaf(-mean_e, mean_e, s2 * inv), 0.0f) + s3 * inv;
}

// Shared-memory views of one CTA.
struct Fp32Smem {
    unsigned char *stage_base;
    float *part, *zbuf, *xbuf, *ybuf, *vbuf, *yrbuf, *qbuf;
    float2 *obs_s;
    uint64_t *full, *empty;
    volatile int *abort_flag;
};

__device__ __forceinline__ Fp32Smem fp32_smem(unsigned char *smem)
{
    Fp32Smem S;
    S.stage_base = smem + OFF_STAGE;
    S.part = reinterpret_cast<float *>(smem + OFF_PART);
    S.zbuf = reinterpret_cast<float *>(smem + OFF_Z);
    S.xbuf = reinterpret_cast<float *>(smem + OFF_X);
    S.ybuf = reinterpret_cast<float *>(smem + OFF_Y);
    S.vbuf = reinterpret_cast<float *>(smem + OFF_V);
    S.yrbuf = reinterpret_cast<float *>(smem + OFF_YREF);
    S.qbuf = reinterpret_cast<float *>(smem + OFF_Q);
    S.obs_s = reinterpret_cast<float2 *>(smem + OFF_OBS);
    S.full = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
    S.empty = S.full + NSTAGE;
    S.abort_flag = reinterpret_cast<volatile int *>(smem + OFF_ABORT);
    return S;
}

__device__ __forceinline__ void fp32_init_barriers(const Fp32Smem &S)
{
    for (int s = 0; s < NSTAGE; ++s) {
        mbar_init(&S.full[s], 1);
        mbar_init(&S.empty[s], CW);
    }
    *S.abort_flag = 0;
    fence_mbar_init();
}

// Producer (one lane): streams the field-pair records of one work item (T
// passes over its outputs) through the stage ring.  Per step it copies the
// outputs out_of(0), ..., out_of(n_out - 1), each in spo stages.  `g0` is the
// ring position at the start of the item; returns the position after it, or
// -1 after a timeout (abort flag set).
template <typename OutOf>
__device__ __forceinline__ long long fp32_produce(const RolloutArgs &a, const Fp32Smem &S, long long g0,
                                                  long long &issued, int n_out, OutOf out_of)
{
    unsigned char *stage_base = S.stage_base;
    uint64_t *full = S.full, *empty = S.empty;
    volatile int *abort_flag = S.abort_flag;
    const int P = a.P, spo = a.stages_per_out;
    const int G = n_out * spo;
    const long long total = g0 + (long long)G * a.T;
        for (long long g = g0; g < total; ++g) {
            const int slot = (int)(g % NSTAGE);
            if (g >= NSTAGE) {
                const uint32_t par = (uint32_t)(((g / NSTAGE) - 1) & 1);
                if (!mbar_wait_bounded(&empty[slot], par, abort_flag)) {
                    if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                    *abort_flag = 1;
                    return -1;
                }
            }
            const int gs = (int)((g - g0) % G);
            const int o = out_of(gs / spo), s = gs % spo;
            const int p0 = s * RF_PAIRS_PER_STAGE;
            const int np = min(RF_PAIRS_PER_STAGE, P - p0);
            const uint32_t bytes = (uint32_t)np * REC_BYTES;
            const float2 *src = a.rec + ((size_t)o * P + p0) * REC_LEN;
            mbar_arrive_expect_tx(&full[slot], bytes);
            bulk_g2s(stage_base + (size_t)slot * STAGE_BYTES, src, bytes, &full[slot]);
            issued = g + 1;
        }
    return total;
}

// All NY outputs in order (one 64-slot block per CTA).
__device__ long long fp32_producer(const RolloutArgs &a, const Fp32Smem &S, long long g0, long long &issued)
{
    return fp32_produce(a, S, g0, issued, NY, [](int i) { return i; });
}

// Initial state of one slot (stepper thread tid of its block): x = x0,
// z = [x0, u_nom[0] + eps_0], y_ref = 0; the writer stores eps_0 (the split
// kernel's copy of fp32_consumer's set-up).
__device__ __forceinline__ void fp32_init_slot(const RolloutArgs &a, const Fp32Smem &S, int tid, int k, bool writer)
{
    float *zbuf = S.zbuf, *xbuf = S.xbuf, *yrbuf = S.yrbuf;
    float4 n = box_muller4(noise_block(a.seed, (uint32_t)k, 0u, 0u, 0u));
    float eps[4] = {a.sqrt_sigma_u[0] * n.x, a.sqrt_sigma_u[1] * n.y,
                    a.sqrt_sigma_u[2] * n.z, a.sqrt_sigma_u[3] * n.w};
#pragma unroll
    for (int c = 0; c < NX; ++c) {
        float xc = a.x0[c];
        xbuf[c * SLOTS + tid] = xc;
        zbuf[c * SLOTS + tid] = xc;
    }
#pragma unroll
    for (int c = 0; c < NU; ++c) zbuf[(NX + c) * SLOTS + tid] = a.u_nom[c] + eps[c];
#pragma unroll
    for (int o = 0; o < NY; ++o) yrbuf[o * SLOTS + tid] = 0.0f;
    if (writer) a.eps_tk[k] = make_float4(eps[0], eps[1], eps[2], eps[3]);
}

// One output's pass over its field-pair records (spo stages of the ring from
// position g) for the warp's slots A = lane and B = lane + 32, whose inputs
// are zA, zB and whose negated reference means are ya, yb.  Writes the
// warp's softmax states into partial buffer `parity` (the buffer's address is
// formed after the record loop, so it takes no register during it).
__device__ __forceinline__ void fp32_output_pass(const RolloutArgs &a, const Fp32Smem &S, const float2 (&zA)[NZ],
                                                 const float2 (&zB)[NZ], float ya, float yb, int parity,
                                                 long long &g, bool &aborted, int P, int spo)
{
    unsigned char *stage_base = S.stage_base;
    uint64_t *full = S.full, *empty = S.empty;
    volatile int *abort_flag = S.abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slotA = lane, slotB = lane + 32;
    const float2 yrA = make_float2(ya, ya), yrB = make_float2(yb, yb);
    Soft stA, stB;
    soft_init(stA);
    soft_init(stB);
    for (int s = 0; s < spo; ++s, ++g) {
        const int slot = (int)(g % NSTAGE);
        if (!aborted && !mbar_wait_bounded(&full[slot], (uint32_t)((g / NSTAGE) & 1), abort_flag)) {
            if (lane == 0) {
                if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
                *abort_flag = 1;
            }
            aborted = true;
        }
#pragma unroll 2
        for (int j = 0; j < RF_PAIRS_PER_STAGE / CW; ++j) {
            const int pair = s * RF_PAIRS_PER_STAGE + j * CW + warp;
            if (!aborted && pair < P) {
                const float4 *r4 = reinterpret_cast<const float4 *>(
                    stage_base + (size_t)slot * STAGE_BYTES + (size_t)(j * CW + warp) * REC_BYTES);
                process_pair(r4, zA, zB, yrA, yrB, stA, stB);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    float *pb = S.part + parity * PART_BUF;
    pb[(warp * 5 + 0) * SLOTS + slotA] = stA.m;
    pb[(warp * 5 + 1) * SLOTS + slotA] = stA.s0;
    pb[(warp * 5 + 2) * SLOTS + slotA] = stA.s1;
    pb[(warp * 5 + 3) * SLOTS + slotA] = stA.s2;
    pb[(warp * 5 + 4) * SLOTS + slotA] = stA.s3;
    pb[(warp * 5 + 0) * SLOTS + slotB] = stB.m;
    pb[(warp * 5 + 1) * SLOTS + slotB] = stB.s0;
    pb[(warp * 5 + 2) * SLOTS + slotB] = stB.s1;
    pb[(warp * 5 + 3) * SLOTS + slotB] = stB.s2;
    pb[(warp * 5 + 4) * SLOTS + slotB] = stB.s3;
}

// The warp's slot inputs, duplicated into both halves of a float2 (the two
// fields of a record), from the [NZ][SLOTS] buffer zsrc.
__device__ __forceinline__ void fp32_load_z(const float *zsrc, float2 (&zA)[NZ], float2 (&zB)[NZ])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NZ; ++c) {
        float va = zsrc[c * SLOTS + lane], vb = zsrc[c * SLOTS + lane + 32];
        zA[c] = make_float2(va, va);
        zB[c] = make_float2(vb, vb);
    }
}

// End of step t for one slot (stepper thread tid; all 64 stepper threads
// call it together): with y and var of every output in ybuf / vbuf, the
// running cost at (x_t, z_t), the sampled Euler step (Sec. 3.2), the next
// control perturbation, and at the last step the terminal cost (the split
// kernel's copy of fp32_consumer's step; tests hold the two bitwise equal).
__device__ __forceinline__ void fp32_step_slot(const RolloutArgs &a, const Fp32Smem &S, int t, int tid, int k, int m,
                                               bool writer)
{
    float *zbuf = S.zbuf, *xbuf = S.xbuf, *ybuf = S.ybuf, *vbuf = S.vbuf, *yrbuf = S.yrbuf, *qbuf = S.qbuf;
    const int M = a.M;
    float y[NY], var[NY];
#pragma unroll
    for (int o = 0; o < NY; ++o) {
        y[o] = ybuf[o * SLOTS + tid];
        var[o] = vbuf[o * SLOTS + tid];
    }
    float x[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) x[c] = xbuf[c * SLOTS + tid];
    // running cost at (x_t, z_t), averaged over the sub-rollouts of k
    qbuf[tid] = running_cost(a.cost, S.obs_s, x, var);
    // sampled Euler step (Sec. 3.2)
    float n[NY];
    if (a.model_noise) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float4 nb = box_muller4(noise_block(a.seed, (uint32_t)k, (uint32_t)t, (uint32_t)(b + 1), (uint32_t)m));
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
        float xdot = fmaf(sqrtf(var[c]), n[c], y[c]);
        x[c] = fmaf(a.dt, xdot, x[c]);
        xbuf[c * SLOTS + tid] = x[c];
        zbuf[c * SLOTS + tid] = x[c];
        yrbuf[c * SLOTS + tid] = y[c];
    }
    named_bar_sync(2, SLOTS);
    if (writer) {
        float qs = 0.0f;
        for (int i = 0; i < M; ++i) qs += qbuf[tid + i];
        a.cost_tk[(size_t)t * a.K + k] = qs / (float)M;
    }
    if (t + 1 < a.T) {
        float4 nn = box_muller4(noise_block(a.seed, (uint32_t)k, (uint32_t)(t + 1), 0u, 0u));
        float eps[4] = {a.sqrt_sigma_u[0] * nn.x, a.sqrt_sigma_u[1] * nn.y,
                        a.sqrt_sigma_u[2] * nn.z, a.sqrt_sigma_u[3] * nn.w};
#pragma unroll
        for (int c = 0; c < NU; ++c) zbuf[(NX + c) * SLOTS + tid] = a.u_nom[(size_t)(t + 1) * NU + c] + eps[c];
        if (writer) a.eps_tk[(size_t)(t + 1) * a.K + k] = make_float4(eps[0], eps[1], eps[2], eps[3]);
    } else {
        named_bar_sync(2, SLOTS);           // qbuf reads done before reuse
        qbuf[tid] = terminal_cost(a.cost, x);
        named_bar_sync(2, SLOTS);
        if (writer) {
            float ps = 0.0f;
            for (int i = 0; i < M; ++i) ps += qbuf[tid + i];
            a.phi[k] = ps / (float)M;
        }
    }
}

// Consumers (8 warps): evaluate the LWPR model for the 64 slots of one work
// item starting at slot_base, step the dynamics and write the item's outputs.
// `g` is the ring position (advanced in step with the producer).  The split
// kernel runs the same arithmetic through fp32_init_slot, fp32_output_pass and
// fp32_step_slot; here it stays written out in one body, which the batch
// kernels (arguments in shared memory) run 3 % faster than the function form.
__device__ void fp32_consumer(const RolloutArgs &a, const Fp32Smem &S, long long slot_base, long long &g, bool &aborted)
{
    unsigned char *stage_base = S.stage_base;
    float *part = S.part, *zbuf = S.zbuf, *xbuf = S.xbuf, *ybuf = S.ybuf, *vbuf = S.vbuf, *yrbuf = S.yrbuf,
          *qbuf = S.qbuf;
    float2 *obs_s = S.obs_s;
    uint64_t *full = S.full, *empty = S.empty;
    volatile int *abort_flag = S.abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.P, spo = a.stages_per_out;
    const int nsteps = a.T;
    const int M = a.M;
    const int slotA = lane, slotB = lane + 32;

    // Step-thread state: thread tid < SLOTS owns slot tid.
    const bool stepper = tid < SLOTS;
    const long long gslot = slot_base + tid;
    const int k = (int)(gslot / M), m = (int)(gslot % M);
    const bool writer = stepper && k < a.K && m == 0;

    if (stepper) {
        {
            float4 n = box_muller4(noise_block(a.seed, (uint32_t)k, 0u, 0u, 0u));
            float eps[4] = {a.sqrt_sigma_u[0] * n.x, a.sqrt_sigma_u[1] * n.y,
                            a.sqrt_sigma_u[2] * n.z, a.sqrt_sigma_u[3] * n.w};
#pragma unroll
            for (int c = 0; c < NX; ++c) {
                float xc = a.x0[c];
                xbuf[c * SLOTS + tid] = xc;
                zbuf[c * SLOTS + tid] = xc;
            }
#pragma unroll
            for (int c = 0; c < NU; ++c) zbuf[(NX + c) * SLOTS + tid] = a.u_nom[c] + eps[c];
#pragma unroll
            for (int o = 0; o < NY; ++o) yrbuf[o * SLOTS + tid] = 0.0f;
            if (writer) a.eps_tk[k] = make_float4(eps[0], eps[1], eps[2], eps[3]);
        }
    }
    named_bar_sync(1, NCONS);

    for (int t = 0; t < nsteps; ++t) {
        float2 zA[NZ], zB[NZ];
#pragma unroll
        for (int c = 0; c < NZ; ++c) {
            float va = zbuf[c * SLOTS + slotA], vb = zbuf[c * SLOTS + slotB];
            zA[c] = make_float2(va, va);
            zB[c] = make_float2(vb, vb);
        }
        for (int o = 0; o < NY; ++o) {
            const float ya = -yrbuf[o * SLOTS + slotA], yb = -yrbuf[o * SLOTS + slotB];
            const float2 yrA = make_float2(ya, ya), yrB = make_float2(yb, yb);
            Soft stA, stB;
            soft_init(stA);
            soft_init(stB);
            for (int s = 0; s < spo; ++s, ++g) {
                const int slot = (int)(g % NSTAGE);
                if (!aborted &&
                    !mbar_wait_bounded(&full[slot], (uint32_t)((g / NSTAGE) & 1), abort_flag)) {
                    if (lane == 0) {
                        if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
                        *abort_flag = 1;
                    }
                    aborted = true;
                }
#pragma unroll 2
                for (int j = 0; j < RF_PAIRS_PER_STAGE / CW; ++j) {
                    const int pair = s * RF_PAIRS_PER_STAGE + j * CW + warp;
                    if (!aborted && pair < P) {
                        const float4 *r4 = reinterpret_cast<const float4 *>(
                            stage_base + (size_t)slot * STAGE_BYTES + (size_t)(j * CW + warp) * REC_BYTES);
                        process_pair(r4, zA, zB, yrA, yrB, stA, stB);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
            }
            float *pb = part + (o & 1) * PART_BUF;
            pb[(warp * 5 + 0) * SLOTS + slotA] = stA.m;
            pb[(warp * 5 + 1) * SLOTS + slotA] = stA.s0;
            pb[(warp * 5 + 2) * SLOTS + slotA] = stA.s1;
            pb[(warp * 5 + 3) * SLOTS + slotA] = stA.s2;
            pb[(warp * 5 + 4) * SLOTS + slotA] = stA.s3;
            pb[(warp * 5 + 0) * SLOTS + slotB] = stB.m;
            pb[(warp * 5 + 1) * SLOTS + slotB] = stB.s0;
            pb[(warp * 5 + 2) * SLOTS + slotB] = stB.s1;
            pb[(warp * 5 + 3) * SLOTS + slotB] = stB.s2;
            pb[(warp * 5 + 4) * SLOTS + slotB] = stB.s3;
            named_bar_sync(1, NCONS);
            if (stepper) {
                float y, var;
                merge_partials(pb, tid, yrbuf[o * SLOTS + tid], y, var);
                ybuf[o * SLOTS + tid] = y;
                vbuf[o * SLOTS + tid] = var;
            }
        }

        if (stepper) {
            float y[NY], var[NY];
#pragma unroll
            for (int o = 0; o < NY; ++o) {
                y[o] = ybuf[o * SLOTS + tid];
                var[o] = vbuf[o * SLOTS + tid];
            }
            {
                float x[NX];
#pragma unroll
                for (int c = 0; c < NX; ++c) x[c] = xbuf[c * SLOTS + tid];
                // running cost at (x_t, z_t), averaged over the sub-rollouts of k
                qbuf[tid] = running_cost(a.cost, obs_s, x, var);
                // sampled Euler step (Sec. 3.2)
                float n[NY];
                if (a.model_noise) {
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        float4 nb = box_muller4(noise_block(a.seed, (uint32_t)k, (uint32_t)t,
                                                            (uint32_t)(b + 1), (uint32_t)m));
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
                    float xdot = fmaf(sqrtf(var[c]), n[c], y[c]);
                    x[c] = fmaf(a.dt, xdot, x[c]);
                    xbuf[c * SLOTS + tid] = x[c];
                    zbuf[c * SLOTS + tid] = x[c];
                    yrbuf[c * SLOTS + tid] = y[c];
                }
                named_bar_sync(2, SLOTS);
                if (writer) {
                    float qs = 0.0f;
                    for (int i = 0; i < M; ++i) qs += qbuf[tid + i];
                    a.cost_tk[(size_t)t * a.K + k] = qs / (float)M;
                }
                if (t + 1 < a.T) {
                    float4 nn = box_muller4(noise_block(a.seed, (uint32_t)k, (uint32_t)(t + 1), 0u, 0u));
                    float eps[4] = {a.sqrt_sigma_u[0] * nn.x, a.sqrt_sigma_u[1] * nn.y,
                                    a.sqrt_sigma_u[2] * nn.z, a.sqrt_sigma_u[3] * nn.w};
#pragma unroll
                    for (int c = 0; c < NU; ++c)
                        zbuf[(NX + c) * SLOTS + tid] = a.u_nom[(size_t)(t + 1) * NU + c] + eps[c];
                    if (writer)
                        a.eps_tk[(size_t)(t + 1) * a.K + k] = make_float4(eps[0], eps[1], eps[2], eps[3]);
                } else {
                    named_bar_sync(2, SLOTS);           // qbuf reads done before reuse
                    qbuf[tid] = terminal_cost(a.cost, x);
                    named_bar_sync(2, SLOTS);
                    if (writer) {
                        float ps = 0.0f;
                        for (int i = 0; i < M; ++i) ps += qbuf[tid + i];
                        a.phi[k] = ps / (float)M;
                    }
                }
            }
        }
        const bool any_abort = bar_sync_or(3, NCONS, aborted || *abort_flag != 0);
        if (any_abort) break;
    }
}

// blockIdx.x = 64-slot block.
__global__ void __launch_bounds__(NTHREADS, 1) rollout_fp32_kernel(const __grid_constant__ RolloutArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const Fp32Smem S = fp32_smem(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) fp32_init_barriers(S);
    for (int i = tid; i < a.cost.n_obs; i += NTHREADS) S.obs_s[i] = a.cost.obs[i];
    __syncthreads();
    if (warp == CW) {
        if (lane != 0) return;
        long long issued = 0;
        fp32_producer(a, S, 0, issued);
        // keep the CTA alive until every copy issued has landed
        for (long long g = (issued > NSTAGE ? issued - NSTAGE : 0); g < issued; ++g)
            if (!mbar_wait_drain(&S.full[g % NSTAGE], (uint32_t)((g / NSTAGE) & 1))) atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
        return;
    }
    long long g = 0;
    bool aborted = false;
    fp32_consumer(a, S, ((long long)a.block0 + blockIdx.x) * SLOTS, g, aborted);
}

// ---------------------------------------------------------------------------
// Output-split launch.  With fewer 64-slot blocks than SMs, the one-CTA-per-
// block launch leaves SMs idle (K = 8192: 128 blocks on 148 SMs), and so does
// the last, partial wave of a larger launch.  Here the split_blocks blocks
// from split_b0 on (numbered b = 0, 1, ... below) are evaluated as
// (block, output) units, unit = b * NY + o, dealt out in runs of `upc`
// consecutive units to gridDim.x co-resident CTAs (one per SM, a cooperative
// launch), upc = ceil(split_blocks * NY / SMs) < NY.  Each CTA's run
// covers the end of at most one block (its *owned* block, whose slots it
// steps) and the start or middle of at most one other (a *non-owned*
// segment).  Every output of a block is evaluated by one CTA with the same
// warps, records and merge as in rollout_fp32_kernel, and the owner steps
// the dynamics with the same code, so the results are identical bit for bit.
//
// Per step t, through the exchange area in global memory (L2):
//   - a non-owned segment waits until the owner has published z_t of its
//     block (ready >= t + 1), evaluates its outputs and writes their y and
//     var, then raises its done flag to t + 1;
//   - the owner evaluates its own outputs, waits for the done flags of the
//     block's other CTAs, reads their y and var, steps the dynamics and
//     publishes z_{t+1} (ready = t + 2).
// Each CTA evaluates its non-owned segment first, so the step's waits point
// only to work that the other CTAs do first in their own step: no wait can
// close a cycle.  Flags hold (epoch << 32 | count) with a per-launch epoch,
// so no flag needs clearing between launches.  Every wait is bounded; on
// expiry the CTA flags DEVERR_TIMEOUT_PEER, stores its epoch into the abort
// word (the other CTAs' waits then give up at once) and leaves at the end of
// the step like any aborted CTA.
// ---------------------------------------------------------------------------
constexpr int OFF_ZH = (SMEM_BYTES + 15) / 16 * 16;                 // [NZ][SLOTS] z of the non-owned block
constexpr int OFF_YRH = OFF_ZH + NZ * SLOTS * 4;                     // [NY][SLOTS] its reference means
constexpr int OFF_SOK = OFF_YRH + NY * SLOTS * 4;                    // stepper decision word
constexpr int SPLIT_SMEM_BYTES = OFF_SOK + 16;
static_assert(SPLIT_SMEM_BYTES <= 232448, "shared memory budget");
constexpr size_t SB_READY = 0, SB_DONE = 8, SB_Z = 128, SB_Y = SB_Z + NZ * SLOTS * 4, SB_V = SB_Y + NY * SLOTS * 4;
static_assert(SB_V + NY * SLOTS * 4 == SPLIT_BLOCK_BYTES && SB_DONE + NY * 8 <= SB_Z, "exchange block layout");

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One CTA's share of the units.  Segments are listed in evaluation order:
// the non-owned one (if any) first.
struct SplitPlan {
    int nseg;
    int b[2], o0[2], o1[2], part[2];   // block, outputs [o0, o1), index among the block's non-owners
    bool owned[2];
    int nparts;                        // owned block: CTAs before this one that hold some of its outputs
    int own;                           // segment index of the owned block, or -1
};

__host__ __device__ __forceinline__ SplitPlan split_plan(int cta, int upc, int units)
{
    SplitPlan p{};
    const int s = cta * upc, e = min(s + upc, units);
    const int b1 = s / NY, end1 = (b1 + 1) * NY;
    const bool own1 = e >= end1;
    int n = 0;
    if (e > end1) {   // the start of block b1 + 1, owned by a later CTA
        p.b[n] = b1 + 1;
        p.o0[n] = 0;
        p.o1[n] = e - end1;
        p.owned[n] = false;
        p.part[n] = cta - ((b1 + 1) * NY) / upc;
        ++n;
    }
    p.b[n] = b1;
    p.o0[n] = s - b1 * NY;
    p.o1[n] = min(e, end1) - b1 * NY;
    p.owned[n] = own1;
    p.part[n] = cta - (b1 * NY) / upc;
    p.own = own1 ? n : -1;
    p.nparts = own1 ? cta - (b1 * NY) / upc : 0;
    p.nseg = n + 1;
    return p;
}

// Bounded wait until *flag >= target; gives up when the abort word holds this
// launch's tag or after WAIT_LIMIT_NS.
__device__ __forceinline__ bool split_wait(const unsigned long long *flag, unsigned long long target, const unsigned long long *abortw,
                           unsigned long long tag)
{
    if (ld_acquire_u64(flag) >= target) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        // a plain spin: the rest of the CTA waits at a barrier meanwhile, so
        // the poll takes no issue slots from work
        if (ld_acquire_u64(flag) >= target) return true;
        if ((it & 63u) == 0u) {
            if (ld_relaxed_u64(abortw) == tag) return false;
            if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
        }
    }
}

__device__ __forceinline__ void split_fail(const RolloutArgs &a, const Fp32Smem &S, unsigned long long *abortw,
                                           unsigned long long tag)
{
    if (ld_relaxed_u64(abortw) != tag) atomicOr(a.err, DEVERR_TIMEOUT_PEER);
    st_release_u64(abortw, tag);
    *S.abort_flag = 1;
}

// Exchange block b of the split area.
__device__ __forceinline__ unsigned char *split_blk(const RolloutArgs &a, int b)
{
    return a.split + SPLIT_HDR_BYTES + (size_t)b * SPLIT_BLOCK_BYTES;
}

__device__ __forceinline__ unsigned long long split_tag(const RolloutArgs &a)
{
    return (unsigned long long)a.split_epoch << 32;
}

// Per-CTA unit table of the split kernel (shared memory): unit u of a step
// evaluates output uo[u] of the owned block (UF_OWNED) or of the non-owned
// one; UF_FIRST / UF_LAST mark the first and last unit of a segment.
constexpr int UF_OWNED = 1, UF_FIRST = 2, UF_LAST = 4;
struct SplitUnits {
    int n;                 // units per step
    int uo[NY], uf[NY];
    int bN, partN;         // non-owned segment (bN < 0: none): block, index among its non-owners
    int o0N, o1N;          // its outputs
    int bO, o0O, npartsO;  // owned block (bO < 0: none), its first output, CTAs before this one holding its outputs
};

__device__ __forceinline__ void split_units(const SplitPlan &p, SplitUnits &u)
{
    u.n = 0;
    u.bN = -1;
    u.partN = 0;
    u.o0N = u.o1N = 0;
    u.bO = -1;
    u.o0O = 0;
    u.npartsO = 0;
    for (int si = 0; si < p.nseg; ++si) {
        for (int o = p.o0[si]; o < p.o1[si]; ++o) {
            u.uo[u.n] = o;
            u.uf[u.n] = (p.owned[si] ? UF_OWNED : 0) | (o == p.o0[si] ? UF_FIRST : 0) | (o + 1 == p.o1[si] ? UF_LAST : 0);
            ++u.n;
        }
        if (p.owned[si]) {
            u.bO = p.b[si];
            u.o0O = p.o0[si];
            u.npartsO = p.nparts;
        } else {
            u.bN = p.b[si];
            u.partN = p.part[si];
            u.o0N = p.o0[si];
            u.o1N = p.o1[si];
        }
    }
}

// One segment of a split CTA's step: outputs [o0, o1) of the owned block
// (OWNED; z, reference means, y and var in the CTA's own buffers) or of the
// non-owned one (z in zH, reference means in yrH, y and var to the exchange
// block bb).  Each instantiation is the plain kernel's output loop: z loaded
// once before it, nothing else live across the record loop but the loop
// bound and the partial-buffer parity.
__shared__ SplitUnits s_split;   // the split kernel's unit table (static shared memory)

template <bool OWNED>
__device__ __forceinline__ void fp32_split_segment(const RolloutArgs &a, const Fp32Smem &S, const float *zsrc, float *yrs,
                                                   int o0, int o1, int &par, long long &g, bool &aborted)
{
    const int tid = threadIdx.x, lane = tid & 31;
    float2 zA[NZ], zB[NZ];
    fp32_load_z(zsrc, zA, zB);
    for (int o = o0; o < o1; ++o) {
        fp32_output_pass(a, S, zA, zB, -yrs[o * SLOTS + lane], -yrs[o * SLOTS + lane + 32], par & 1, g, aborted,
                         a.P, a.stages_per_out);
        named_bar_sync(1, NCONS);
        const float *pb = S.part + (par & 1) * PART_BUF;
        ++par;
        if (tid < SLOTS) {
            float y, var;
            merge_partials(pb, tid, yrs[o * SLOTS + tid], y, var);
            if (OWNED) {
                S.ybuf[o * SLOTS + tid] = y;
                S.vbuf[o * SLOTS + tid] = var;
            } else {
                // the exchange block is found again here rather than kept in
                // registers across the record loop
                unsigned char *bb = split_blk(a, *(volatile int *)&s_split.bN);
                __stcg(reinterpret_cast<float *>(bb + SB_Y) + o * SLOTS + tid, y);
                __stcg(reinterpret_cast<float *>(bb + SB_V) + o * SLOTS + tid, var);
                yrs[o * SLOTS + tid] = y;
            }
        }
    }
}

// Consumers of the split kernel: per step the non-owned segment (after the
// owner has published its block's z), then the owned one, then the owned
// block's dynamics (after the other CTAs' outputs of it have arrived).
__device__ __forceinline__ void fp32_split_consumer(const RolloutArgs &a, const Fp32Smem &S, const volatile SplitUnits &U,
                                                    float *zH, float *yrH, volatile int *s_ok)
{
    const int tid = threadIdx.x;
    const bool stepper = tid < SLOTS;
    unsigned long long *abortw = reinterpret_cast<unsigned long long *>(a.split);
    long long g = 0;
    bool aborted = false;

    if (stepper) {
#pragma unroll
        for (int o = 0; o < NY; ++o) yrH[o * SLOTS + tid] = 0.0f;
        if (U.bO >= 0) {
            const long long gslot = (long long)(a.split_b0 + U.bO) * SLOTS + tid;
            const int k = (int)(gslot / a.M), m = (int)(gslot % a.M);
            fp32_init_slot(a, S, tid, k, k < a.K && m == 0);
            unsigned char *ob = split_blk(a, U.bO);
            float *zg = reinterpret_cast<float *>(ob + SB_Z);
#pragma unroll
            for (int c = 0; c < NZ; ++c) __stcg(&zg[c * SLOTS + tid], S.zbuf[c * SLOTS + tid]);
            named_bar_sync(2, SLOTS);
            if (tid == 0) st_release_u64(reinterpret_cast<unsigned long long *>(ob + SB_READY), split_tag(a) | 1ull);
        }
    }
    named_bar_sync(1, NCONS);

    int par = 0;   // partial-buffer parity, alternating over the CTA's units
    for (int t = 0; t < a.T; ++t) {
        if (U.bN >= 0) {
            unsigned char *bb = split_blk(a, U.bN);
            if (stepper) {
                if (tid == 0 && !aborted &&
                    !split_wait(reinterpret_cast<const unsigned long long *>(bb + SB_READY),
                                split_tag(a) | (unsigned long long)(t + 1), abortw, split_tag(a))) {
                    split_fail(a, S, abortw, split_tag(a));
                    aborted = true;
                }
                named_bar_sync(2, SLOTS);
                const float *zg = reinterpret_cast<const float *>(bb + SB_Z);
#pragma unroll
                for (int c = 0; c < NZ; ++c) zH[c * SLOTS + tid] = __ldcg(&zg[c * SLOTS + tid]);
            }
            named_bar_sync(1, NCONS);
            fp32_split_segment<false>(a, S, zH, yrH, U.o0N, U.o1N, par, g, aborted);
            if (stepper) {
                named_bar_sync(2, SLOTS);
                if (tid == 0)
                    st_release_u64(reinterpret_cast<unsigned long long *>(split_blk(a, U.bN) + SB_DONE) + U.partN,
                                   split_tag(a) | (unsigned long long)(t + 1));
            }
        }
        if (U.bO >= 0) {
            fp32_split_segment<true>(a, S, S.zbuf, S.yrbuf, U.o0O, NY, par, g, aborted);
            if (stepper) {
                unsigned char *ob = split_blk(a, U.bO);
                if (tid == 0) {
                    bool ok = !aborted && *S.abort_flag == 0;
                    for (int p = 0; ok && p < U.npartsO; ++p)
                        ok = split_wait(reinterpret_cast<const unsigned long long *>(ob + SB_DONE) + p,
                                        split_tag(a) | (unsigned long long)(t + 1), abortw, split_tag(a));
                    if (!ok && !aborted) {
                        split_fail(a, S, abortw, split_tag(a));
                        aborted = true;
                    }
                    *s_ok = ok ? 1 : 0;
                }
                named_bar_sync(2, SLOTS);
                if (*s_ok) {
                    const float *yg = reinterpret_cast<const float *>(ob + SB_Y), *vg = reinterpret_cast<const float *>(ob + SB_V);
                    for (int o = 0; o < U.o0O; ++o) {
                        S.ybuf[o * SLOTS + tid] = __ldcg(&yg[o * SLOTS + tid]);
                        S.vbuf[o * SLOTS + tid] = __ldcg(&vg[o * SLOTS + tid]);
                    }
                    const long long gslot = (long long)(a.split_b0 + U.bO) * SLOTS + tid;
                    const int k = (int)(gslot / a.M), m = (int)(gslot % a.M);
                    fp32_step_slot(a, S, t, tid, k, m, k < a.K && m == 0);
                    if (t + 1 < a.T) {
                        float *zg = reinterpret_cast<float *>(ob + SB_Z);
#pragma unroll
                        for (int c = 0; c < NZ; ++c) __stcg(&zg[c * SLOTS + tid], S.zbuf[c * SLOTS + tid]);
                        named_bar_sync(2, SLOTS);
                        if (tid == 0)
                            st_release_u64(reinterpret_cast<unsigned long long *>(ob + SB_READY),
                                           split_tag(a) | (unsigned long long)(t + 2));
                    }
                }
            }
        }
        const bool any_abort = bar_sync_or(3, NCONS, aborted || *S.abort_flag != 0);
        if (any_abort) {
            if (tid == 0) st_release_u64(abortw, split_tag(a));   // the other CTAs stop waiting for this one
            break;
        }
    }
}

// Release stores after a CTA barrier: the barrier orders the other stepper
// threads' stores before thread 0's release, which makes them visible to the
// CTA that acquires the flag (the acquirer's threads then read after their own
// barrier, through L2).
__global__ void __launch_bounds__(NTHREADS, 1) rollout_fp32_split_kernel(const __grid_constant__ RolloutArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    SplitUnits &s_units = s_split;
    const Fp32Smem S = fp32_smem(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        split_units(split_plan((int)blockIdx.x, a.split_upc, a.split_blocks * NY), s_units);
        fp32_init_barriers(S);
    }
    for (int i = tid; i < a.cost.n_obs; i += NTHREADS) S.obs_s[i] = a.cost.obs[i];
    __syncthreads();
    const volatile SplitUnits &pl = s_units;
    if (warp == CW) {
        if (lane != 0) return;
        long long issued = 0;
        fp32_produce(a, S, 0, issued, pl.n, [&](int i) { return pl.uo[i]; });
        for (long long g = (issued > NSTAGE ? issued - NSTAGE : 0); g < issued; ++g)
            if (!mbar_wait_drain(&S.full[g % NSTAGE], (uint32_t)((g / NSTAGE) & 1))) atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
        return;
    }
    fp32_split_consumer(a, S, pl, reinterpret_cast<float *>(smem + OFF_ZH), reinterpret_cast<float *>(smem + OFF_YRH),
                        reinterpret_cast<volatile int *>(smem + OFF_SOK));
}

// Persistent batched form: CTAs take (controller, slot block) work items from
// an atomic counter until the list is exhausted; every controller has its own
// RolloutArgs (model, cost, sizes, buffers).  Ring positions carry over
// between items, so the barriers are initialized once.
__global__ void __launch_bounds__(NTHREADS, 1) rollout_fp32_batch_kernel(const __grid_constant__ BatchArgs b)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ RolloutArgs s_args;
    __shared__ int s_item;
    const Fp32Smem S = fp32_smem(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) fp32_init_barriers(S);
    long long g = 0, issued = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= b.n_items || *S.abort_flag) break;
        const int2 it = b.items[item];
        if (tid == 0) s_args = b.args[it.x];
        __syncthreads();
        const RolloutArgs &a = s_args;
        for (int i = tid; i < a.cost.n_obs; i += NTHREADS) S.obs_s[i] = a.cost.obs[i];
        __syncthreads();
        if (warp == CW) {
            if (lane == 0) {
                const long long next = fp32_producer(a, S, g, issued);
                g = next < 0 ? g : next;
            }
        } else {
            fp32_consumer(a, S, (long long)it.y * SLOTS, g, aborted);
        }
        __syncthreads();
    }
    if (warp == CW && lane == 0)
        for (long long r = (issued > NSTAGE ? issued - NSTAGE : 0); r < issued; ++r)
            if (!mbar_wait_drain(&S.full[r % NSTAGE], (uint32_t)((r / NSTAGE) & 1))) atomicOr(b.err, DEVERR_TIMEOUT_DRAIN);
}

// One (controller, 64-slot block) item per CTA, arguments from the device
// table (the plain-launch form of the batch: the block scheduler fills SMs as
// items finish).
__global__ void __launch_bounds__(NTHREADS, 1) rollout_fp32_group_kernel(const __grid_constant__ BatchArgs b)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ RolloutArgs s_args;
    const Fp32Smem S = fp32_smem(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int2 it = b.items[blockIdx.x];
    if (tid == 0) {
        s_args = b.args[it.x];
        fp32_init_barriers(S);
    }
    __syncthreads();
    const RolloutArgs &a = s_args;
    for (int i = tid; i < a.cost.n_obs; i += NTHREADS) S.obs_s[i] = a.cost.obs[i];
    __syncthreads();
    if (warp == CW) {
        if (lane != 0) return;
        long long issued = 0;
        fp32_producer(a, S, 0, issued);
        for (long long g = (issued > NSTAGE ? issued - NSTAGE : 0); g < issued; ++g)
            if (!mbar_wait_drain(&S.full[g % NSTAGE], (uint32_t)((g / NSTAGE) & 1))) atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
        return;
    }
    long long g = 0;
    bool aborted = false;
    fp32_consumer(a, S, (long long)it.y * SLOTS, g, aborted);
}

std::atomic<uint64_t> g_attr_set;

// Prediction of a few rows (the receding-horizon plant step, one row, and a
// serving group's plant steps, one row per agent): one cluster of PR_SPLIT
// CTAs per (row, output), PR_THREADS threads in all.  Thread v of the cluster
// takes the output's field pairs p = v, v + PR_THREADS, ... for that one row;
// it copies each record into shared memory with all of its 16-byte copies in
// flight (cp.async), which turns the walk through the record from a chain of
// dependent global loads into one round trip.  The per-thread softmax states
// are merged in a fixed order (a shuffle tree per warp, then the warps in
// order by cluster rank 0 over distributed shared memory), so every row's
// result is deterministic and independent of the other rows.  Two passes: the
// second centres the local predictions on the first pass's mean (the centring
// the rollout kernel gets from the last step); with at most PR_THREADS pairs
// the records stay in shared memory for it.
constexpr int PR_THREADS = 256;

__device__ __forceinline__ void soft_merge(Soft &a, const Soft &b)
{
    const float M = fmaxf(a.m, b.m);
    if (M == -INFINITY) return;   // neither holds a field yet
    const float ca = ex2(a.m - M), cb = ex2(b.m - M);
    a.s0 = fmaf(a.s0, ca, b.s0 * cb);
    a.s1 = fmaf(a.s1, ca, b.s1 * cb);
    a.s2 = fmaf(a.s2, ca, b.s2 * cb);
    a.s3 = fmaf(a.s3, ca, b.s3 * cb);
    a.m = M;
}

constexpr int PR_SPLIT = 4;                               // CTAs per (row, output): one cluster
constexpr int PR_CTA_THREADS = PR_THREADS / PR_SPLIT;     // 64
constexpr int PR_SMEM = PR_CTA_THREADS * REC_BYTES;       // one record per thread: 88,064 B

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ float ld_cluster_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// blockIdx = (row, output, cluster rank).  Thread t of rank c is thread
// v = c * PR_CTA_THREADS + t of the cluster.
__global__ void __launch_bounds__(PR_CTA_THREADS) predict_rows_kernel(const __grid_constant__ RolloutArgs a)
{
    extern __shared__ __align__(16) unsigned char pr_rec[];
    __shared__ Soft wpart[PR_CTA_THREADS / 32];
    __shared__ float yvar[2];
    const int row = blockIdx.x, o = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t crank = cluster_rank();
    const int vt = (int)crank * PR_CTA_THREADS + tid;
    float2 z2[NZ];
#pragma unroll
    for (int c = 0; c < NZ; ++c) {
        const float zc = a.z_in[(size_t)row * NZ + c];
        z2[c] = make_float2(zc, zc);
    }
    float4 *mine = reinterpret_cast<float4 *>(pr_rec + (size_t)tid * REC_BYTES);
    const int rounds = (a.P + PR_THREADS - 1) / PR_THREADS;
    float yref = 0.0f, y = 0.0f, var = 0.0f;
    for (int pass = 0; pass < 2; ++pass) {
        const float2 yr = make_float2(-yref, -yref);
        Soft st, unused;
        soft_init(st);
        soft_init(unused);
        for (int i = 0; i < rounds; ++i) {
            const int p = vt + i * PR_THREADS;
            if (p >= a.P) break;
            if (pass == 0 || rounds > 1) {   // with one round the record stays for the second pass
                const float4 *src = reinterpret_cast<const float4 *>(a.rec + ((size_t)o * a.P + p) * REC_LEN);
#pragma unroll 2
                for (int j = 0; j < REC_BYTES / 16; ++j) cp_async16(mine + j, src + j);
                cp_async_wait_all();
            }
            process_pair(mine, z2, z2, yr, yr, st, unused);   // the second slot is not needed
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Soft other{__shfl_down_sync(0xffffffffu, st.m, off), __shfl_down_sync(0xffffffffu, st.s0, off),
                             __shfl_down_sync(0xffffffffu, st.s1, off), __shfl_down_sync(0xffffffffu, st.s2, off),
                             __shfl_down_sync(0xffffffffu, st.s3, off)};
            soft_merge(st, other);
        }
        if (lane == 0) wpart[warp] = st;
        cluster_sync_all();   // every rank's warp states written
        if (crank == 0 && tid == 0) {
            Soft all = wpart[0];
            for (int w = 1; w < PR_THREADS / 32; ++w) {
                const uint32_t base = mapa_shared(&wpart[w % (PR_CTA_THREADS / 32)], (uint32_t)(w / (PR_CTA_THREADS / 32)));
                const Soft other{ld_cluster_f32(base), ld_cluster_f32(base + 4), ld_cluster_f32(base + 8),
                                 ld_cluster_f32(base + 12), ld_cluster_f32(base + 16)};
                soft_merge(all, other);
            }
            const float inv = 1.0f / all.s0;
            const float mean_e = all.s1 * inv;
            const float yv = yref + mean_e;
            const float vv = fmaxf(fmaf(-mean_e, mean_e, all.s2 * inv), 0.0f) + all.s3 * inv;
            for (uint32_t r = 0; r < PR_SPLIT; ++r) {
                st_cluster_f32(mapa_shared(&yvar[0], r), yv);
                st_cluster_f32(mapa_shared(&yvar[1], r), vv);
            }
        }
        cluster_sync_all();   // yvar everywhere; the warp states read
        y = yvar[0];
        var = yvar[1];
        yref = y;
    }
    if (crank == 0 && tid == 0) {
        a.y_out[(size_t)row * NY + o] = y;
        a.var_out[(size_t)row * NY + o] = var;
    }
}

std::atomic<uint64_t> g_pred_attr;

// One CTA per 64-slot block for blocks [block0, block0 + blocks).
cudaError_t launch_impl(const RolloutArgs &a, cudaStream_t s, long long block0, long long blocks)
{
    if (a.cost.n_obs > MAX_OBS || a.P <= 0 || a.stages_per_out <= 0) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_once(g_attr_set, rollout_fp32_kernel, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (blocks <= 0 || blocks > 0x7fffffffLL || block0 < 0 || block0 > 0x7fffffffLL) return cudaErrorInvalidValue;
    RolloutArgs b = a;
    b.block0 = (int)block0;
    rollout_fp32_kernel<<<(unsigned)blocks, NTHREADS, SMEM_BYTES, s>>>(b);
    return cudaGetLastError();
}

}  // namespace

std::atomic<uint64_t> g_split_attr;

Fp32Launch fp32_plan_blocks(long long blocks, int nsm, int P, int mode, int max_blocks)
{
    Fp32Launch L{};
    L.plain_blocks = (int)blocks;
    if (mode == PI_SPLIT_OFF || blocks <= 0 || nsm <= 0) return L;
    // Whole waves of blocks keep the plain launch (every SM busy); only the
    // blocks of a last, partial wave are split over all SMs.
    const long long tail = blocks % nsm;
    if (tail == 0 || tail > max_blocks) return L;
    const long long upc = (tail * NY + nsm - 1) / nsm;
    if (upc >= NY) return L;
    // In auto mode, split only where the per-step work it takes off the
    // busiest CTA (NY - upc outputs of P records) clearly outweighs the two
    // flag round trips through L2 that it adds to each step.
    if (mode == PI_SPLIT_AUTO && (NY - upc) * (long long)P < 64) return L;
    L.plain_blocks = (int)(blocks - tail);
    L.split_b0 = (int)(blocks - tail);
    L.split_blocks = (int)tail;
    L.upc = (int)upc;
    L.split_ctas = (int)((tail * NY + upc - 1) / upc);
    return L;
}

int fp32_split_partition(int blocks, int upc, int cta, int *seg)
{
    if (blocks < 1 || upc < 1 || upc >= NY || cta < 0 || cta * upc >= blocks * NY) return 0;
    const SplitPlan p = split_plan(cta, upc, blocks * NY);
    for (int i = 0; i < p.nseg; ++i) {
        seg[5 * i + 0] = p.b[i];
        seg[5 * i + 1] = p.o0[i];
        seg[5 * i + 2] = p.o1[i];
        seg[5 * i + 3] = p.owned[i] ? 1 : 0;
        seg[5 * i + 4] = p.owned[i] ? p.nparts : p.part[i];
    }
    return p.nseg;
}

Fp32Launch fp32_launch_plan(const RolloutArgs &a, cudaStream_t s)
{
    const long long blocks = a.K >= 1 && a.M >= 1 ? ((long long)a.K * a.M + SLOTS - 1) / SLOTS : 0;
    Fp32Launch L{};
    L.plain_blocks = (int)blocks;
    if (!a.split || a.split_mode == PI_SPLIT_OFF || blocks <= 0) return L;
    // A launch captured into a CUDA graph would replay with the epoch of the
    // capture, and the flags of one replay would satisfy the waits of the
    // next: captured updates take the plain launch.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return L;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return L;
    return fp32_plan_blocks(blocks, nsm, a.P, a.split_mode, a.split_max_blocks);
}

cudaError_t launch_rollout_fp32(const RolloutArgs &a, cudaStream_t s, int *n_launched)
{
    if (n_launched) *n_launched = 0;
    if (a.M < 1 || a.M > SLOTS || (a.M & (a.M - 1)) != 0) return cudaErrorInvalidValue;
    const Fp32Launch L = fp32_launch_plan(a, s);
    if (L.upc <= 0) {
        cudaError_t e = launch_impl(a, s, 0, L.plain_blocks);
        if (e == cudaSuccess && n_launched) *n_launched = 1;
        return e;
    }
    if (a.cost.n_obs > MAX_OBS || a.P <= 0 || a.stages_per_out <= 0 || a.split_epoch == 0)
        return cudaErrorInvalidValue;
    if (L.plain_blocks > 0) {   // the whole waves: blocks [0, plain_blocks)
        cudaError_t e = launch_impl(a, s, 0, L.plain_blocks);
        if (e != cudaSuccess) return e;
        if (n_launched) *n_launched = 1;
    }
    cudaError_t e = set_smem_once(g_split_attr, rollout_fp32_split_kernel, SPLIT_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    RolloutArgs b = a;
    b.split_upc = L.upc;
    b.split_b0 = L.split_b0;
    b.split_blocks = L.split_blocks;
    const int grid = L.split_ctas - (a.split_drop > 0 ? 1 : 0);
    if (grid < 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = SPLIT_SMEM_BYTES;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeCooperative;   // every CTA resident at once: they wait on one another
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = a.split_drop == 2 ? cudaErrorCooperativeLaunchTooLarge : cudaLaunchKernelEx(&cfg, rollout_fp32_split_kernel, b);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        // Fewer SMs than the device has are open to this process (MPS, green
        // contexts), so the CTAs cannot all be resident: the split blocks run
        // as plain blocks instead, with the same results.
        if (a.split_drop != 2) (void)cudaGetLastError();
        e = launch_impl(a, s, L.split_b0, L.split_blocks);
    }
    if (e == cudaSuccess && n_launched) *n_launched += 1;
    return e;
}

cudaError_t launch_predict_fp32(const RolloutArgs &a, cudaStream_t s)
{
    if (a.n_pred <= 0 || a.P <= 0) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_once(g_pred_attr, predict_rows_kernel, PR_SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3((unsigned)a.n_pred, NY, PR_SPLIT);
    cfg.blockDim = dim3(PR_CTA_THREADS);
    cfg.dynamicSmemBytes = PR_SMEM;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = PR_SPLIT;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, predict_rows_kernel, a);
}

std::atomic<uint64_t> g_batch_attr, g_group_attr;

cudaError_t launch_rollout_fp32_batch(const BatchArgs &b, int grid, cudaStream_t s)
{
    cudaError_t e = set_smem_once(g_batch_attr, rollout_fp32_batch_kernel, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaErrorInvalidValue;
    rollout_fp32_batch_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_rollout_fp32_group(const BatchArgs &b, cudaStream_t s)
{
    cudaError_t e = set_smem_once(g_group_attr, rollout_fp32_group_kernel, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (b.n_items <= 0) return cudaErrorInvalidValue;
    rollout_fp32_group_kernel<<<b.n_items, NTHREADS, SMEM_BYTES, s>>>(b);
    return cudaGetLastError();
}

}  // namespace pi2rh

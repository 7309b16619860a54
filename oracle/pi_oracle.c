/*
 * pi_oracle.c -- FP64 CPU oracle for one PI^2-RH control update over a learned
 * LWPR dynamics model ("GPU based Path Integral Control with Learned Dynamics",
 * Williams, Rombokas, Daniel; arXiv 1503.00330).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant generator with
 * the CUDA library; the two meet only in the seeded input generator, which holds
 * none of the method's arithmetic.
 *
 * Every step is written out plainly in double precision, in the order the paper
 * states it, with no blocking, fusion or reordering:
 *
 *   Sec. 2, Eq. 1      LWPR prediction: normalized Gaussian receptive-field
 *                      weights, weighted mean of local linear models, weighted
 *                      variance (spread of the local predictions + per-field noise).
 *   Sec. 3.2           sampled next state from the predicted mean and variance,
 *                      M sub-rollouts per rollout with the cost averaged over them.
 *   Table 1 caption    Euler integration of the predicted state derivatives.
 *   Sec. 3.1, after Eq. 2   passive cost-to-go S(tau_i) = phi + sum_{j>=i} q dt.
 *   Sec. 3.1, Eq. 2    per-timestep weights exp(-S/lambda) / sum, and the weighted
 *                      average of the control perturbations (u_L reduces to the
 *                      control perturbation when G_c = B_c on the control channel).
 *   Sec. 5             experiment cost (waypoint distance, angles, velocities,
 *                      Gaussian obstacle bumps, crash indicator); terminal cost
 *                      and control-cost terms set to zero in the paper.
 *
 * Readings taken where the paper is silent or garbled (each is listed in the
 * design notes of the repository):
 *   - Eq. 1 prints D_j in the denominator and sigma_k in the variance; read as
 *     D_i (the only normalizing reading) and sigma_j of field j.
 *   - exp(-q/2) is evaluated min-shifted (equal to Eq. 1 wherever Eq. 1 is
 *     defined, and defined where the unshifted form underflows).
 *   - local linear model y_j(z) = b_j + beta_j . (z - c_j).
 *   - sampled step: x_{t+1} = x_t + dt * (y + sigma (.) n), n ~ N(0, I).
 *   - running cost q_j is evaluated at (x_j, z_j = [x_j, u_j]) for j = i..T-1,
 *     plus the terminal cost phi(x_T).
 *   - noise: Philox4x32-10 (Salmon et al., SC'11) with counter (k, t, blk, m) and
 *     key (seed lo, seed hi); uniforms u = (2*(r >> 9) + 1) * 2^-24 (exact in
 *     FP32 and FP64); Box-Muller in double precision.
 *   - the obstacle indicator of Sec. 5 (inside a cylinder of radius r, strict
 *     "<": a point on the boundary is outside) is decided in FP64 on the FP64
 *     state, like every other step here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NX 12
#define ORC_NU 4
#define ORC_NZ 16
#define ORC_NY 12

/* ------------------------------------------------------------------------ */
/* Parameter structures (plain double arrays, row-major).                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int L;               /* receptive fields per output                      */
    double dt;           /* Euler step                                       */
    const double *c;     /* [NY][L][NZ]     centers                          */
    const double *D;     /* [NY][L][NZ][NZ] distance metrics                 */
    const double *beta;  /* [NY][L][NZ]     local slopes                     */
    const double *b;     /* [NY][L]         local offsets (value at c_j)     */
    const double *sigma; /* [NY][L]         per-field noise std              */
} orc_lwpr;

typedef struct {
    double goal[3];
    double Q_pos[3];     /* weights on (p - goal)^2 per axis                 */
    double Q_vel;        /* weight on |velocity|^2                           */
    double Q_ang;        /* weight on |roll, pitch, yaw|^2                   */
    double w_obs;        /* obstacle weight                                  */
    double obs_sharp;    /* exponent scale of the Gaussian bump (kind 1)     */
    double radius;       /* cylinder radius                                  */
    double w_crash;      /* weight on the crash indicator                    */
    double w_var;        /* weight on the predicted variance                 */
    double w_T;          /* terminal-cost weight                             */
    int obs_kind;        /* 0: w_obs * indicator, 1: w_obs * sum of bumps    */
    int n_obs;
    const double *obs_xy;/* [n_obs][2]                                       */
} orc_cost;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with    */
/* the key bumped by the Weyl increments between rounds.                    */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += weyl0; k1 += weyl1; }
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0, 1) from the top 23 bits: odd multiples of 2^-24. */
double orc_uniform(uint32_t r)
{
    return (double)(2u * (r >> 9) + 1u) * 0x1p-24;
}

/* Four standard normals from one Philox block by Box-Muller on the pairs
 * (u0, u1) and (u2, u3). */
static void box_muller4(const uint32_t r[4], double n[4])
{
    for (int p = 0; p < 2; ++p) {
        double ua = orc_uniform(r[2 * p]);
        double ub = orc_uniform(r[2 * p + 1]);
        double rad = sqrt(-2.0 * log(ua));
        n[2 * p]     = rad * cos(2.0 * M_PI * ub);
        n[2 * p + 1] = rad * sin(2.0 * M_PI * ub);
    }
}

/* Raw Philox block for (rollout k, step t, block blk, sub-rollout m). */
void orc_noise_raw(uint64_t seed, uint32_t k, uint32_t t, uint32_t blk, uint32_t m, uint32_t out[4])
{
    uint32_t ctr[4] = {k, t, blk, m};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Standard normals for one rollout-step: block 0 (always sub-rollout 0, so the
 * control perturbation is shared by the sub-rollouts of a rollout) gives the 4
 * control normals; blocks 1..3 of sub-rollout m give the 12 model normals. */
void orc_normals(uint64_t seed, uint32_t k, uint32_t t, uint32_t m, double ctrl[4], double model[12])
{
    uint32_t r[4];
    orc_noise_raw(seed, k, t, 0, 0, r);
    box_muller4(r, ctrl);
    for (uint32_t blk = 1; blk <= 3; ++blk) {
        orc_noise_raw(seed, k, t, blk, m, r);
        box_muller4(r, model + 4 * (blk - 1));
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, Eq. 1: LWPR mean and variance at input z (NZ dims), per output.  */
/* ------------------------------------------------------------------------ */
void orc_lwpr_predict(const orc_lwpr *P, const double *z, double *y_out, double *var_out)
{
    const int L = P->L;
    double *s = (double *)malloc(sizeof(double) * (size_t)L);
    double *w = (double *)malloc(sizeof(double) * (size_t)L);
    double *yj = (double *)malloc(sizeof(double) * (size_t)L);
    for (int o = 0; o < ORC_NY; ++o) {
        /* exponent -1/2 (z - c_j)^T D_j (z - c_j) of every field */
        for (int j = 0; j < L; ++j) {
            const double *c = P->c + ((size_t)o * L + j) * ORC_NZ;
            const double *D = P->D + ((size_t)o * L + j) * ORC_NZ * ORC_NZ;
            double dz[ORC_NZ];
            for (int a = 0; a < ORC_NZ; ++a) dz[a] = z[a] - c[a];
            double q = 0.0;
            for (int a = 0; a < ORC_NZ; ++a)
                for (int bb = 0; bb < ORC_NZ; ++bb)
                    q += dz[a] * D[a * ORC_NZ + bb] * dz[bb];
            s[j] = -0.5 * q;
            /* local linear model centered at c_j */
            const double *beta = P->beta + ((size_t)o * L + j) * ORC_NZ;
            double yl = P->b[(size_t)o * L + j];
            for (int a = 0; a < ORC_NZ; ++a) yl += beta[a] * dz[a];
            yj[j] = yl;
        }
        /* normalized weights, shifted by the largest exponent */
        double smax = s[0];
        for (int j = 1; j < L; ++j) if (s[j] > smax) smax = s[j];
        double denom = 0.0;
        for (int j = 0; j < L; ++j) { w[j] = exp(s[j] - smax); denom += w[j]; }
        for (int j = 0; j < L; ++j) w[j] /= denom;
        /* mean: y = sum_j w_j y_j */
        double y = 0.0;
        for (int j = 0; j < L; ++j) y += w[j] * yj[j];
        /* variance: sum_j w_j ((y - y_j)^2 + sigma_j^2), second pass */
        double var = 0.0;
        for (int j = 0; j < L; ++j) {
            double sj = P->sigma[(size_t)o * L + j];
            double dy = y - yj[j];
            var += w[j] * (dy * dy + sj * sj);
        }
        y_out[o] = y;
        var_out[o] = var;
    }
    free(s); free(w); free(yj);
}

/* ------------------------------------------------------------------------ */
/* Sec. 5 (and the obstacle-navigation configurations): running cost q(x)   */
/* plus the variance penalty, and the terminal cost phi(x_T).               */
/* State layout: x[0..2] position, x[3..5] velocity, x[6..8] roll, pitch,   */
/* yaw, x[9..11] body rates.                                                */
/* ------------------------------------------------------------------------ */

/* Sec. 5 crash indicator C: 1 when the position lies strictly inside some
 * vertical cylinder of radius r (d^2 < r^2), decided in FP64. */
int orc_inside_any(const orc_cost *C, double px, double py)
{
    const double r2 = C->radius * C->radius;
    for (int i = 0; i < C->n_obs; ++i) {
        double dx = px - C->obs_xy[2 * i];
        double dy = py - C->obs_xy[2 * i + 1];
        if (dx * dx + dy * dy < r2) return 1;
    }
    return 0;
}

double orc_running_cost(const orc_cost *C, const double *x, const double *var)
{
    double q = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = x[d] - C->goal[d];
        q += C->Q_pos[d] * e * e;
    }
    double v2 = x[3] * x[3] + x[4] * x[4] + x[5] * x[5];
    double a2 = x[6] * x[6] + x[7] * x[7] + x[8] * x[8];
    q += C->Q_vel * v2 + C->Q_ang * a2;
    int inside = orc_inside_any(C, x[0], x[1]);
    if (C->obs_kind == 0) {
        q += C->w_obs * (double)inside;
    } else {
        double bump = 0.0;
        for (int i = 0; i < C->n_obs; ++i) {
            double dx = x[0] - C->obs_xy[2 * i];
            double dy = x[1] - C->obs_xy[2 * i + 1];
            bump += exp(-C->obs_sharp * (dx * dx + dy * dy));
        }
        q += C->w_obs * bump;
    }
    q += C->w_crash * (double)inside;
    double vs = 0.0;
    for (int o = 0; o < ORC_NY; ++o) vs += var[o];
    q += C->w_var * vs;
    return q;
}

double orc_terminal_cost(const orc_cost *C, const double *x)
{
    double phi = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = x[d] - C->goal[d];
        phi += C->Q_pos[d] * e * e;
    }
    return C->w_T * phi;
}

/* ------------------------------------------------------------------------ */
/* Rollouts (Sec. 3.1 sampling, Sec. 3.2 sub-rollouts, Euler steps).        */
/*   eps  [K][T][NU]  control perturbations (shared by the sub-rollouts)    */
/*   cost [K][T]      running cost averaged over the M sub-rollouts         */
/*   phi  [K]         terminal cost averaged over the M sub-rollouts        */
/*   xtraj[K][M][T+1][NX] (optional, may be NULL) visited states            */
/* model_noise: 1 = sampled draw, 0 = mean prediction only.                 */
/* ------------------------------------------------------------------------ */
/* Rollouts k0 .. k0+K-1 of an update (row r of the outputs is rollout k0 + r);
 * rollout k only depends on its own noise counters, so any subset can be run. */
void orc_rollouts_from(const orc_lwpr *P, const orc_cost *C, const double *x0, const double *u_nom,
                       int k0, int K, int T, int M, const double *sigma_u, uint64_t seed,
                       int model_noise, double *eps_out, double *cost_out, double *phi_out,
                       double *xtraj_out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < K; ++r) {
        const int k = k0 + r;
        double *eps = eps_out - (size_t)k0 * T * ORC_NU;
        double *cost = cost_out - (size_t)k0 * T;
        double *phi = phi_out - k0;
        double *xtraj = xtraj_out ? xtraj_out - (size_t)k0 * M * (T + 1) * ORC_NX : NULL;
        for (int t = 0; t < T; ++t) cost[(size_t)k * T + t] = 0.0;
        phi[k] = 0.0;
        for (int m = 0; m < M; ++m) {
            double x[ORC_NX];
            memcpy(x, x0, sizeof(x));
            if (xtraj) memcpy(xtraj + (((size_t)k * M + m) * (T + 1)) * ORC_NX, x, sizeof(x));
            for (int t = 0; t < T; ++t) {
                double nc[4], nm[12];
                orc_normals(seed, (uint32_t)k, (uint32_t)t, (uint32_t)m, nc, nm);
                double z[ORC_NZ];
                for (int a = 0; a < ORC_NX; ++a) z[a] = x[a];
                for (int a = 0; a < ORC_NU; ++a) {
                    double e = sqrt(sigma_u[a]) * nc[a];
                    if (m == 0) eps[((size_t)k * T + t) * ORC_NU + a] = e;
                    z[ORC_NX + a] = u_nom[(size_t)t * ORC_NU + a] + e;
                }
                double y[ORC_NY], var[ORC_NY];
                orc_lwpr_predict(P, z, y, var);
                cost[(size_t)k * T + t] += orc_running_cost(C, x, var) / (double)M;
                for (int a = 0; a < ORC_NX; ++a) {
                    double xdot = y[a];
                    if (model_noise) xdot += sqrt(var[a]) * nm[a];
                    x[a] = x[a] + P->dt * xdot;
                }
                if (xtraj) memcpy(xtraj + (((size_t)k * M + m) * (T + 1) + t + 1) * ORC_NX, x, sizeof(x));
            }
            phi[k] += orc_terminal_cost(C, x) / (double)M;
        }
    }
}

void orc_rollouts(const orc_lwpr *P, const orc_cost *C, const double *x0, const double *u_nom,
                  int K, int T, int M, const double *sigma_u, uint64_t seed, int model_noise,
                  double *eps, double *cost, double *phi, double *xtraj)
{
    orc_rollouts_from(P, C, x0, u_nom, 0, K, T, M, sigma_u, seed, model_noise, eps, cost, phi, xtraj);
}

/* Cost-to-go S(tau_i) = phi + sum_{j=i}^{T-1} q_j dt, accumulated from the end. */
void orc_cost_to_go(const double *cost, const double *phi, int K, int T, double dt, double *S)
{
    for (int k = 0; k < K; ++k) {
        double acc = phi[k];
        for (int i = T - 1; i >= 0; --i) {
            acc += cost[(size_t)k * T + i] * dt;
            S[(size_t)k * T + i] = acc;
        }
    }
}

/* Eq. 2 per timestep i: P_k = exp(-S_k/lambda) / sum_k exp(-S_k/lambda),
 * evaluated with the minimum over k subtracted, and
 * u_out_i = u_nom_i + sum_k P_k eps_{k,i}.  Sums run in k order. */
void orc_weighted_update(const double *S, const double *eps, const double *u_nom, int K, int T,
                         double lambda, double *u_out)
{
    for (int i = 0; i < T; ++i) {
        double smin = S[i];
        for (int k = 1; k < K; ++k) if (S[(size_t)k * T + i] < smin) smin = S[(size_t)k * T + i];
        double Z = 0.0, v[ORC_NU] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < K; ++k) {
            double w = exp(-(S[(size_t)k * T + i] - smin) / lambda);
            Z += w;
            for (int a = 0; a < ORC_NU; ++a) v[a] += w * eps[((size_t)k * T + i) * ORC_NU + a];
        }
        for (int a = 0; a < ORC_NU; ++a) u_out[(size_t)i * ORC_NU + a] = u_nom[(size_t)i * ORC_NU + a] + v[a] / Z;
    }
}

/* One full control update: rollouts -> cost-to-go -> weighted average.
 * costs_out[k] = S_{k,0}.  Scratch is allocated here (the oracle is not a
 * performance path). Returns 0, or -1 on allocation failure. */
int orc_pi_update(const orc_lwpr *P, const orc_cost *C, const double *x0, const double *u_nom,
                  int K, int T, int M, double lambda, const double *sigma_u, uint64_t seed,
                  int model_noise, double *u_out, double *costs_out)
{
    double *eps = (double *)malloc(sizeof(double) * (size_t)K * T * ORC_NU);
    double *cost = (double *)malloc(sizeof(double) * (size_t)K * T);
    double *phi = (double *)malloc(sizeof(double) * (size_t)K);
    double *S = (double *)malloc(sizeof(double) * (size_t)K * T);
    if (!eps || !cost || !phi || !S) { free(eps); free(cost); free(phi); free(S); return -1; }
    orc_rollouts(P, C, x0, u_nom, K, T, M, sigma_u, seed, model_noise, eps, cost, phi, NULL);
    orc_cost_to_go(cost, phi, K, T, P->dt, S);
    orc_weighted_update(S, eps, u_nom, K, T, lambda, u_out);
    for (int k = 0; k < K; ++k) costs_out[k] = S[(size_t)k * T];
    free(eps); free(cost); free(phi); free(S);
    return 0;
}

/* Threads the rollout loop may use (reported beside the CPU timing). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the threads of the rollout loop (the single-thread CPU timing). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

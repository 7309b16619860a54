"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-run the oracle's own formula: each compares it with an
independent computation (cuRAND's Philox compiled from its header, 50-digit
``decimal`` brute force of Eq. 1 and Eq. 2, closed forms of special cases,
exact rational sums, distributional tests), chosen so that a dropped term, a
wrong sign or factor, or a swapped index in the oracle fails one of them.
"""
import ctypes
import os
import subprocess
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats
from scipy.special import expit

from paper_1503_00330_b300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
getcontext().prec = 50


# ---------------------------------------------------------------------------
# Philox4x32-10 vs cuRAND's implementation (header compiled for the host)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def curand_philox(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("curand") / "cph.so")
    subprocess.run(["nvcc", "-O2", "-Xcompiler", "-fPIC", "-shared",
                    os.path.join(HERE, "curand_philox_host.cu"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.curand_philox_blocks.argtypes = [p, p, p, ctypes.c_int]

    def run(ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32)
        key = np.ascontiguousarray(key, np.uint32)
        out = np.zeros_like(ctr)
        lib.curand_philox_blocks(ctr.ctypes.data_as(p), key.ctypes.data_as(p),
                                 out.ctypes.data_as(p), ctr.shape[0])
        return out
    return run


def test_philox_matches_curand(oracle, curand_philox):
    g = np.random.default_rng(11)
    ctr = g.integers(0, 2**32, (300, 4), dtype=np.uint64).astype(np.uint32)
    key = g.integers(0, 2**32, (300, 2), dtype=np.uint64).astype(np.uint32)
    # include structured counters as used by the kernels: (k, t, blk, m)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 2, 0], [8191, 99, 3, 31]]
    key[:4] = [[0, 0], [0, 0], [7, 0], [0xffffffff, 0xffffffff]]
    ref = curand_philox(ctr, key)
    mine = np.stack([oracle.philox(c, k) for c, k in zip(ctr, key)])
    assert np.array_equal(mine, ref)


def test_noise_raw_counter_layout(oracle):
    """Block (k, t, blk, m) is Philox of counter (k, t, blk, m) under key (seed lo, seed hi)."""
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    raw = oracle.noise_raw(seed, 3, 4, m=5)
    for k in range(3):
        for t in range(4):
            for blk in range(4):
                m = 0 if blk == 0 else 5
                assert np.array_equal(raw[k, t, blk], oracle.philox([k, t, blk, m], key))


def test_uniforms_exact_and_open_interval(oracle):
    for r in [0, 1, 511, 512, 2**31, 2**32 - 1, 123456789]:
        u = oracle.uniform(r)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u          # exactly representable in FP32
        assert u == (2 * (r >> 9) + 1) / 2**24


def test_normals_distribution(oracle):
    n = []
    for k in range(2500):
        for t in range(4):
            nc, nm = oracle.normals(1234, k, t, 0)
            n.append(np.concatenate([nc, nm]))
    n = np.array(n)                                # [10000, 16]
    flat = n.ravel()
    N = flat.size
    assert abs(flat.mean()) < 5 / np.sqrt(N)
    assert abs(flat.var() - 1.0) < 5 * np.sqrt(2.0 / N)
    assert abs(stats.kurtosis(flat, fisher=False) - 3.0) < 5 * np.sqrt(24.0 / N)
    assert stats.kstest(flat, "norm").pvalue > 1e-4
    c = np.corrcoef(n.T)
    assert np.max(np.abs(c - np.eye(16))) < 5 / np.sqrt(n.shape[0])


def test_normals_box_muller_mapping(oracle):
    """Block 0 -> control normals, blocks 1..3 -> model normals, pairs (u0,u1),(u2,u3)."""
    seed = 99
    raw = oracle.noise_raw(seed, 2, 3, m=2)
    for k in range(2):
        for t in range(3):
            nc, nm = oracle.normals(seed, k, t, 2)
            allz = np.concatenate([nc, nm])
            for blk in range(4):
                u = (2 * (raw[k, t, blk].astype(np.int64) >> 9) + 1) / 2**24
                r0, r1 = np.sqrt(-2 * np.log(u[0])), np.sqrt(-2 * np.log(u[2]))
                ref = [r0 * np.cos(2 * np.pi * u[1]), r0 * np.sin(2 * np.pi * u[1]),
                       r1 * np.cos(2 * np.pi * u[3]), r1 * np.sin(2 * np.pi * u[3])]
                np.testing.assert_allclose(allz[4 * blk:4 * blk + 4], ref, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# Eq. 1: LWPR prediction
# ---------------------------------------------------------------------------
def _dec_lwpr(model, z):
    """50-digit brute force of Eq. 1 with the unshifted exponentials."""
    L = model.L
    ys, vs = [], []
    for o in range(12):
        es, yl, sg = [], [], []
        for j in range(L):
            d = [Decimal(float(z[a])) - Decimal(float(model.c[o, j, a])) for a in range(16)]
            q = sum(d[a] * Decimal(float(model.D[o, j, a, b])) * d[b]
                    for a in range(16) for b in range(16))
            es.append((-q / 2).exp())
            yl.append(Decimal(float(model.b[o, j])) +
                      sum(Decimal(float(model.beta[o, j, a])) * d[a] for a in range(16)))
            sg.append(Decimal(float(model.sigma[o, j])))
        tot = sum(es)
        w = [e / tot for e in es]
        y = sum(wj * yj for wj, yj in zip(w, yl))
        v = sum(wj * ((y - yj) ** 2 + s ** 2) for wj, yj, s in zip(w, yl, sg))
        ys.append(float(y))
        vs.append(float(v))
    return np.array(ys), np.array(vs)


def _scaled_model(L, seed, scale=0.3):
    m = W.make_lwpr(L, seed)
    # keep exponents moderate so the unshifted brute force is well conditioned
    m.D = (m.D * np.float32(scale)).astype(np.float32)
    return m


@pytest.mark.parametrize("L,seed", [(1, 0), (2, 1), (3, 2)])
def test_lwpr_decimal_bruteforce(oracle, L, seed):
    m = _scaled_model(L, seed)
    g = np.random.default_rng(seed + 100)
    for _ in range(3):
        z = g.normal(0, 0.7, 16).astype(np.float32)
        y, v = oracle.lwpr_predict(m, z)
        yd, vd = _dec_lwpr(m, z)
        np.testing.assert_allclose(y[0], yd, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(v[0], vd, rtol=1e-11, atol=1e-14)


def test_lwpr_L1_closed_form(oracle):
    m = W.make_lwpr(1, 5)
    z = np.random.default_rng(0).normal(0, 1, 16).astype(np.float32)
    y, v = oracle.lwpr_predict(m, z)
    c, beta = m.c[:, 0].astype(np.float64), m.beta[:, 0].astype(np.float64)
    yref = m.b[:, 0].astype(np.float64) + np.einsum("oa,oa->o", beta, z.astype(np.float64) - c)
    np.testing.assert_allclose(y[0], yref, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(v[0], m.sigma[:, 0].astype(np.float64) ** 2, rtol=1e-14)


def test_lwpr_L2_logistic_weights(oracle):
    """With two fields the normalized weight of field 1 is expit((q2 - q1) / 2)."""
    m = W.make_lwpr(2, 9)
    m.beta[:] = 0.0
    m.sigma[:] = 0.0
    m.b[:, 0], m.b[:, 1] = 1.0, 0.0               # y = w_1 exactly
    z = np.random.default_rng(1).normal(0, 0.5, 16)
    y, v = oracle.lwpr_predict(m, z.astype(np.float32))
    zz = z.astype(np.float32).astype(np.float64)
    for o in range(12):
        q = []
        for j in range(2):
            d = zz - m.c[o, j].astype(np.float64)
            q.append(d @ m.D[o, j].astype(np.float64) @ d)
        w1 = expit((q[1] - q[0]) / 2)
        assert abs(y[0, o] - w1) < 1e-14
        assert abs(v[0, o] - w1 * (1 - w1)) < 1e-14  # Bernoulli spread of y_j in {1, 0}


def test_lwpr_weights_sum_to_one(oracle):
    m = W.make_lwpr(64, 3)
    m.beta[:] = 0.0
    m.b[:] = 1.0
    m.sigma[:] = 0.0
    z = np.random.default_rng(2).normal(0, 1, (5, 16)).astype(np.float32)
    y, v = oracle.lwpr_predict(m, z)
    np.testing.assert_allclose(y, 1.0, rtol=0, atol=64 * 2.3e-16)
    np.testing.assert_allclose(v, 0.0, rtol=0, atol=1e-28)


def test_lwpr_zero_metric_uniform_weights(oracle):
    """D = 0 makes every weight 1/L: y is the plain mean of the local models."""
    m = W.make_lwpr(7, 4)
    m.D[:] = 0.0
    z = np.random.default_rng(3).normal(0, 1, 16).astype(np.float32)
    y, v = oracle.lwpr_predict(m, z)
    zz = z.astype(np.float64)
    yl = m.b.astype(np.float64) + np.einsum("oja,oja->oj", m.beta.astype(np.float64),
                                            zz[None, None, :] - m.c.astype(np.float64))
    np.testing.assert_allclose(y[0], yl.mean(1), rtol=1e-13, atol=1e-14)
    vref = yl.var(1) + (m.sigma.astype(np.float64) ** 2).mean(1)
    np.testing.assert_allclose(v[0], vref, rtol=1e-12)


def test_lwpr_duplicate_and_permuted_fields(oracle):
    m = W.make_lwpr(5, 6)
    z = np.random.default_rng(4).normal(0, 0.5, (3, 16)).astype(np.float32)
    y, v = oracle.lwpr_predict(m, z)
    dup = W.LwprModel(*(np.concatenate([a, a], axis=1) for a in (m.c, m.D, m.beta, m.b, m.sigma)), dt=m.dt)
    y2, v2 = oracle.lwpr_predict(dup, z)
    np.testing.assert_allclose(y2, y, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(v2, v, rtol=1e-12, atol=1e-14)
    perm = np.random.default_rng(5).permutation(5)
    pm = W.LwprModel(*(a[:, perm] for a in (m.c, m.D, m.beta, m.b, m.sigma)), dt=m.dt)
    y3, v3 = oracle.lwpr_predict(pm, z)
    np.testing.assert_allclose(y3, y, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(v3, v, rtol=1e-12, atol=1e-14)


def test_lwpr_far_input_no_underflow(oracle):
    """Far from every center exp(-q/2) underflows in any float format; the
    normalized weights are still defined (the largest one dominates)."""
    m = W.make_lwpr(3, 7)
    z = np.full(16, 30.0, np.float32)
    y, v = oracle.lwpr_predict(m, z)
    assert np.all(np.isfinite(y)) and np.all(np.isfinite(v)) and np.all(v > 0)


# ---------------------------------------------------------------------------
# Sec. 5 cost
# ---------------------------------------------------------------------------
def _cost(**kw):
    base = dict(goal=(1.0, -2.0, 0.5), Q_pos=(1.0, 2.0, 3.0), w_obs=1000.0, radius=0.5,
                w_var=0.0, w_T=2.0, obs_xy=np.array([[0.0, 0.0], [5.0, 5.0]], np.float32))
    base.update(kw)
    return W.CostParams(**base).rounded()


def test_cost_closed_forms(oracle):
    cp = _cost()
    x = np.zeros(12)
    x[:3] = [2.0, -1.0, 1.5]                       # offsets (1, 1, 1) from the goal
    assert oracle.running_cost(cp, x, np.zeros(12)) == 1 + 2 + 3
    assert oracle.terminal_cost(cp, x) == 2.0 * (1 + 2 + 3)
    # variance penalty
    cp2 = _cost(w_var=0.5)
    assert oracle.running_cost(cp2, x, np.arange(12.0)) == 6 + 0.5 * 66
    # inside the first cylinder
    xin = np.zeros(12)
    xin[:3] = [0.1, 0.2, 7.0]
    base = 1 * (0.1 - 1) ** 2 + 2 * (0.2 + 2) ** 2 + 3 * (7.0 - 0.5) ** 2
    assert abs(oracle.running_cost(cp, xin, np.zeros(12)) - (base + 1000.0)) < 1e-9
    # velocity and angle weights
    cp3 = _cost(Q_vel=0.25, Q_ang=4.0)
    xv = x.copy()
    xv[3:6] = [1, 2, 2]
    xv[6:9] = [0.5, 0, 0]
    assert abs(oracle.running_cost(cp3, xv, np.zeros(12)) - (6 + 0.25 * 9 + 4.0 * 0.25)) < 1e-12


def test_cost_boundary_is_outside(oracle):
    cp = _cost()
    assert oracle.inside_any(cp, 0.5, 0.0) == 0    # d^2 == r^2 exactly: outside
    assert oracle.inside_any(cp, 0.0, -0.5) == 0
    assert oracle.inside_any(cp, 0.4999, 0.0) == 1
    assert oracle.inside_any(cp, 5.3, 5.3) == 1
    assert oracle.inside_any(cp, 2.0, 2.0) == 0


def test_cost_indicator_is_decided_on_the_fp64_state(oracle):
    """Sec. 5's crash indicator is a property of the real position: points 1e-12
    inside and outside the boundary of radius 0.3 (0.3 rounded to FP32, as the
    kernels receive it) are told apart.  Both round to the same FP32 position,
    so an indicator taken in FP32 would give them the same answer."""
    cp = _cost(radius=0.3)
    r = float(np.float32(0.3))
    assert np.float32(r * (1 - 1e-12)) == np.float32(r * (1 + 1e-12))
    assert oracle.inside_any(cp, r * (1 - 1e-12), 0.0) == 1
    assert oracle.inside_any(cp, r * (1 + 1e-12), 0.0) == 0
    assert oracle.inside_any(cp, 0.0, -r * (1 - 1e-12)) == 1
    d = r / np.sqrt(2.0) * (1 - 1e-12)                # off the axes as well
    assert oracle.inside_any(cp, d, d) == 1


def test_cost_gaussian_bumps(oracle):
    """The paper's obstacle term 100 sum_i exp(-10 (dx^2 + dy^2)) plus 10 C."""
    cp = W.CostParams(goal=(0, 0, 0), Q_pos=(0, 0, 0), w_obs=100.0, obs_sharp=10.0, radius=0.3,
                      w_crash=10.0, w_var=0.0, w_T=0.0, obs_kind=1,
                      obs_xy=np.array([[0.0, 0.0], [1.0, 0.0]], np.float32)).rounded()
    x = np.zeros(12)
    x[0] = 0.5
    ref = 100 * (np.exp(-10 * 0.25) + np.exp(-10 * 0.25))
    assert abs(oracle.running_cost(cp, x, np.zeros(12)) - ref) < 1e-12
    x[0] = 0.1
    ref = 100 * (np.exp(-10 * 0.01) + np.exp(-10 * 0.81)) + 10
    assert abs(oracle.running_cost(cp, x, np.zeros(12)) - ref) < 1e-9


# ---------------------------------------------------------------------------
# Rollouts: Euler steps, noise placement, sub-rollouts
# ---------------------------------------------------------------------------
def _linear_problem(seed=0, T=12, K=3, sigma=0.0):
    p = W.problem(K, T, 1, seed=seed, n_obs=2)
    p.model.sigma[:] = np.float32(sigma)
    p.u_nom = np.random.default_rng(seed).normal(0, 0.2, (T, 4)).astype(np.float32)
    p.x0 = np.random.default_rng(seed + 1).normal(0, 0.3, 12).astype(np.float32)
    return p


def test_rollout_L1_linear_closed_form(oracle):
    """L = 1 and sigma = 0: x_{t+1} = (I + dt B_x) x_t + dt (b - B c + B_u u_t), so
    x_T = A^T x0 + dt sum_t A^(T-1-t) (g + B_u u_t)."""
    p = _linear_problem()
    sig0 = np.zeros(4, np.float32)
    r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, sig0, p.seed, want_traj=True)
    dt = float(p.model.dt)
    beta = p.model.beta[:, 0].astype(np.float64)
    Bx, Bu = beta[:, :12], beta[:, 12:]
    g = p.model.b[:, 0].astype(np.float64) - np.einsum("oa,oa->o", beta, p.model.c[:, 0].astype(np.float64))
    A = np.eye(12) + dt * Bx
    for T in (1, 5, p.T):
        xT = np.linalg.matrix_power(A, T) @ p.x0.astype(np.float64)
        for t in range(T):
            xT += dt * np.linalg.matrix_power(A, T - 1 - t) @ (g + Bu @ p.u_nom[t].astype(np.float64))
        for k in range(p.K):
            np.testing.assert_allclose(r["traj"][k, 0, T], xT, rtol=1e-11, atol=1e-13)
    assert np.all(r["eps"] == 0.0)


def test_rollout_noise_enters_as_dt_sigma_n(oracle):
    """L = 1 with sigma_j > 0: the sampled step adds dt * sigma * n_model (Sec. 3.2,
    Euler), and the perturbation is sqrt(Sigma_u) * n_ctrl."""
    p = _linear_problem(sigma=0.05, T=6, K=2)
    r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, want_traj=True)
    dt = float(p.model.dt)
    beta = p.model.beta[:, 0].astype(np.float64)
    A = np.eye(12) + dt * beta[:, :12]
    g = p.model.b[:, 0].astype(np.float64) - np.einsum("oa,oa->o", beta, p.model.c[:, 0].astype(np.float64))
    sd = float(np.float32(0.05))
    for k in range(p.K):
        x = p.x0.astype(np.float64)
        for t in range(p.T):
            nc, nm = oracle.normals(p.seed, k, t, 0)
            eps = np.sqrt(p.sigma_u.astype(np.float64)) * nc
            np.testing.assert_allclose(r["eps"][k, t], eps, rtol=1e-14, atol=1e-16)
            u = p.u_nom[t].astype(np.float64) + eps
            x = A @ x + dt * (g + beta[:, 12:] @ u) + dt * sd * nm
            np.testing.assert_allclose(r["traj"][k, 0, t + 1], x, rtol=1e-11, atol=1e-13)


def test_rollout_zero_noise_all_equal_nominal(oracle):
    p = W.problem(6, 10, 8, seed=3)
    z4 = np.zeros(4, np.float32)
    r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, z4, p.seed, model_noise=False,
                        want_traj=True)
    for k in range(1, p.K):
        assert np.array_equal(r["traj"][k], r["traj"][0])
        assert np.array_equal(r["cost"][k], r["cost"][0])
    u, c = oracle.pi_update(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.lam, z4, p.seed,
                            model_noise=False)
    assert np.array_equal(u, p.u_nom.astype(np.float64))
    assert np.all(c == c[0])


def test_rollout_cost_indexing(oracle):
    """cost[k, t] = q(x_t, var(z_t)) for t = 0..T-1 and phi = phi(x_T) (Sec. 3.1)."""
    p = W.problem(2, 7, 4, seed=8, n_obs=3)
    r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, want_traj=True)
    for k in range(p.K):
        for t in range(p.T):
            x = r["traj"][k, 0, t]
            z = np.concatenate([x, p.u_nom[t] + r["eps"][k, t]])
            _, var = oracle.lwpr_predict(p.model, z)
            assert abs(r["cost"][k, t] - oracle.running_cost(p.cost, x, var[0])) < 1e-12
        assert abs(r["phi"][k] - oracle.terminal_cost(p.cost, r["traj"][k, 0, p.T])) < 1e-12


def test_subrollouts_average(oracle):
    """Sec. 3.2: M sub-rollouts share the control perturbation; sub-rollout 0 is the
    M = 1 rollout, and the rollout cost is the mean over the sub-rollouts."""
    p = W.problem(3, 8, 6, seed=2)
    r1 = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, M=1, want_traj=True)
    r4 = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, M=4, want_traj=True)
    assert np.array_equal(r4["traj"][:, 0], r1["traj"][:, 0])
    assert np.array_equal(r4["eps"], r1["eps"])
    assert not np.array_equal(r4["traj"][:, 1], r4["traj"][:, 0])
    for k in range(p.K):
        for t in range(p.T):
            qs = []
            for m in range(4):
                x = r4["traj"][k, m, t]
                z = np.concatenate([x, p.u_nom[t] + r4["eps"][k, t]])
                _, var = oracle.lwpr_predict(p.model, z)
                qs.append(oracle.running_cost(p.cost, x, var[0]))
            assert abs(r4["cost"][k, t] - np.mean(qs)) < 1e-11
    # mean-only prediction: sub-rollouts coincide, so M changes nothing
    a = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, M=1, model_noise=False)
    b = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, M=4, model_noise=False)
    np.testing.assert_allclose(b["cost"], a["cost"], rtol=1e-15)


# ---------------------------------------------------------------------------
# Cost-to-go and Eq. 2
# ---------------------------------------------------------------------------
def test_cost_to_go_exact_sum(oracle):
    g = np.random.default_rng(0)
    K, T = 4, 9
    cost = g.uniform(0, 50, (K, T))
    phi = g.uniform(0, 5, K)
    dt = 0.02
    S = oracle.cost_to_go(cost, phi, dt)
    for k in range(K):
        for i in range(T):
            exact = Fraction(phi[k]) + sum(Fraction(cost[k, j]) * Fraction(dt) for j in range(i, T))
            assert abs(Fraction(S[k, i]) - exact) <= abs(exact) * Fraction(1, 10**14)
    S1 = oracle.cost_to_go(cost[:, :1], phi, dt)
    np.testing.assert_array_equal(S1[:, 0], phi + cost[:, 0] * dt)


def _dec_update(S, eps, u_nom, lam):
    K, T = S.shape
    out = np.zeros((T, 4))
    for i in range(T):
        w = [(-Decimal(float(S[k, i])) / Decimal(float(lam))).exp() for k in range(K)]
        Z = sum(w)
        for a in range(4):
            out[i, a] = float(u_nom[i, a]) + float(sum(wk * Decimal(float(eps[k, i, a])) for k, wk in enumerate(w)) / Z)
    return out


def test_weighted_update_decimal_bruteforce(oracle):
    g = np.random.default_rng(1)
    K, T = 5, 4
    S = g.uniform(0, 8, (K, T))
    eps = g.normal(0, 0.3, (K, T, 4))
    u_nom = g.normal(0, 1, (T, 4))
    for lam in (0.5, 1.0, 7.0):
        np.testing.assert_allclose(oracle.weighted_update(S, eps, u_nom, lam),
                                   _dec_update(S, eps, u_nom, lam), rtol=1e-13, atol=1e-14)


def test_weighted_update_limits(oracle):
    g = np.random.default_rng(2)
    K, T = 16, 5
    S = g.uniform(10, 20, (K, T))
    eps = g.normal(0, 0.3, (K, T, 4))
    u_nom = g.normal(0, 1, (T, 4))
    # lambda -> infinity: plain mean of the perturbations
    np.testing.assert_allclose(oracle.weighted_update(S, eps, u_nom, 1e30), u_nom + eps.mean(0),
                               rtol=1e-13, atol=1e-14)
    # lambda -> 0: the arg-min rollout's perturbation
    am = S.argmin(0)
    ref = u_nom + eps[am, np.arange(T)]
    np.testing.assert_allclose(oracle.weighted_update(S, eps, u_nom, 1e-9), ref, rtol=1e-13, atol=1e-14)
    # exact ties at the minimum share the weight
    S2 = S.copy()
    S2[3] = S2.min(0) - 1.0
    S2[7] = S2[3]
    np.testing.assert_allclose(oracle.weighted_update(S2, eps, u_nom, 1e-9),
                               u_nom + 0.5 * (eps[3] + eps[7]), rtol=1e-13, atol=1e-14)
    # a constant added to every cost-to-go changes nothing
    np.testing.assert_allclose(oracle.weighted_update(S + 1234.5, eps, u_nom, 1.0),
                               oracle.weighted_update(S, eps, u_nom, 1.0), rtol=1e-11, atol=1e-12)
    # K = 2: weight of rollout 0 is expit((S1 - S0)/lambda)
    w0 = expit((S[1] - S[0]) / 2.0)
    ref = u_nom + w0[:, None] * eps[0] + (1 - w0)[:, None] * eps[1]
    np.testing.assert_allclose(oracle.weighted_update(S[:2], eps[:2], u_nom, 2.0), ref, rtol=1e-13, atol=1e-14)


def test_pi_update_zero_cost_uniform_weights(oracle):
    """Every cost zero: Eq. 2 gives uniform weights, so u_out = u_nom + mean_k eps."""
    p2 = W.problem(16, 6, 4, seed=4)
    p2.cost.w_obs = 0.0
    p2.cost.w_var = 0.0
    p2.cost.Q_pos = (0.0, 0.0, 0.0)                 # every cost is 0: uniform weights
    u, c = oracle.pi_update(p2.model, p2.cost, p2.x0, p2.u_nom, p2.K, p2.T, p2.lam, p2.sigma_u, p2.seed)
    r = oracle.rollouts(p2.model, p2.cost, p2.x0, p2.u_nom, p2.K, p2.T, p2.sigma_u, p2.seed)
    np.testing.assert_allclose(u, p2.u_nom + r["eps"].mean(0), rtol=1e-13, atol=1e-15)
    assert np.all(c == 0.0)


def test_golden_tiny_update(oracle):
    """Regression of the oracle against the stored tiny case (written by
    tests/golden/make_golden.py, which calls only the oracle)."""
    import json
    with open(os.path.join(HERE, "golden", "tiny_update.json")) as f:
        gold = json.load(f)
    p = W.problem(gold["K"], gold["T"], gold["L"], seed=gold["seed"], n_obs=gold["n_obs"])
    u, c = oracle.pi_update(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    np.testing.assert_allclose(u, np.array(gold["u_out"]), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(c, np.array(gold["costs_out"]), rtol=1e-12)


def test_update_converges_as_inverse_sqrt_K(oracle):
    """Eq. 2 is a self-normalised Monte Carlo estimate over K rollouts: its
    error against the large-K limit shrinks like K^(-1/2).  The reference is
    one update with K = 65536; the error at K = 64 ... 4096 is the RMS over 8
    independent seeds; the fitted log-log slope must be -1/2 within 0.15.
    Noise shared between rollouts would break the rate; weights that ignored
    the costs would put the limit at u_nom + E[eps] = 0."""
    p = W.problem(16, 6, 2, seed=9, n_obs=2)
    p.u_nom = np.zeros((p.T, 4), np.float32)
    lam = 0.5
    ref, _ = oracle.pi_update(p.model, p.cost, p.x0, p.u_nom, 65536, p.T, lam, p.sigma_u, 10_000)
    Ks = [64, 256, 1024, 4096]
    rms = []
    for K in Ks:
        errs = [oracle.pi_update(p.model, p.cost, p.x0, p.u_nom, K, p.T, lam, p.sigma_u, 100 + s)[0] - ref
                for s in range(8)]
        rms.append(np.sqrt(np.mean(np.square(errs))))
    slope = np.polyfit(np.log(Ks), np.log(rms), 1)[0]
    assert -0.65 <= slope <= -0.35, (rms, slope)
    # the limit is not u_nom + E[eps] = 0: the costs move it by many standard
    # errors of the K = 65536 reference (about rms(4096) * sqrt(4096 / 65536))
    assert np.abs(ref).max() > 5 * rms[-1] * np.sqrt(4096 / 65536)

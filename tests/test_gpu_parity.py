"""GPU parity: every stage of the CUDA path, called through the C ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances (FP32 kernels vs FP64 oracle):
  * Philox raw blocks: bit-exact.
  * normals: |dn| <= 4e-6 (1 + |n|)  (FP32 log / sqrt / sincospi of exact uniforms).
  * LWPR mean/variance: |dy| <= 2e-5 (1 + |y|), |dvar| <= 2e-5 var + 1e-6.  FP32
    rounding of the exponent s_j = -q_j/2 is about 1e-7 |q_j| with q_j up to ~100,
    i.e. ~1e-5 absolute in a weight's log, which moves y by ~1e-5 of the spread
    of the local predictions (O(1)).
  * u_out (end to end): max_{t,c} |du| / scale_c <= 1e-5 per channel, the FP32
    target of the method's accuracy contract, with scale_c = max_t |u_ref[., c]|
    floored at sqrt(Sigma_u,c / K), the standard error of the mean perturbation
    (with T = 1 a single |u_ref| can sit arbitrarily close to 0).
  * costs_out: max_k |dS_k| / S_k <= 1e-5.
"""
import numpy as np
import pytest
import torch

from paper_1503_00330_b300 import workloads as W

pytestmark = pytest.mark.gpu

U_TOL = 1e-5
S_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    build.build()


def _ctrl(p, **kw):
    from paper_1503_00330_b300.api import Controller
    return Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, **kw)


def _u_err(u, ref, sigma_u=None, K=None):
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max(axis=0)
    if sigma_u is not None:
        scale = np.maximum(scale, np.sqrt(np.asarray(sigma_u, np.float64) / K))
    return np.abs(u - ref).max(axis=0) / np.maximum(scale, 1e-30)


def _oracle_update(oracle, p):
    return oracle.pi_update(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed,
                            M=p.M, model_noise=p.model_noise)


# ---------------------------------------------------------------------------
# noise
# ---------------------------------------------------------------------------
def test_noise_raw_bit_exact(oracle):
    from paper_1503_00330_b300.api import debug_noise
    seed = 0x9E3779B97F4A7C15
    raw = debug_noise(seed, 37, 11, m=5).cpu().numpy().view(np.uint32)
    ref = oracle.noise_raw(seed, 37, 11, m=5)
    assert np.array_equal(raw, ref)


def test_normals_fp32(oracle):
    from paper_1503_00330_b300.api import debug_normals
    seed = 12345
    K, T, m = 40, 9, 2
    c, mo = debug_normals(seed, K, T, m)
    c, mo = c.cpu().numpy(), mo.cpu().numpy()
    worst = 0.0
    for k in range(K):
        for t in range(T):
            nc, nm = oracle.normals(seed, k, t, m)
            d = np.abs(np.concatenate([c[k, t], mo[k, t]]) - np.concatenate([nc, nm]))
            worst = max(worst, float(np.max(d / (1 + np.abs(np.concatenate([nc, nm]))))))
    print("normals worst", worst)
    assert worst <= 4e-6


# ---------------------------------------------------------------------------
# LWPR prediction (Eq. 1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,n", [(1, 5), (3, 70), (17, 130), (64, 200), (255, 65), (700, 40), (1025, 9)])
def test_lwpr_predict(oracle, L, n):
    """L = 700 and 1025 give 350 and 513 field pairs: two and three rounds of the
    prediction kernel's 256 threads, with the records reloaded for the second pass."""
    p = W.problem(8, 4, L, seed=L)
    ctl = _ctrl(p)
    g = np.random.default_rng(L)
    z = np.concatenate([g.normal(0, 0.5, (n, 12)), g.normal(0, 0.3, (n, 4))], 1).astype(np.float32)
    y, v = ctl.debug_lwpr(z)
    torch.cuda.synchronize()
    ctl.sync()
    y, v = y.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    yr, vr = oracle.lwpr_predict(p.model, z)
    ey = np.max(np.abs(y - yr) / (1 + np.abs(yr)))
    ev = np.max(np.abs(v - vr) / (vr + 1e-6 / 2e-5))
    print(f"L={L} n={n} y err {ey:.3g} var err {ev:.3g}")
    assert ey <= 2e-5
    assert np.all(np.abs(v - vr) <= 2e-5 * vr + 1e-6)


# ---------------------------------------------------------------------------
# reduction stage (cost-to-go + Eq. 2) on oracle-made inputs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K,T,lam", [(1, 1, 1.0), (64, 50, 1.0), (100, 33, 0.3), (777, 150, 5.0),
                                     (4096, 7, 1.0)])
def test_reduce_stage(oracle, K, T, lam):
    g = np.random.default_rng(K + T)
    cost = g.uniform(0, 40, (K, T)).astype(np.float32)
    cost[g.random((K, T)) < 0.05] += np.float32(1000.0)        # obstacle hits
    phi = g.uniform(0, 10, K).astype(np.float32)
    eps = g.normal(0, 0.3, (K, T, 4)).astype(np.float32)
    u_nom = g.normal(0, 0.5, (T, 4)).astype(np.float32)
    p = W.problem(8, 4, 2, seed=0)
    ctl = _ctrl(p)
    u, c = ctl.debug_reduce(cost.T.copy(), phi, np.transpose(eps, (1, 0, 2)).copy(), u_nom, lam)
    ctl.sync()
    dt = float(p.model.dt)
    S = oracle.cost_to_go(cost, phi, dt)
    uref = oracle.weighted_update(S, eps, u_nom, lam)
    eu = _u_err(u.cpu().numpy(), uref)
    ec = np.max(np.abs(c.cpu().numpy() - S[:, 0]) / np.abs(S[:, 0]))
    print(f"K={K} T={T} u err {eu} cost err {ec:.3g}")
    assert np.all(eu <= U_TOL)
    assert ec <= 1e-6


def test_reduce_stage_negative_costs(oracle):
    """Costs of either sign (a cost with negative weights): the exact minimum over
    the rollouts is taken on order-preserving integer keys of the doubles, whose
    negative branch this exercises (S spans zero)."""
    K, T, lam = 333, 40, 0.7
    g = np.random.default_rng(5)
    cost = g.uniform(-40, 40, (K, T)).astype(np.float32)
    phi = g.uniform(-10, 10, K).astype(np.float32)
    eps = g.normal(0, 0.3, (K, T, 4)).astype(np.float32)
    u_nom = g.normal(0, 0.5, (T, 4)).astype(np.float32)
    p = W.problem(8, 4, 2, seed=0)
    ctl = _ctrl(p)
    u, c = ctl.debug_reduce(cost.T.copy(), phi, np.transpose(eps, (1, 0, 2)).copy(), u_nom, lam)
    ctl.sync()
    S = oracle.cost_to_go(cost, phi, float(p.model.dt))
    assert S.min() < 0 < S.max()
    uref = oracle.weighted_update(S, eps, u_nom, lam)
    assert np.all(_u_err(u.cpu().numpy(), uref) <= U_TOL)
    assert np.max(np.abs(c.cpu().numpy() - S[:, 0]) / (np.abs(S[:, 0]) + 1.0)) <= 1e-6


def test_pipe_rate_probes():
    """The measured pipe rates behind the rooflines are positive and of the size a
    B300 can have (FFMA2 10-200 TFLOP/s, MUFU ex2 1e11-1e14/s, DFMA 1e10-1e13/s)."""
    from paper_1503_00330_b300.api import fp64_rate, pipe_rates
    r = pipe_rates(0)
    assert 10.0 < r["ffma_tflops"] < 200.0
    assert 1e11 < r["ex2_per_s"] < 1e14
    assert 1e10 < fp64_rate(0) < 1e13


def test_reduce_stage_large_costs_small_lambda(oracle):
    """Costs near 1e8 (cost-to-go near 1e8 too) with lambda = 0.01: the shift of the
    exponents must be the exact minimum, else exp2 over- or underflows; u_out is
    then essentially the argmin rollout's perturbation, as in the oracle."""
    K, T, lam = 300, 9, 0.01
    g = np.random.default_rng(77)
    cost = (1e8 + g.uniform(0, 2e3, (K, T))).astype(np.float32)
    phi = g.uniform(0, 10, K).astype(np.float32)
    eps = g.normal(0, 0.3, (K, T, 4)).astype(np.float32)
    u_nom = g.normal(0, 0.5, (T, 4)).astype(np.float32)
    p = W.problem(8, 4, 2, seed=0)
    ctl = _ctrl(p)
    u, c = ctl.debug_reduce(cost.T.copy(), phi, np.transpose(eps, (1, 0, 2)).copy(), u_nom, lam)
    ctl.sync()
    u = u.cpu().numpy()
    S = oracle.cost_to_go(cost, phi, float(p.model.dt))
    uref = oracle.weighted_update(S, eps, u_nom, lam)
    assert np.all(np.isfinite(u))
    assert np.all(_u_err(u, uref) <= U_TOL)


# ---------------------------------------------------------------------------
# rollout stage and end to end
# ---------------------------------------------------------------------------
def _rollout_compare(oracle, p):
    ctl = _ctrl(p)
    cost, eps, phi = ctl.debug_rollout(p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed)
    ctl.sync()
    r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, M=p.M,
                        model_noise=p.model_noise)
    cost = cost.cpu().numpy().T.astype(np.float64)
    eps = np.transpose(eps.cpu().numpy(), (1, 0, 2)).astype(np.float64)
    phi = phi.cpu().numpy().astype(np.float64)
    e_eps = np.max(np.abs(eps - r["eps"]) / (np.abs(r["eps"]) + 1e-3))
    # indicator flips: a step whose cost differs by about w_obs
    flips = int(np.sum(np.abs(cost - r["cost"]) > 0.5 * max(p.cost.w_obs, 1.0)))
    ok = np.abs(cost - r["cost"]) <= 0.5 * max(p.cost.w_obs, 1.0)
    e_cost = np.max(np.abs(cost - r["cost"])[ok] / (np.abs(r["cost"][ok]) + 1e-3))
    e_phi = np.max(np.abs(phi - r["phi"]) / (np.abs(r["phi"]) + 1e-3))
    return e_eps, e_cost, e_phi, flips


@pytest.mark.parametrize("K,T,L,M,noise", [(64, 20, 8, 1, True), (100, 13, 3, 1, True),
                                           (50, 9, 5, 4, True), (70, 6, 2, 1, False)])
def test_rollout_stage(oracle, K, T, L, M, noise):
    p = W.problem(K, T, L, seed=K + L, n_obs=6, M=M, model_noise=noise)
    e_eps, e_cost, e_phi, flips = _rollout_compare(oracle, p)
    print(f"K={K} T={T} L={L} M={M}: eps {e_eps:.3g} cost {e_cost:.3g} phi {e_phi:.3g} flips {flips}")
    assert e_eps <= 2e-6
    assert flips == 0
    assert e_cost <= 1e-4 and e_phi <= 1e-4


def test_end_to_end_small_workload(oracle):
    """K=256 rollouts, T=50 steps, L=64 fields per output, 4 obstacles."""
    p = W.small()
    ctl = _ctrl(p)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    uref, cref = _oracle_update(oracle, p)
    eu = _u_err(u.cpu().numpy(), uref)
    ec = np.max(np.abs(c.cpu().numpy() - cref) / cref)
    print("small workload: u_out rel err per channel", eu, "costs rel err", ec)
    assert np.all(eu <= U_TOL)
    assert ec <= S_TOL


@pytest.mark.parametrize("K,T,L,M,noise,kind", [(1, 1, 1, 1, True, 0), (65, 1, 2, 1, True, 0),
                                                (130, 17, 9, 2, True, 0), (33, 25, 16, 8, True, 1),
                                                (96, 30, 5, 1, False, 1)])
def test_end_to_end_ragged(oracle, K, T, L, M, noise, kind):
    cost = W.paper_cost(3, seed=K) if kind == 1 else None
    p = W.problem(K, T, L, seed=1000 + K, n_obs=5, M=M, model_noise=noise, cost=cost)
    ctl = _ctrl(p)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    uref, cref = _oracle_update(oracle, p)
    eu = _u_err(u.cpu().numpy(), uref, p.sigma_u, p.K)
    ec = np.max(np.abs(c.cpu().numpy() - cref) / np.maximum(cref, 1e-3))
    print(f"K={K} T={T} L={L} M={M}: u err {eu} cost err {ec:.3g}")
    assert np.all(eu <= U_TOL)
    assert ec <= S_TOL


def test_zero_noise_returns_nominal():
    p = W.problem(200, 12, 6, seed=5, model_noise=False)
    p.sigma_u = np.zeros(4, np.float32)
    p.u_nom = np.random.default_rng(0).normal(0, 0.3, (p.T, 4)).astype(np.float32)
    ctl = _ctrl(p)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    assert np.array_equal(u.cpu().numpy(), p.u_nom)
    cc = c.cpu().numpy()
    assert np.all(cc == cc[0])


def test_deterministic_and_host_path_agree():
    p = W.problem(300, 20, 10, seed=9)
    ctl = _ctrl(p)
    u1, c1 = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    u2, c2 = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    u3, c3 = ctl.update_host(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    assert torch.equal(u1, u2) and torch.equal(c1, c2)
    assert np.array_equal(u1.cpu().numpy(), u3) and np.array_equal(c1.cpu().numpy(), c3)
    u4, _ = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed + 1)
    assert not torch.equal(u1, u4)


def test_update_composes_stages():
    """pi_update equals the rollout stage followed by the reduction stage."""
    p = W.problem(500, 15, 12, seed=3)
    ctl = _ctrl(p)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    cost, eps, phi = ctl.debug_rollout(p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed)
    u2, c2 = ctl.debug_reduce(cost, phi, eps, p.u_nom, p.lam)
    ctl.sync()
    assert torch.equal(u, u2) and torch.equal(c, c2)


def test_fault_injection_host_side(monkeypatch):
    from paper_1503_00330_b300._lib import PiError, PI_ERR_OOM, PI_ERR_CUDA, PI_ERR_TIMEOUT
    p = W.problem(16, 4, 2, seed=1)
    ctl = _ctrl(p)
    for val, code in (("alloc", PI_ERR_OOM), ("launch", PI_ERR_CUDA), ("timeout", PI_ERR_TIMEOUT)):
        monkeypatch.setenv("PI_FAULT", val)
        with pytest.raises(PiError) as ei:
            ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
        assert ei.value.code == code
    monkeypatch.delenv("PI_FAULT")
    ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()


def test_device_wait_timeout_reports_and_recovers():
    """A device-side wait that nothing satisfies gives up after its limit: the
    kernel returns, pi_sync reports PI_ERR_TIMEOUT once, and the context keeps
    working (the next update matches a fresh context bitwise)."""
    import time
    from paper_1503_00330_b300._lib import PiError, PI_ERR_TIMEOUT
    p = W.problem(64, 5, 8, seed=3)
    ctl = _ctrl(p)
    t0 = time.perf_counter()
    ctl.debug_wait_timeout(20_000_000)            # 20 ms
    with pytest.raises(PiError) as ei:
        ctl.sync()
    assert ei.value.code == PI_ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.019
    ctl.sync()                                    # the error word was cleared
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    fresh = _ctrl(p)
    u2, c2 = fresh.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    fresh.sync()
    assert torch.equal(u, u2) and torch.equal(c, c2)
    with pytest.raises(PiError):
        ctl.debug_wait_timeout(10)                # limit below 1 us is rejected on the host


def test_invalid_update_arguments():
    from paper_1503_00330_b300._lib import PiError
    p = W.problem(16, 4, 2, seed=1)
    ctl = _ctrl(p)
    with pytest.raises(PiError):
        ctl.update(p.x0, p.u_nom, p.K, p.T, 0.0, p.sigma_u, p.seed)
    with pytest.raises(PiError):
        ctl.update(p.x0, p.u_nom, p.K, p.T, 1.0, [-1, 0, 0, 0], p.seed)
    with pytest.raises(PiError):
        ctl.update(p.x0, p.u_nom, 0, p.T, 1.0, p.sigma_u, p.seed)


# ---------------------------------------------------------------------------
# full-size workloads: sampled rollouts against the oracle
# ---------------------------------------------------------------------------
def _sampled_S0(oracle, p, ranges):
    """Oracle S_{k,0} of the rollouts in `ranges` ((k0, n) pairs; rollout k depends
    only on its own noise counters, so a range is run alone, over the oracle's
    threads).  Returns (ks, S0)."""
    ks, out = [], []
    for k0, n in ranges:
        r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, n, p.T, p.sigma_u, p.seed, k0=int(k0))
        out.append(oracle.cost_to_go(r["cost"], r["phi"], float(p.model.dt))[:, 0])
        ks.append(np.arange(k0, k0 + n))
    return np.concatenate(ks), np.concatenate(out)


# 512 sampled rollouts of a full-size launch: the first and the last 256 (the first
# and last slot blocks of either form, and the ragged end of the launch)
def _edge_ranges(K, n=256):
    return [(0, n), (K - n, n)]


def test_precision_workload_sampled(oracle):
    """K=65536, T=100, L=2048, cond(D_j) log-uniform in [1, 1e3]: 512 sampled
    rollouts' S_{k,0} at full K (the full update at K=2048 and the realtime
    update in full are checked in the full-size parity tests)."""
    p = W.precision()
    ctl = _ctrl(p)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    c = c.cpu().numpy().astype(np.float64)
    ks, S0 = _sampled_S0(oracle, p, _edge_ranges(p.K))
    err = np.abs(c[ks] - S0) / S0
    print("precision sampled S0 (512 rollouts) max rel err", err.max())
    assert np.all(err <= S_TOL)
    assert np.all(np.isfinite(u.cpu().numpy()))


@pytest.mark.parametrize("L,form", [(70, "fp32"), (1, "fp32"), (257, "tc")])
def test_rh_advance_plant_step(oracle, L, form):
    """The receding-horizon step (Sec. 3.1): the plant, the LWPR mean model, moves x0 by
    one Euler step under u_out[0] (R13), against the oracle's Eq. 1 prediction; the plan
    is shifted left with its last control repeated (bitwise)."""
    from paper_1503_00330_b300.api import Controller
    p = W.problem(64, 9, L, seed=40 + L)
    ctl = Controller(p.model, p.cost, precision=form)
    g = np.random.default_rng(L)
    x0 = (p.x0 + g.normal(0, 0.3, 12)).astype(np.float32)
    u = g.normal(0, 0.3, (p.T, 4)).astype(np.float32)
    xd = torch.as_tensor(x0, device="cuda").clone()
    ud = torch.as_tensor(u, device="cuda").clone()
    un = torch.empty_like(ud)
    ctl.rh_advance(xd, ud, un)
    ctl.sync()
    y, _ = oracle.lwpr_predict(p.model, np.concatenate([x0, u[0]]))
    x_ref = x0.astype(np.float64) + float(p.model.dt) * y.reshape(-1)
    err = np.max(np.abs(xd.cpu().numpy() - x_ref) / (1.0 + np.abs(x_ref)))
    print(f"plant step L={L} ({form}): rel err {err:.3g}")
    assert err <= 1e-6
    assert np.array_equal(un.cpu().numpy(), np.concatenate([u[1:], u[-1:]]))


@pytest.mark.parametrize("form", ["fp32", "tc"])
def test_u_out_may_alias_u_nominal(form):
    """The header lets u_out alias u_nominal (an in-place plan update): the
    result equals the one written to a separate buffer, bitwise."""
    from paper_1503_00330_b300.api import Controller
    p = W.problem(300, 17, 40, seed=8, n_obs=3)
    p.u_nom = np.random.default_rng(1).normal(0, 0.2, (p.T, 4)).astype(np.float32)
    ctl = Controller(p.model, p.cost, precision=form)
    u_sep, c_sep = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    plan = torch.as_tensor(p.u_nom, device="cuda").clone()
    u_in, c_in = ctl.update(p.x0, plan, p.K, p.T, p.lam, p.sigma_u, p.seed, u_out=plan)
    ctl.sync()
    assert u_in.data_ptr() == plan.data_ptr()
    assert torch.equal(plan, u_sep) and torch.equal(c_in, c_sep)


def _damped_model(L, seed):
    """The synthetic model with each output's slope on its own state set to -3
    and the other slopes scaled by 0.3, so that long rollouts stay bounded
    (the undamped draw grows without bound over thousands of steps)."""
    m = W.make_lwpr(L, seed)
    beta = m.beta.astype(np.float64) * 0.3
    for o in range(beta.shape[0]):
        beta[o, :, o] = -3.0
    m.beta = np.ascontiguousarray(beta.astype(np.float32))
    return m


@pytest.mark.parametrize("form", ["fp32", "tc"])
@pytest.mark.parametrize("K,T,L,M,lam,damped", [(3, 4096, 1, 1, 1.0, True), (24, 1000, 5, 2, 5.0, True),
                                                (5, 12, 3, 64, 1.0, False)])
def test_end_to_end_long_horizon_and_most_subrollouts(oracle, form, K, T, L, M, lam, damped):
    """T = 4096 (the longest horizon the no-alloc entry point takes; 128 scan
    chunks) and T = 1000 with sub-rollouts, and M = 64 sub-rollouts per rollout
    (the largest M), in both forms, at the end-to-end tolerances."""
    model = _damped_model(L, 2000 + K) if damped else None
    p = W.problem(K, T, L, seed=2000 + K, n_obs=5, M=M, model=model, lam=lam)
    ctl = _ctrl(p, precision=form)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    uref, cref = _oracle_update(oracle, p)
    eu = _u_err(u.cpu().numpy(), uref)
    ec = np.max(np.abs(c.cpu().numpy() - cref) / cref)
    print(f"K={K} T={T} L={L} M={M} ({form}): u err {eu} cost err {ec:.3g}")
    assert np.all(eu <= U_TOL)
    assert ec <= S_TOL


def test_stage_times_ring():
    """With timing on, the context keeps the stage events of its last 64 timed
    updates: updates enqueued back to back can be read afterwards, oldest with the
    largest `back`; asking past what is kept is an argument error."""
    from paper_1503_00330_b300._lib import PiError
    p = W.problem(300, 20, 40, seed=4)
    ctl = _ctrl(p)
    ctl.set_timing(True)
    for i in range(3):
        ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed + i)
    times = [ctl.stage_times(back=b) for b in (2, 1, 0)]
    assert all(all(v > 0 for v in t) for t in times)
    assert ctl.stage_times() == times[-1]
    with pytest.raises(PiError):
        ctl.stage_times(back=3)
    ctl.sync()

"""Tensor-core form: the tcgen05 GEMM core against a float64 product of the
same fp16 operands, and the tensor-core rollout path (fp16 hi/lo split,
three products per term) against the FP64 oracle.

The split keeps each product to ~2^-22 relative, so the tensor-core form is
held to the same tolerances as the FP32 form: LWPR mean |dy| <= 2e-5 (1 + |y|),
variance |dvar| <= 2e-5 var + 1e-6, u_out 1e-5 per channel (scale as in the
parity tests), costs 1e-5 relative.  The method's stated bound for this form
(2e-3) is looser; the tests use the FP32 one."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1503_00330_b300 import _lib
from paper_1503_00330_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    from paper_1503_00330_b300.api import Controller
    build.build()
    p = W.problem(8, 4, 2, seed=0)
    return Controller(p.model, p.cost)


@pytest.mark.parametrize("K", [16, 32, 160])
def test_tc_gemm_core(ctl, K):
    g = np.random.default_rng(K)
    A = torch.from_numpy(g.normal(0, 1, (128, K)).astype(np.float16)).cuda()
    B = torch.from_numpy(g.normal(0, 1, (64, K)).astype(np.float16)).cuda()
    D = torch.full((128, 64), np.nan, dtype=torch.float32, device="cuda")
    lib = _lib.load()
    ctl._use_current_stream()
    _lib.check(lib.pi_debug_tc_gemm(ctl.handle, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), K,
                                    ctypes.c_void_p(D.data_ptr())))
    ctl.sync()
    a, b = A.cpu().double().numpy(), B.cpu().double().numpy()
    ref = a @ b.T
    bound = 1e-6 * (np.abs(a) @ np.abs(b).T) + 1e-6
    d = D.cpu().double().numpy()
    err = np.abs(d - ref)
    print(f"K={K}: max err {err.max():.3g}, worst ratio {np.max(err / bound):.3g}")
    assert np.all(np.isfinite(d))
    assert np.all(err <= bound)


def _tc(p):
    from paper_1503_00330_b300.api import Controller
    return Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, precision="tc")


def _u_err(u, ref, sigma_u, K):
    u, ref = np.asarray(u, np.float64), np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref).max(0), np.sqrt(np.asarray(sigma_u, np.float64) / K))
    return np.abs(u - ref).max(0) / scale


@pytest.mark.parametrize("L,n,cond", [(1, 5, False), (3, 70, False), (64, 200, False), (100, 130, True),
                                      (257, 129, False)])
def test_tc_lwpr_predict(ctl, oracle, L, n, cond):
    p = W.problem(8, 4, L, seed=L, conditioned=cond)
    tc = _tc(p)
    g = np.random.default_rng(L)
    z = np.concatenate([g.normal(0, 0.5, (n, 12)), g.normal(0, 0.3, (n, 4))], 1).astype(np.float32)
    y, v = tc.debug_lwpr(z)
    tc.sync()
    y, v = y.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    yr, vr = oracle.lwpr_predict(p.model, z)
    ey = np.max(np.abs(y - yr) / (1 + np.abs(yr)))
    print(f"TC L={L} n={n}: y err {ey:.3g}, var worst {np.max(np.abs(v - vr) / (2e-5 * vr + 1e-6)):.3g} of bound")
    assert ey <= 2e-5
    assert np.all(np.abs(v - vr) <= 2e-5 * vr + 1e-6)


@pytest.mark.parametrize("K,T,L,M,noise", [(256, 50, 64, 1, True), (65, 3, 2, 1, True), (130, 17, 70, 2, True),
                                           (200, 12, 33, 1, False)])
def test_tc_end_to_end(ctl, oracle, K, T, L, M, noise):
    p = W.problem(K, T, L, seed=7 + K, n_obs=4, M=M, model_noise=noise)
    tc = _tc(p)
    u, c = tc.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    tc.sync()
    uref, cref = oracle.pi_update(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed, M=p.M,
                                  model_noise=p.model_noise)
    eu = _u_err(u.cpu().numpy(), uref, p.sigma_u, p.K)
    ec = np.max(np.abs(c.cpu().numpy() - cref) / cref)
    print(f"TC K={K} T={T} L={L} M={M}: u err {eu}, cost err {ec:.3g}")
    assert np.all(eu <= 1e-5)
    assert ec <= 1e-5


def test_tc_precision_workload_sampled(ctl, oracle):
    """K=65536, T=100, L=2048, cond(D) in [1, 1e3]: S_{k,0} of 512 sampled rollouts."""
    p = W.precision()
    tc = _tc(p)
    u, c = tc.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    tc.sync()
    c = c.cpu().numpy().astype(np.float64)
    # 512 rollouts: the first and the last 256 of the launch (first and last slot blocks)
    for k0 in (0, p.K - 256):
        r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, 256, p.T, p.sigma_u, p.seed, k0=k0)
        S0 = oracle.cost_to_go(r["cost"], r["phi"], float(p.model.dt))[:, 0]
        err = np.abs(c[k0:k0 + 256] - S0) / S0
        print(f"TC precision rollouts {k0}..{k0 + 255}: max rel err {err.max():.3g}")
        assert np.all(err <= 1e-5)
    assert np.all(np.isfinite(u.cpu().numpy()))


@pytest.mark.parametrize("K,T,L,M", [(256, 20, 300, 1), (300, 9, 64, 2), (1, 4, 5, 1)])
def test_tc_output_split_is_bitwise_invariant(ctl, monkeypatch, K, T, L, M):
    """The single-controller rollout may split a slot block's 12 outputs over
    a cluster of 2, 3 or 4 CTAs that exchange their means and variances
    through distributed shared memory; every split gives the same bits."""
    p = W.problem(K, T, L, seed=21, n_obs=5, M=M)
    p.u_nom = np.random.default_rng(2).normal(0, 0.2, (T, 4)).astype(np.float32)
    c = _tc(p)
    out = {}
    for split in ("1", "2", "3", "4"):
        monkeypatch.setenv("PI2RH_TC_SPLIT", split)
        u, cs = c.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
        c.sync()
        out[split] = (u.cpu().numpy(), cs.cpu().numpy())
    for split in ("2", "3", "4"):
        assert np.array_equal(out[split][0], out["1"][0]), f"u_out differs with split {split}"
        assert np.array_equal(out[split][1], out["1"][1]), f"costs differ with split {split}"
    assert np.all(np.isfinite(out["1"][0]))

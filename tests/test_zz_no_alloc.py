"""pi_update_noalloc against pi_update, through the C ABI.

pi_update_noalloc serves callers that cannot allocate device memory once they
run (a real-time control loop that forbids cudaMalloc after start-up, or a
host program that owns all GPU memory through its own pool): it keeps its
scratch in a fixed array inside the library.  Its results must match the
ordinary entry point's within the end-to-end tolerances of the parity tests,
in every form (FP32 and both tensor-core forms), on two calls in a row with
different sizes and seeds: the
second call is the smaller one, so it runs over the first call's leftovers
in the shared array and must not read them.  After one set-up call, further
calls must leave the device's free memory unchanged.  This file sorts last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1503_00330_b300 import _lib
from paper_1503_00330_b300 import workloads as W

pytestmark = pytest.mark.gpu

U_TOL = 1e-5      # same end-to-end tolerances as the parity tests
S_TOL = 1e-5


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _call(lib, fn, h, x0, un, K, T, lam, su, seed, u, c):
    rc = getattr(lib, fn)(h, ctypes.c_void_p(x0.data_ptr()), ctypes.c_void_p(un.data_ptr()), K, T, lam, _fp(su),
                          ctypes.c_uint64(seed), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(c.data_ptr()))
    _lib.check(rc)


@pytest.mark.parametrize("form", ["fp32", "tc", "tc_fp16x2"])
def test_noalloc_matches_update_two_calls(form):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    from paper_1503_00330_b300.api import Controller
    build.build()
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    # first call the larger (K*T = 25000), then the smaller (K*T = 12000)
    cases = [W.problem(1000, 25, 9, seed=22, n_obs=4), W.problem(300, 40, 16, seed=21, n_obs=6)]
    runs = []
    for p in cases:
        ctl = Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, precision=form)
        lib.pi_set_stream(ctl.handle, ctypes.c_void_p(stream.cuda_stream))
        x0 = torch.as_tensor(p.x0, device=dev)
        un = torch.as_tensor(np.random.default_rng(p.seed).normal(0, 0.2, (p.T, 4)).astype(np.float32), device=dev)
        su = np.ascontiguousarray(p.sigma_u, np.float32)
        out = {k: (torch.empty((p.T, 4), dtype=torch.float32, device=dev),
                   torch.empty((p.K,), dtype=torch.float32, device=dev)) for k in ("ref", "na")}
        _call(lib, "pi_update", ctl.handle, x0, un, p.K, p.T, p.lam, su, p.seed, *out["ref"])
        _lib.check(lib.pi_sync(ctl.handle))
        runs.append((p, ctl, x0, un, su, out))

    # set-up call: loads the fixed array on the device (lazy module loading)
    p, ctl, x0, un, su, out = runs[1]
    _call(lib, "pi_update_noalloc", ctl.handle, x0, un, 64, p.T, p.lam, su, 5, *out["na"])
    _lib.check(lib.pi_sync(ctl.handle))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]

    for p, ctl, x0, un, su, out in runs:
        _call(lib, "pi_update_noalloc", ctl.handle, x0, un, p.K, p.T, p.lam, su, p.seed, *out["na"])
        _lib.check(lib.pi_sync(ctl.handle))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(dev)[0]
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes across no-alloc calls"

    for p, ctl, x0, un, su, out in runs:
        u_ref, c_ref = (t.cpu().numpy().astype(np.float64) for t in out["ref"])
        u_na, c_na = (t.cpu().numpy().astype(np.float64) for t in out["na"])
        scale = np.maximum(np.abs(u_ref).max(0), np.sqrt(su.astype(np.float64) / p.K))
        eu = np.abs(u_na - u_ref).max(0) / scale
        ec = np.max(np.abs(c_na - c_ref) / c_ref)
        print(f"{form} K={p.K} T={p.T}: u_out rel err {eu.max():.3g}, costs rel err {ec:.3g}")
        assert np.all(eu <= U_TOL)
        assert ec <= S_TOL
        ctl.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300.api import Controller
    lib = _lib.load()
    p = W.problem(8, 4, 2, seed=1)
    ctl = Controller(p.model, p.cost)
    dev = torch.device("cuda", 0)
    x0 = torch.zeros(12, device=dev)
    su = np.ascontiguousarray(p.sigma_u, np.float32)
    for K, T in ((65537, 1), (1, 4097), (8192, 129)):
        un = torch.zeros((T, 4), device=dev)
        u = torch.empty((T, 4), device=dev)
        c = torch.empty((K,), device=dev)
        with pytest.raises(_lib.PiError) as ei:
            _call(lib, "pi_update_noalloc", ctl.handle, x0, un, K, T, 1.0, su, 0, u, c)
        assert ei.value.code == _lib.PI_ERR_INVALID_ARG
        assert "fixed scratch" in str(ei.value)
    ctl.close()

"""pi_update_noalloc against pi_update, through the C ABI.

pi_update_noalloc serves callers that cannot allocate device memory once they
run (a real-time control loop that forbids cudaMalloc after start-up, or a
host program that owns all GPU memory through its own pool): it keeps its
scratch in a fixed array inside the library.  Its results must match the
ordinary entry point's within the end-to-end tolerances of the parity tests,
on two calls in a row with different sizes and seeds (the second call must not
see the first call's leftovers).  This file sorts last so that a run stopping
at the first failure has already run every other test.
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


def _call(lib, fn, h, x0, un, K, T, lam, su, seed, dev):
    u = torch.empty((T, 4), dtype=torch.float32, device=dev)
    c = torch.empty((K,), dtype=torch.float32, device=dev)
    rc = getattr(lib, fn)(h, ctypes.c_void_p(x0.data_ptr()), ctypes.c_void_p(un.data_ptr()), K, T, lam, _fp(su),
                          ctypes.c_uint64(seed), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(c.data_ptr()))
    _lib.check(rc)
    return u, c


def test_noalloc_matches_update_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    from paper_1503_00330_b300.api import Controller
    build.build()
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    cases = [W.problem(300, 40, 16, seed=21, n_obs=6), W.problem(1000, 25, 9, seed=22, n_obs=4)]
    for p in cases:
        ctl = Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise)
        lib.pi_set_stream(ctl.handle, ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
        x0 = torch.as_tensor(p.x0, device=dev)
        un = torch.as_tensor(np.random.default_rng(p.seed).normal(0, 0.2, (p.T, 4)).astype(np.float32), device=dev)
        su = np.ascontiguousarray(p.sigma_u, np.float32)
        u_ref, c_ref = _call(lib, "pi_update", ctl.handle, x0, un, p.K, p.T, p.lam, su, p.seed, dev)
        u_na, c_na = _call(lib, "pi_update_noalloc", ctl.handle, x0, un, p.K, p.T, p.lam, su, p.seed, dev)
        _lib.check(lib.pi_sync(ctl.handle))
        u_ref, c_ref = u_ref.cpu().numpy().astype(np.float64), c_ref.cpu().numpy().astype(np.float64)
        u_na, c_na = u_na.cpu().numpy().astype(np.float64), c_na.cpu().numpy().astype(np.float64)
        scale = np.maximum(np.abs(u_ref).max(0), np.sqrt(su.astype(np.float64) / p.K))
        assert np.all(np.abs(u_na - u_ref).max(0) / scale <= U_TOL)
        assert np.max(np.abs(c_na - c_ref) / c_ref) <= S_TOL
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
        with pytest.raises(_lib.PiError) as ei:
            _call(lib, "pi_update_noalloc", ctl.handle, x0, un, K, T, 1.0, su, 0, dev)
        assert ei.value.code == _lib.PI_ERR_INVALID_ARG
        assert "fixed scratch" in str(ei.value)
    ctl.close()

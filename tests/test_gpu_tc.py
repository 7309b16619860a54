"""Tensor-core GEMM core (tcgen05.mma kind::f16, fp32 accumulate in TMEM)
against a float64 product of the same fp16 operands."""
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

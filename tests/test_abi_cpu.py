"""C-ABI checks that need no GPU: the in-tree library builds, loads, exports
every function ``include/pi2rh.h`` declares, and rejects invalid arguments
before touching a device."""
import ctypes

import numpy as np
import pytest

from paper_1503_00330_b300 import _lib, build
from paper_1503_00330_b300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_exports_every_declared_function(lib):
    names = _lib.declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/pi2rh.h but not exported"
    assert set(names) == set(_lib._SIGS), "binding signatures out of sync with the header"


def test_default_opts(lib):
    o = _lib.OptsC(-1, -1, -1, -1)
    lib.pi_default_opts(ctypes.byref(o))
    assert (o.precision, o.model_noise, o.M, o.device) == (0, 1, 1, 0)


def _create(lib, model, cost, M=1, n_in=16, n_out=12):
    arrs = [np.ascontiguousarray(a, np.float32) for a in (model.c, model.D, model.beta, model.b, model.sigma)]
    lw = _lib.LwprParamsC(n_in, n_out, model.L, float(model.dt), *[a.ctypes.data for a in arrs])
    obs = np.ascontiguousarray(cost.obs_xy, np.float32)
    cp = _lib.CostParamsC((ctypes.c_float * 3)(*cost.goal), (ctypes.c_float * 3)(*cost.Q_pos), cost.Q_vel,
                          cost.Q_ang, cost.w_obs, cost.obs_sharp, cost.radius, cost.w_crash, cost.w_var,
                          cost.w_T, cost.obs_kind, obs.shape[0], obs.ctypes.data)
    opts = _lib.OptsC(0, 1, M, 0)
    h = ctypes.c_void_p()
    rc = lib.pi_create(ctypes.byref(lw), ctypes.byref(cp), ctypes.byref(opts), ctypes.byref(h))
    return rc, h


def test_create_rejects_bad_arguments(lib):
    m = W.make_lwpr(3, 0)
    c = W.make_cost(2, 0)
    assert _create(lib, m, c, n_in=15)[0] == _lib.PI_ERR_INVALID_ARG
    assert b"n_in" in lib.pi_last_error()
    assert _create(lib, m, c, n_out=3)[0] == _lib.PI_ERR_INVALID_ARG
    assert _create(lib, m, c, M=3)[0] == _lib.PI_ERR_INVALID_ARG
    assert _create(lib, m, c, M=128)[0] == _lib.PI_ERR_INVALID_ARG
    bad = W.make_lwpr(3, 0)
    bad.D[0, 0, 0, 0] = np.nan
    assert _create(lib, bad, c)[0] == _lib.PI_ERR_INVALID_ARG
    assert b"finite" in lib.pi_last_error()
    many = W.make_cost(300, 0)
    assert _create(lib, m, many)[0] == _lib.PI_ERR_INVALID_ARG


def test_null_context_rejected(lib):
    s = np.zeros(4, np.float32)
    sp = s.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    rc = lib.pi_update(None, None, None, 4, 4, 1.0, sp, 0, None, None)
    assert rc == _lib.PI_ERR_INVALID_ARG
    assert lib.pi_sync(None) == _lib.PI_ERR_INVALID_ARG
    lib.pi_destroy(None)                      # accepted, no-op
    assert lib.pi_launch_count(None) == 0


def test_debug_noise_rejects_sizes(lib):
    assert lib.pi_debug_noise(0, 0, 5, 0, None, None) == _lib.PI_ERR_INVALID_ARG
    assert lib.pi_debug_noise(0, 5, 5, 0, None, None) == _lib.PI_ERR_INVALID_ARG


def test_ctypes_structs_match_the_c_layout():
    """Every struct the binding passes across the boundary has the C compiler's
    size and member offsets (a drifted field would corrupt data silently)."""
    import ctypes
    from paper_1503_00330_b300 import _lib
    lib = _lib.load()
    buf = (ctypes.c_size_t * 128)()
    n = ctypes.c_int()
    _lib.check(lib.pi_debug_struct_layout(buf, 128, ctypes.byref(n)))
    c_side = list(buf[:n.value])
    names = {"LwprParamsC": ["n_in", "n_out", "L", "dt", "c", "D", "beta", "b", "sigma"],
             "CostParamsC": ["goal", "Q_pos", "Q_vel", "Q_ang", "w_obs", "obs_sharp", "radius", "w_crash", "w_var",
                             "w_T", "obs_kind", "n_obs", "obs_xy"],
             "OptsC": ["precision", "model_noise", "M", "device"],
             "BatchItemC": ["ctx", "K", "T", "x0", "u_nominal", "u_out", "costs_out"],
             "ServerOptsC": ["n_agents", "K_max", "T_max", "max_inflight", "max_group", "hbm_budget", "want_costs"],
             "ServeRequestC": ["agent", "K", "T", "lam", "sigma_u", "x0", "keep_result"],
             "ServeDoneC": ["ticket", "agent", "K", "T", "status", "group_size", "t_submit_ns", "t_launch_ns",
                            "t_result_ns"],
             "ServeArrivalC": ["t_ns", "agent", "K", "T"],
             "ServerStatsC": ["submitted", "completed", "groups", "launches", "memory_waits", "pool_bytes",
                              "pool_peak_bytes", "peak_inflight_requests", "peak_group_size"]}
    py_side = []
    for cls, fields in names.items():
        st = getattr(_lib, cls)
        assert [f for f, _ in st._fields_] == fields, cls
        py_side.append(ctypes.sizeof(st))
        py_side += [getattr(st, f).offset for f in fields]
    assert py_side == c_side

"""ctypes view of the C ABI declared in ``include/pi2rh.h`` (argument marshalling only).

The shared library is built in-tree by ``paper_1503_00330_b300.build``.  If it is
missing, loading raises: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libpi2rh.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "pi2rh.h")

(PI_OK, PI_ERR_INVALID_ARG, PI_ERR_OOM, PI_ERR_CUDA, PI_ERR_TIMEOUT, PI_ERR_INTERNAL, PI_ERR_UNSUPPORTED,
 PI_ERR_BUSY, PI_ERR_CANCELLED) = range(9)
PI_SPLIT_OFF, PI_SPLIT_AUTO, PI_SPLIT_ALWAYS = range(3)
ERR_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "INTERNAL", 6: "UNSUPPORTED",
             7: "BUSY", 8: "CANCELLED"}

_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p


class LwprParamsC(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int), ("n_out", ctypes.c_int), ("L", ctypes.c_int), ("dt", ctypes.c_float),
                ("c", _vp), ("D", _vp), ("beta", _vp), ("b", _vp), ("sigma", _vp)]


class CostParamsC(ctypes.Structure):
    _fields_ = [("goal", ctypes.c_float * 3), ("Q_pos", ctypes.c_float * 3), ("Q_vel", ctypes.c_float),
                ("Q_ang", ctypes.c_float), ("w_obs", ctypes.c_float), ("obs_sharp", ctypes.c_float),
                ("radius", ctypes.c_float), ("w_crash", ctypes.c_float), ("w_var", ctypes.c_float),
                ("w_T", ctypes.c_float), ("obs_kind", ctypes.c_int), ("n_obs", ctypes.c_int),
                ("obs_xy", _vp)]


class OptsC(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("model_noise", ctypes.c_int), ("M", ctypes.c_int),
                ("device", ctypes.c_int)]


class BatchItemC(ctypes.Structure):
    _fields_ = [("ctx", _vp), ("K", ctypes.c_int), ("T", ctypes.c_int), ("x0", _vp), ("u_nominal", _vp),
                ("u_out", _vp), ("costs_out", _vp)]


class ServerOptsC(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int), ("K_max", ctypes.c_int), ("T_max", ctypes.c_int),
                ("max_inflight", ctypes.c_int), ("max_group", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("want_costs", ctypes.c_int)]


class ServeRequestC(ctypes.Structure):
    _fields_ = [("agent", ctypes.c_int), ("K", ctypes.c_int), ("T", ctypes.c_int), ("lam", ctypes.c_float),
                ("sigma_u", ctypes.c_float * 4), ("x0", _vp), ("keep_result", ctypes.c_int)]


class ServeDoneC(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("agent", ctypes.c_int), ("K", ctypes.c_int), ("T", ctypes.c_int),
                ("status", ctypes.c_int), ("group_size", ctypes.c_int), ("t_submit_ns", ctypes.c_int64),
                ("t_launch_ns", ctypes.c_int64), ("t_result_ns", ctypes.c_int64)]


class ServeArrivalC(ctypes.Structure):
    _fields_ = [("t_ns", ctypes.c_int64), ("agent", ctypes.c_int), ("K", ctypes.c_int), ("T", ctypes.c_int)]


class ServerStatsC(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("groups", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("memory_waits", ctypes.c_uint64), ("pool_bytes", ctypes.c_size_t),
                ("pool_peak_bytes", ctypes.c_size_t), ("peak_inflight_requests", ctypes.c_int),
                ("peak_group_size", ctypes.c_int)]


class PiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pi2rh error {ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "pi_default_opts": (None, [ctypes.POINTER(OptsC)]),
    "pi_create": (ctypes.c_int, [ctypes.POINTER(LwprParamsC), ctypes.POINTER(CostParamsC),
                                 ctypes.POINTER(OptsC), ctypes.POINTER(_vp)]),
    "pi_set_stream": (ctypes.c_int, [_vp, _vp]),
    "pi_reserve": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "pi_update": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, _fp,
                                 ctypes.c_uint64, _vp, _vp]),
    "pi_update_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, _fp,
                                         ctypes.c_uint64, _vp, _vp]),
    "pi_update_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, _fp,
                                      ctypes.c_uint64, _vp, _vp]),
    "pi_sync": (ctypes.c_int, [_vp]),
    "pi_destroy": (None, [_vp]),
    "pi_last_error": (ctypes.c_char_p, []),
    "pi_launch_count": (ctypes.c_uint64, [_vp]),
    "pi_rh_advance": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "pi_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pi_set_output_split": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pi_debug_split_plan": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
    "pi_debug_split_drop_cta": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pi_debug_split_plan_sizes": (ctypes.c_int, [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_int)] * 3),
    "pi_debug_split_partition": (ctypes.c_int, [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int)] * 2),
    "pi_stage_times": (ctypes.c_int, [_vp, _fp]),
    "pi_stage_times_at": (ctypes.c_int, [_vp, ctypes.c_int, _fp]),
    "pi_debug_tc_gemm": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "pi_debug_wait_timeout": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "pi_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchItemC), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    "pi_batch_set_schedule": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "pi_batch_set_tile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pi_batch_set_stream": (ctypes.c_int, [_vp, _vp]),
    "pi_batch_update": (ctypes.c_int, [_vp, _fp, _fp, ctypes.POINTER(ctypes.c_uint64)]),
    "pi_batch_sync": (ctypes.c_int, [_vp]),
    "pi_batch_launch_count": (ctypes.c_uint64, [_vp]),
    "pi_batch_destroy": (None, [_vp]),
    "pi_server_default_opts": (None, [ctypes.POINTER(ServerOptsC)]),
    "pi_server_create": (ctypes.c_int, [_vp, ctypes.POINTER(ServerOptsC), ctypes.POINTER(_vp)]),
    "pi_server_set_agent": (ctypes.c_int, [_vp, ctypes.c_int, _fp, _fp, ctypes.c_uint64]),
    "pi_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(ServeRequestC), ctypes.POINTER(ctypes.c_uint64)]),
    "pi_server_cancel": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "pi_server_poll": (ctypes.c_int, [_vp, ctypes.POINTER(ServeDoneC), ctypes.c_int, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int)]),
    "pi_server_result": (ctypes.c_int, [_vp, ctypes.c_uint64, _fp, _fp]),
    "pi_server_drain": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "pi_server_replay": (ctypes.c_int, [_vp, ctypes.POINTER(ServeArrivalC), ctypes.c_int,
                                        ctypes.POINTER(ServeRequestC), ctypes.POINTER(ServeDoneC),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pi_server_state_save": (ctypes.c_int, [_vp, _fp, _fp, ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_uint64)]),
    "pi_server_state_load": (ctypes.c_int, [_vp, _fp, _fp, ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_uint64)]),
    "pi_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ServerStatsC)]),
    "pi_server_destroy": (None, [_vp]),
    "pi_debug_struct_layout": (ctypes.c_int, [ctypes.POINTER(ctypes.c_size_t), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
    "pi_debug_pipe_rates": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]),
    "pi_debug_fp64_rate": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "pi_debug_pool": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]),
    "pi_debug_noise": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "pi_debug_normals": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                        _vp]),
    "pi_debug_lwpr": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "pi_debug_rollout": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _fp, ctypes.c_uint64,
                                        _vp, _vp, _vp]),
    "pi_debug_reduce": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                       _vp, _vp]),
}


def load():
    """Loads the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1503_00330_b300.build`; there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc: int) -> None:
    if rc != PI_OK:
        msg = load().pi_last_error()
        raise PiError(rc, msg.decode() if msg else "")


def declared_functions() -> list[str]:
    """Names of the functions declared in include/pi2rh.h."""
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pi_[a-z0-9_]+)\s*\(", src)))

"""Python front end of the FP64 CPU oracle (``pi_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark call this module; the product path never does.  It shares no
code with the CUDA library.  Inputs are the FP32-rounded arrays of the seeded
workload generator, widened exactly to float64 here.

Functions mirror the steps of the method:
  * ``philox`` / ``noise_raw`` / ``normals``  -- counter-based noise (Philox4x32-10,
    Salmon et al. SC'11) and Box-Muller normals.
  * ``lwpr_predict``      -- Sec. 2, Eq. 1 (mean and variance of the LWPR model).
  * ``running_cost`` / ``terminal_cost`` -- Sec. 5 cost (indicator or bump form).
  * ``rollouts``          -- Sec. 3.1 sampling with Sec. 3.2 sub-rollouts, Euler steps.
  * ``cost_to_go``        -- S(tau_i) = phi + sum_{j>=i} q_j dt (Sec. 3.1).
  * ``weighted_update``   -- Eq. 2 per timestep.
  * ``pi_update``         -- the whole update.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NX, NU, NZ, NY = 12, 4, 16, 12

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)


class _Lwpr(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("dt", ctypes.c_double), ("c", _dp), ("D", _dp),
                ("beta", _dp), ("b", _dp), ("sigma", _dp)]


class _Cost(ctypes.Structure):
    _fields_ = [("goal", ctypes.c_double * 3), ("Q_pos", ctypes.c_double * 3),
                ("Q_vel", ctypes.c_double), ("Q_ang", ctypes.c_double),
                ("w_obs", ctypes.c_double), ("obs_sharp", ctypes.c_double),
                ("radius", ctypes.c_double), ("w_crash", ctypes.c_double),
                ("w_var", ctypes.c_double), ("w_T", ctypes.c_double),
                ("obs_kind", ctypes.c_int), ("n_obs", ctypes.c_int), ("obs_xy", _dp)]


def build(force: bool = False) -> str:
    """Compile ``pi_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_uniform.argtypes = [ctypes.c_uint32]
        lib.orc_uniform.restype = ctypes.c_double
        lib.orc_noise_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint32, _u32p]
        lib.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, _dp, _dp]
        lib.orc_lwpr_predict.argtypes = [ctypes.POINTER(_Lwpr), _dp, _dp, _dp]
        lib.orc_inside_any.argtypes = [ctypes.POINTER(_Cost), ctypes.c_double, ctypes.c_double]
        lib.orc_inside_any.restype = ctypes.c_int
        lib.orc_running_cost.argtypes = [ctypes.POINTER(_Cost), _dp, _dp]
        lib.orc_running_cost.restype = ctypes.c_double
        lib.orc_terminal_cost.argtypes = [ctypes.POINTER(_Cost), _dp]
        lib.orc_terminal_cost.restype = ctypes.c_double
        lib.orc_rollouts.argtypes = [ctypes.POINTER(_Lwpr), ctypes.POINTER(_Cost), _dp, _dp,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                     ctypes.c_uint64, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.orc_rollouts_from.argtypes = [ctypes.POINTER(_Lwpr), ctypes.POINTER(_Cost), _dp, _dp,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                          ctypes.c_uint64, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.orc_cost_to_go.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
        lib.orc_weighted_update.argtypes = [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, _dp]
        lib.orc_pi_update.argtypes = [ctypes.POINTER(_Lwpr), ctypes.POINTER(_Cost), _dp, _dp,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      _dp, ctypes.c_uint64, ctypes.c_int, _dp, _dp]
        lib.orc_pi_update.restype = ctypes.c_int
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


@dataclass
class _Held:
    """Keeps the widened arrays alive while a C struct points into them."""
    arrays: list
    lwpr: _Lwpr | None = None
    cost: _Cost | None = None


def _lwpr_struct(model) -> _Held:
    arrs = [_f64(model.c), _f64(model.D), _f64(model.beta), _f64(model.b), _f64(model.sigma)]
    L = int(arrs[0].shape[1])
    assert arrs[0].shape == (NY, L, NZ) and arrs[1].shape == (NY, L, NZ, NZ)
    assert arrs[2].shape == (NY, L, NZ) and arrs[3].shape == (NY, L) and arrs[4].shape == (NY, L)
    s = _Lwpr(L, float(np.float64(model.dt)), *[_ptr(a) for a in arrs])
    return _Held(arrs, lwpr=s)


def _cost_struct(cp) -> _Held:
    obs = _f64(np.asarray(cp.obs_xy).reshape(-1, 2)) if len(cp.obs_xy) else np.zeros((1, 2))
    n_obs = int(np.asarray(cp.obs_xy).reshape(-1, 2).shape[0]) if len(cp.obs_xy) else 0
    s = _Cost((ctypes.c_double * 3)(*map(float, cp.goal)), (ctypes.c_double * 3)(*map(float, cp.Q_pos)),
              float(cp.Q_vel), float(cp.Q_ang), float(cp.w_obs), float(cp.obs_sharp),
              float(cp.radius), float(cp.w_crash), float(cp.w_var), float(cp.w_T),
              int(cp.obs_kind), n_obs, _ptr(obs))
    return _Held([obs], cost=s)


# ---------------------------------------------------------------------------
# noise
# ---------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    """Raw Philox4x32-10 block for a 4-word counter and 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p), out.ctypes.data_as(_u32p))
    return out


def uniform(r: int) -> float:
    return _load().orc_uniform(int(r))


def noise_raw(seed: int, K: int, T: int, m: int = 0) -> np.ndarray:
    """Raw blocks [K][T][4 blocks][4 words]; block 0 always uses sub-rollout 0
    (the shared control perturbation), blocks 1..3 use sub-rollout ``m``."""
    lib = _load()
    out = np.zeros((K, T, 4, 4), dtype=np.uint32)
    tmp = np.zeros(4, dtype=np.uint32)
    for k in range(K):
        for t in range(T):
            for blk in range(4):
                lib.orc_noise_raw(seed, k, t, blk, 0 if blk == 0 else m, tmp.ctypes.data_as(_u32p))
                out[k, t, blk] = tmp
    return out


def normals(seed: int, k: int, t: int, m: int = 0):
    lib = _load()
    nc = np.zeros(4)
    nm = np.zeros(12)
    lib.orc_normals(seed, k, t, m, _ptr(nc), _ptr(nm))
    return nc, nm


# ---------------------------------------------------------------------------
# LWPR, cost
# ---------------------------------------------------------------------------
def lwpr_predict(model, z) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 1 at each row of ``z`` ([n, 16] or [16]) -> (y [n, 12], var [n, 12])."""
    lib = _load()
    h = _lwpr_struct(model)
    Z = _f64(z).reshape(-1, NZ)
    y = np.zeros((Z.shape[0], NY))
    v = np.zeros((Z.shape[0], NY))
    for i in range(Z.shape[0]):
        zi = np.ascontiguousarray(Z[i])
        yi = np.zeros(NY)
        vi = np.zeros(NY)
        lib.orc_lwpr_predict(ctypes.byref(h.lwpr), _ptr(zi), _ptr(yi), _ptr(vi))
        y[i] = yi
        v[i] = vi
    return y, v


def inside_any(cost_params, px: float, py: float) -> int:
    h = _cost_struct(cost_params)
    return int(_load().orc_inside_any(ctypes.byref(h.cost), float(px), float(py)))


def running_cost(cost_params, x, var) -> float:
    h = _cost_struct(cost_params)
    xs, vs = _f64(x), _f64(var)
    return float(_load().orc_running_cost(ctypes.byref(h.cost), _ptr(xs), _ptr(vs)))


def terminal_cost(cost_params, x) -> float:
    h = _cost_struct(cost_params)
    xs = _f64(x)
    return float(_load().orc_terminal_cost(ctypes.byref(h.cost), _ptr(xs)))


# ---------------------------------------------------------------------------
# rollouts, cost-to-go, weighted update
# ---------------------------------------------------------------------------
def rollouts(model, cost_params, x0, u_nom, K, T, sigma_u, seed, M=1, model_noise=True,
             want_traj=False, k0=0):
    """Rollouts k0 .. k0+K-1 -> dict(eps [K,T,4], cost [K,T], phi [K],
    traj [K,M,T+1,12] or None)."""
    lib = _load()
    hl, hc = _lwpr_struct(model), _cost_struct(cost_params)
    x0a, un, su = _f64(x0), _f64(u_nom).reshape(T, NU), _f64(sigma_u)
    eps = np.zeros((K, T, NU))
    cost = np.zeros((K, T))
    phi = np.zeros(K)
    traj = np.zeros((K, M, T + 1, NX)) if want_traj else None
    lib.orc_rollouts_from(ctypes.byref(hl.lwpr), ctypes.byref(hc.cost), _ptr(x0a), _ptr(un), int(k0), K, T,
                          M, _ptr(su), int(seed), int(bool(model_noise)), _ptr(eps), _ptr(cost), _ptr(phi),
                          _ptr(traj) if want_traj else None)
    return {"eps": eps, "cost": cost, "phi": phi, "traj": traj}


def cost_to_go(cost, phi, dt) -> np.ndarray:
    c, p = _f64(cost), _f64(phi)
    K, T = c.shape
    S = np.zeros((K, T))
    _load().orc_cost_to_go(_ptr(c), _ptr(p), K, T, float(dt), _ptr(S))
    return S


def weighted_update(S, eps, u_nom, lam) -> np.ndarray:
    s, e = _f64(S), _f64(eps)
    K, T = s.shape
    un = _f64(u_nom).reshape(T, NU)
    out = np.zeros((T, NU))
    _load().orc_weighted_update(_ptr(s), _ptr(e), _ptr(un), K, T, float(lam), _ptr(out))
    return out


def pi_update(model, cost_params, x0, u_nom, K, T, lam, sigma_u, seed, M=1, model_noise=True):
    """One control update -> (u_out [T,4], costs_out [K] = S_{k,0})."""
    lib = _load()
    hl, hc = _lwpr_struct(model), _cost_struct(cost_params)
    x0a, un, su = _f64(x0), _f64(u_nom).reshape(T, NU), _f64(sigma_u)
    u_out = np.zeros((T, NU))
    costs = np.zeros(K)
    rc = lib.orc_pi_update(ctypes.byref(hl.lwpr), ctypes.byref(hc.cost), _ptr(x0a), _ptr(un), K, T, M,
                           float(lam), _ptr(su), int(seed), int(bool(model_noise)), _ptr(u_out),
                           _ptr(costs))
    if rc != 0:
        raise MemoryError("oracle pi_update: allocation failed")
    return u_out, costs


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(n: int) -> None:
    """Threads of the rollout loop from now on (OpenMP)."""
    _load().orc_set_threads(int(n))

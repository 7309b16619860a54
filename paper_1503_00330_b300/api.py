"""Python front end of the PI^2-RH / LWPR library.

Thin marshalling over the C ABI (``include/pi2rh.h``): every step of the
update runs in the library's CUDA kernels.  PyTorch provides device memory
and the current CUDA stream; nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import PiError, check  # noqa: F401
from .workloads import CostParams, LwprModel

NX, NU, NZ, NY = 12, 4, 16, 12


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _f32_dev(a, device) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.float32).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)


def _sigma4(sigma_u):
    s = np.ascontiguousarray(np.asarray(sigma_u, np.float32).reshape(4))
    return s, s.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Controller:
    """One LWPR model + cost on one GPU (a ``pi_ctx``)."""

    PRECISIONS = {"fp32": 0, "tc": 1, "tc_fp16x2": 2}

    def __init__(self, model: LwprModel, cost: CostParams, M: int = 1, model_noise: bool = True,
                 device: int = 0, precision: str = "fp32"):
        lib = _lib.load()
        self._lib = lib
        self.device = torch.device("cuda", device)
        self.model, self.cost, self.M = model, cost, M
        arrs = [np.ascontiguousarray(a, np.float32) for a in (model.c, model.D, model.beta, model.b, model.sigma)]
        lw = _lib.LwprParamsC(NZ, NY, int(model.L), float(model.dt), *[a.ctypes.data for a in arrs])
        obs = np.ascontiguousarray(np.asarray(cost.obs_xy, np.float32).reshape(-1, 2))
        cp = _lib.CostParamsC((ctypes.c_float * 3)(*cost.goal), (ctypes.c_float * 3)(*cost.Q_pos),
                              cost.Q_vel, cost.Q_ang, cost.w_obs, cost.obs_sharp, cost.radius,
                              cost.w_crash, cost.w_var, cost.w_T, int(cost.obs_kind), int(obs.shape[0]),
                              obs.ctypes.data if obs.size else None)
        self.precision = precision
        opts = _lib.OptsC(self.PRECISIONS[precision], 1 if model_noise else 0, int(M), int(device))
        h = ctypes.c_void_p()
        check(lib.pi_create(ctypes.byref(lw), ctypes.byref(cp), ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self._stream = None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _use_current_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            check(self._lib.pi_set_stream(self._h, ctypes.c_void_p(s)))
            self._stream = s

    def launch_count(self) -> int:
        return int(self._lib.pi_launch_count(self._h))

    def reserve(self, K: int, T: int):
        self._use_current_stream()
        check(self._lib.pi_reserve(self._h, K, T))

    def update(self, x0, u_nom, K: int, T: int, lam: float, sigma_u, seed: int,
               u_out: torch.Tensor | None = None, costs_out: torch.Tensor | None = None):
        """pi_update on device tensors; returns (u_out [T,4], costs_out [K]) (async)."""
        self._use_current_stream()
        x0 = _f32_dev(x0, self.device)
        u_nom = _f32_dev(u_nom, self.device)
        if u_out is None:
            u_out = torch.empty((T, NU), dtype=torch.float32, device=self.device)
        if costs_out is None:
            costs_out = torch.empty((K,), dtype=torch.float32, device=self.device)
        _, sp = _sigma4(sigma_u)
        check(self._lib.pi_update(self._h, _ptr(x0), _ptr(u_nom), K, T, float(lam), sp,
                                  ctypes.c_uint64(seed), _ptr(u_out), _ptr(costs_out)))
        return u_out, costs_out

    def update_host(self, x0, u_nom, K: int, T: int, lam: float, sigma_u, seed: int,
                    u_out: np.ndarray | None = None, costs_out: np.ndarray | None = None):
        """pi_update_host on host (numpy) buffers; synchronous."""
        self._use_current_stream()
        x0 = np.ascontiguousarray(x0, np.float32)
        u_nom = np.ascontiguousarray(u_nom, np.float32)
        if u_out is None:
            u_out = np.empty((T, NU), np.float32)
        if costs_out is None:
            costs_out = np.empty(K, np.float32)
        _, sp = _sigma4(sigma_u)
        check(self._lib.pi_update_host(self._h, x0.ctypes.data, u_nom.ctypes.data, K, T, float(lam), sp,
                                       ctypes.c_uint64(seed), u_out.ctypes.data, costs_out.ctypes.data))
        return u_out, costs_out

    def rh_advance(self, x0: torch.Tensor, u_out: torch.Tensor, u_nom_next: torch.Tensor):
        """In place: x0 <- plant step with u_out[0]; u_nom_next <- shifted plan."""
        self._use_current_stream()
        T = u_out.shape[0]
        check(self._lib.pi_rh_advance(self._h, _ptr(x0), _ptr(u_out), T, _ptr(u_nom_next)))

    def set_timing(self, enable: bool = True):
        check(self._lib.pi_set_timing(self._h, 1 if enable else 0))

    def set_output_split(self, mode: str = "auto"):
        """Launch of the FP32 rollout: "off" (one CTA per 64-slot block), "auto"
        (default: the output-split launch where it uses SMs the plain one leaves
        idle) or "always".  The results are the same bit for bit."""
        modes = {"off": _lib.PI_SPLIT_OFF, "auto": _lib.PI_SPLIT_AUTO, "always": _lib.PI_SPLIT_ALWAYS}
        check(self._lib.pi_set_output_split(self._h, modes[mode]))

    def split_plan(self, K: int):
        """(plain_blocks, units_per_cta, ctas) of the FP32 rollout launch for K
        rollouts: plain_blocks 64-slot blocks one CTA each, then (units_per_cta
        > 0) the rest as the output-split launch of ctas CTAs."""
        pb, upc, ctas = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._lib.pi_debug_split_plan(self._h, int(K), ctypes.byref(pb), ctypes.byref(upc), ctypes.byref(ctas)))
        return pb.value, upc.value, ctas.value

    def stage_times(self, back: int = 0):
        """(rollout_ms, scan_ms, merge_ms) of the timed update `back` calls before the
        last (0 = the last; the context keeps the last PI2RH_TIMING_RING = 64)."""
        ms = (ctypes.c_float * 3)()
        check(self._lib.pi_stage_times_at(self._h, int(back), ms))
        return tuple(float(v) for v in ms)

    def sync(self):
        check(self._lib.pi_sync(self._h))

    # ------------------------------------------------------------- staged
    def debug_wait_timeout(self, limit_ns: int = 5_000_000):
        """One device-side bounded wait that nothing satisfies (see pi_debug_wait_timeout)."""
        self._use_current_stream()
        check(self._lib.pi_debug_wait_timeout(self._h, int(limit_ns)))

    def debug_lwpr(self, z):
        self._use_current_stream()
        z = _f32_dev(z, self.device).reshape(-1, NZ)
        n = z.shape[0]
        y = torch.empty((n, NY), dtype=torch.float32, device=self.device)
        v = torch.empty((n, NY), dtype=torch.float32, device=self.device)
        check(self._lib.pi_debug_lwpr(self._h, _ptr(z), n, _ptr(y), _ptr(v)))
        return y, v

    def debug_rollout(self, x0, u_nom, K, T, sigma_u, seed):
        """Returns (cost [T,K], eps [T,K,4], phi [K])."""
        self._use_current_stream()
        x0 = _f32_dev(x0, self.device)
        u_nom = _f32_dev(u_nom, self.device)
        cost = torch.empty((T, K), dtype=torch.float32, device=self.device)
        eps = torch.empty((T, K, NU), dtype=torch.float32, device=self.device)
        phi = torch.empty((K,), dtype=torch.float32, device=self.device)
        _, sp = _sigma4(sigma_u)
        check(self._lib.pi_debug_rollout(self._h, _ptr(x0), _ptr(u_nom), K, T, sp, ctypes.c_uint64(seed),
                                          _ptr(cost), _ptr(eps), _ptr(phi)))
        return cost, eps, phi

    def debug_reduce(self, cost_tk, phi, eps_tk, u_nom, lam):
        """From cost [T,K], phi [K], eps [T,K,4] -> (u_out [T,4], costs_out [K])."""
        self._use_current_stream()
        cost_tk = _f32_dev(cost_tk, self.device)
        phi = _f32_dev(phi, self.device)
        eps_tk = _f32_dev(eps_tk, self.device)
        u_nom = _f32_dev(u_nom, self.device)
        T, K = cost_tk.shape
        u_out = torch.empty((T, NU), dtype=torch.float32, device=self.device)
        costs = torch.empty((K,), dtype=torch.float32, device=self.device)
        check(self._lib.pi_debug_reduce(self._h, _ptr(cost_tk), _ptr(phi), _ptr(eps_tk), _ptr(u_nom), K, T,
                                         float(lam), _ptr(u_out), _ptr(costs)))
        return u_out, costs


def debug_noise(seed: int, K: int, T: int, m: int = 0, device: int = 0) -> torch.Tensor:
    """Raw Philox blocks [K, T, 4, 4] (uint32 stored in int32)."""
    lib = _lib.load()
    raw = torch.empty((K, T, 4, 4), dtype=torch.int32, device=torch.device("cuda", device))
    s = torch.cuda.current_stream(raw.device).cuda_stream
    check(lib.pi_debug_noise(ctypes.c_uint64(seed), K, T, m, _ptr(raw), ctypes.c_void_p(s)))
    return raw


def debug_normals(seed: int, K: int, T: int, m: int = 0, device: int = 0):
    """(ctrl [K, T, 4], model [K, T, 12]) standard normals."""
    lib = _lib.load()
    dev = torch.device("cuda", device)
    ctrl = torch.empty((K, T, 4), dtype=torch.float32, device=dev)
    model = torch.empty((K, T, 12), dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    check(lib.pi_debug_normals(ctypes.c_uint64(seed), K, T, m, _ptr(ctrl), _ptr(model), ctypes.c_void_p(s)))
    return ctrl, model


class Batch:
    """Many controllers updated by one persistent launch under a CUDA graph.

    Each controller keeps its own device buffers (x0, u_nom, u_out, costs),
    exposed as lists of tensors; write new x0 / u_nom into them between
    updates.  All controllers must use the batch's precision form."""

    ORDERS = {"as_given": 0, "longest_first": 1, "round_robin": 2}

    def __init__(self, controllers: list, Ks: list[int], Ts: list[int], precision: str = "fp32",
                 x0=None, u_nom=None):
        lib = _lib.load()
        self._lib = lib
        n = len(controllers)
        self.controllers, self.Ks, self.Ts, self.precision = controllers, list(Ks), list(Ts), precision
        dev = controllers[0].device
        self.device = dev
        self.x0 = [(_f32_dev(x0[i], dev) if x0 is not None else torch.zeros(NX, device=dev)).clone() for i in range(n)]
        self.u_nom = [(_f32_dev(u_nom[i], dev) if u_nom is not None else torch.zeros((Ts[i], NU), device=dev)).clone()
                      for i in range(n)]
        self.u_out = [torch.empty((Ts[i], NU), dtype=torch.float32, device=dev) for i in range(n)]
        self.costs = [torch.empty((Ks[i],), dtype=torch.float32, device=dev) for i in range(n)]
        items = (_lib.BatchItemC * n)()
        for i, c in enumerate(controllers):
            items[i] = _lib.BatchItemC(c.handle, int(Ks[i]), int(Ts[i]), self.x0[i].data_ptr(), self.u_nom[i].data_ptr(),
                                       self.u_out[i].data_ptr(), self.costs[i].data_ptr())
        h = ctypes.c_void_p()
        check(lib.pi_batch_create(items, n, Controller.PRECISIONS[precision], ctypes.byref(h)))
        self._h = h
        self._stream = None

    @property
    def n(self) -> int:
        return len(self.controllers)

    def rollout_steps(self) -> int:
        return sum(K * T * c.M for K, T, c in zip(self.Ks, self.Ts, self.controllers))

    def set_schedule(self, order: str = "longest_first", grid: int = 0):
        check(self._lib.pi_batch_set_schedule(self._h, self.ORDERS[order], int(grid)))

    def set_tile(self, split: int = 0):
        """Tensor-core tile shape: 0 persistent work list; 1..4 CTAs per 128-slot item (outputs split)."""
        check(self._lib.pi_batch_set_tile(self._h, int(split)))

    def update(self, lam, sigma_u, seeds):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            check(self._lib.pi_batch_set_stream(self._h, ctypes.c_void_p(s)))
            self._stream = s
        lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float32), (self.n,)))
        su = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma_u, np.float32).reshape(-1, 4), (self.n, 4)))
        sd = np.ascontiguousarray(np.asarray(seeds, np.uint64).reshape(self.n))
        check(self._lib.pi_batch_update(self._h, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        su.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        sd.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return self.u_out, self.costs

    def sync(self):
        check(self._lib.pi_batch_sync(self._h))

    def launch_count(self) -> int:
        return int(self._lib.pi_batch_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SEED_STEP = 0x9E3779B97F4A7C15   # seed of an agent's n-th update: seed + n * SEED_STEP (mod 2^64)

DONE_DTYPE = np.dtype([("ticket", np.uint64), ("agent", np.int32), ("K", np.int32), ("T", np.int32),
                       ("status", np.int32), ("group_size", np.int32), ("t_submit_ns", np.int64),
                       ("t_launch_ns", np.int64), ("t_result_ns", np.int64)])


def update_seed(seed: int, n: int) -> int:
    """Noise seed of an agent's n-th served update."""
    return (int(seed) + int(n) * SEED_STEP) % (1 << 64)


def _done_array(buf, n: int) -> np.ndarray:
    out = np.zeros(n, DONE_DTYPE)
    for i in range(n):
        d = buf[i]
        out[i] = (d.ticket, d.agent, d.K, d.T, d.status, d.group_size, d.t_submit_ns, d.t_launch_ns, d.t_result_ns)
    return out


class Server:
    """Receding-horizon serving loop over one shared model (``pi_server``).

    ``controller`` supplies the model, cost, M and precision form; it must
    outlive the server.  Agents' states, warm-start plans and update counters
    stay in device memory; requests are queued with :meth:`submit` and their
    completion records read with :meth:`poll`."""

    def __init__(self, controller: Controller, n_agents: int, K_max: int = 16384, T_max: int = 128,
                 max_inflight: int = 2, max_group: int = 64, hbm_budget: int = 0, want_costs: bool = False):
        lib = _lib.load()
        self._lib = lib
        self.controller = controller
        o = _lib.ServerOptsC()
        lib.pi_server_default_opts(ctypes.byref(o))
        o.n_agents, o.K_max, o.T_max = int(n_agents), int(K_max), int(T_max)
        o.max_inflight, o.max_group, o.hbm_budget = int(max_inflight), int(max_group), int(hbm_budget)
        o.want_costs = 1 if want_costs else 0
        self.n_agents, self.K_max, self.T_max, self.want_costs = int(n_agents), int(K_max), int(T_max), want_costs
        h = ctypes.c_void_p()
        check(lib.pi_server_create(controller.handle, ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def set_agent(self, agent: int, x0, u_warm=None, seed: int = 0):
        x = np.ascontiguousarray(np.asarray(x0, np.float32).reshape(NX))
        w = None if u_warm is None else np.ascontiguousarray(np.asarray(u_warm, np.float32).reshape(self.T_max, NU))
        fp = ctypes.POINTER(ctypes.c_float)
        check(self._lib.pi_server_set_agent(self._h, int(agent), x.ctypes.data_as(fp),
                                            None if w is None else w.ctypes.data_as(fp), int(seed) % (1 << 64)))

    @staticmethod
    def _request(agent, K, T, lam, sigma_u, x0=None, keep=True):
        s = np.asarray(sigma_u, np.float32).reshape(4)
        q = _lib.ServeRequestC(int(agent), int(K), int(T), float(lam), (ctypes.c_float * 4)(*s), None,
                               1 if keep else 0)
        xbuf = None
        if x0 is not None:
            xbuf = np.ascontiguousarray(np.asarray(x0, np.float32).reshape(NX))
            q.x0 = xbuf.ctypes.data
        return q, xbuf

    def submit(self, agent: int, K: int, T: int, lam: float, sigma_u, x0=None, keep: bool = True) -> int:
        q, _xbuf = self._request(agent, K, T, lam, sigma_u, x0, keep)
        t = ctypes.c_uint64()
        check(self._lib.pi_server_submit(self._h, ctypes.byref(q), ctypes.byref(t)))
        return int(t.value)

    def cancel(self, ticket: int) -> bool:
        """Cancels a queued request; False if it is already on the GPU or finished."""
        rc = self._lib.pi_server_cancel(self._h, int(ticket))
        if rc == _lib.PI_ERR_BUSY:
            return False
        check(rc)
        return True

    def poll(self, max_n: int = 1024, timeout_us: int = 0) -> np.ndarray:
        buf = (_lib.ServeDoneC * max_n)()
        n = ctypes.c_int()
        check(self._lib.pi_server_poll(self._h, buf, int(max_n), int(timeout_us), ctypes.byref(n)))
        return _done_array(buf, n.value)

    def result(self, ticket: int, T: int, K: int | None = None):
        u = np.empty((T, NU), np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        c = np.empty(K, np.float32) if (K is not None and self.want_costs) else None
        check(self._lib.pi_server_result(self._h, int(ticket), u.ctypes.data_as(fp),
                                         None if c is None else c.ctypes.data_as(fp)))
        return u, c

    def drain(self, timeout_ms: int = 600_000):
        check(self._lib.pi_server_drain(self._h, int(timeout_ms)))

    def wait(self, tickets, timeout_s: float = 600.0) -> dict:
        """Polls until every ticket in ``tickets`` has a completion record; returns them by ticket."""
        want = set(int(t) for t in tickets)
        got = {}
        import time
        t_end = time.monotonic() + timeout_s
        while want - got.keys():
            if time.monotonic() > t_end:
                raise TimeoutError("requests did not complete")
            for d in self.poll(1024, 100_000):
                got[int(d["ticket"])] = d
        return got

    def replay(self, arrivals, lam: float, sigma_u):
        """Real-time replay of ``arrivals`` = [(t_s, agent, K, T), ...] (sorted by time).

        Returns (completion records, number of dropped arrivals)."""
        n = len(arrivals)
        arr = (_lib.ServeArrivalC * max(n, 1))()
        for i, (t, a, K, T) in enumerate(arrivals):
            arr[i] = _lib.ServeArrivalC(int(round(t * 1e9)), int(a), int(K), int(T))
        proto, _ = self._request(0, 1, 1, lam, sigma_u, None, False)
        done = (_lib.ServeDoneC * max(n, 1))()
        nd, ndrop = ctypes.c_int(), ctypes.c_int()
        check(self._lib.pi_server_replay(self._h, arr, n, ctypes.byref(proto), done, ctypes.byref(nd),
                                         ctypes.byref(ndrop)))
        return _done_array(done, nd.value), int(ndrop.value)

    def state_save(self):
        na = self.n_agents
        x0 = np.empty((na, NX), np.float32)
        w = np.empty((na, self.T_max, NU), np.float32)
        ctr = np.empty(na, np.uint64)
        sd = np.empty(na, np.uint64)
        fp, up = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64)
        check(self._lib.pi_server_state_save(self._h, x0.ctypes.data_as(fp), w.ctypes.data_as(fp),
                                             ctr.ctypes.data_as(up), sd.ctypes.data_as(up)))
        return {"x0": x0, "u_warm": w, "counter": ctr, "seed": sd}

    def state_load(self, state: dict):
        fp, up = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64)
        x0 = np.ascontiguousarray(state["x0"], np.float32)
        w = np.ascontiguousarray(state["u_warm"], np.float32)
        ctr = np.ascontiguousarray(state["counter"], np.uint64)
        sd = np.ascontiguousarray(state["seed"], np.uint64)
        check(self._lib.pi_server_state_load(self._h, x0.ctypes.data_as(fp), w.ctypes.data_as(fp),
                                             ctr.ctypes.data_as(up), sd.ctypes.data_as(up)))

    def stats(self) -> dict:
        s = _lib.ServerStatsC()
        check(self._lib.pi_server_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pipe_rates(device: int = 0) -> dict:
    """Measured FFMA2 TFLOP/s and MUFU ex2 results/s of the device (see pi_debug_pipe_rates)."""
    lib = _lib.load()
    f, e = ctypes.c_double(), ctypes.c_double()
    check(lib.pi_debug_pipe_rates(int(device), ctypes.byref(f), ctypes.byref(e)))
    return {"ffma_tflops": f.value, "ex2_per_s": e.value}


def fp64_rate(device: int = 0) -> float:
    """Measured FP64 FMA lane results per second of the device (see pi_debug_fp64_rate)."""
    lib = _lib.load()
    r = ctypes.c_double()
    check(lib.pi_debug_fp64_rate(int(device), ctypes.byref(r)))
    return r.value


def debug_pool(capacity: int, ops):
    """Runs the serving pool allocator on the host: ops = [("alloc", nbytes) | ("free", op_index)].

    Returns (offsets, free_extents); offsets[i] is the allocation's offset, -1 if it did not fit,
    or the freed block's offset for a free."""
    lib = _lib.load()
    n = len(ops)
    op = np.array([1 if k == "alloc" else 0 for k, _ in ops], np.int32)
    sz = np.array([v for _, v in ops], np.uint64)
    off = np.zeros(max(n, 1), np.int64)
    ext = ctypes.c_int()
    check(lib.pi_debug_pool(int(capacity), op.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            sz.ctypes.data_as(ctypes.POINTER(ctypes.c_size_t)), n,
                            off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(ext)))
    return off[:n], int(ext.value)

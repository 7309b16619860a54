#!/usr/bin/env python3
"""Benchmark of the PI^2-RH / LWPR update on one B300.

Workload (default ``realtime``): K=8192 rollouts, T=100 steps, L=512 receptive
fields per output (12 outputs over a 16-dim input), 16 cylinder obstacles; a
receding-horizon loop of ``--steps`` iterations (20 by default), each one
``pi_update`` (seed = seed + iteration) followed by ``pi_rh_advance`` (plant
step with the first control, warm-start shift of the plan).  Synthetic inputs
from the seeded generator; everything is resident in HBM before timing.

Prints ONE JSON line (rank 0).  ``value`` = rollout-steps/s (K*T*M per update)
over the timed iterations, device-timed with CUDA events on the launching
stream; ``e2e`` is the same metric through ``pi_update_host`` (host buffers,
copies inside the timed region); ``roofline`` is the rollout kernel's FP32
rate from per-launch event times; ``cpu_baseline`` is the FP64 oracle timed on
a bounded sample of the same workload.

At N=1 the default line also carries, beside the FP32 headline:
  * ``forms``: the realtime loop in the tensor-core forms (three and two split
    products), each with its roofline, clocks and error against the oracle;
  * ``precision_workload``: K=65536, T=100, L=2048 (conditioned D) in every form;
  * ``batched_workload``: 64 uneven controllers in one graph-captured launch,
    every form;
  * ``serving_workload``: 256 quadrotors at 50 Hz through the continuous-batching
    server (throughput, capacity, p50/p99 latency saturated and at half load).
Each form's error is measured on the workload's seed-0 update against the
oracle run that the CPU-baseline leg times (so the oracle runs nowhere else).

``--impl reference`` times the oracle itself (there is no reference
implementation of the paper's method other than the oracle written from it).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LWPR rollout-steps/s (ms per PI^2 update alongside)"
PAPER_CONTEXT = ("paper (context only, other hardware and a ~1000x smaller model): one PI^2 iteration of "
                 "1000 rollouts x 50 steps in ~6.5 ms on a GTX 780 Ti (~7.7e6 rollout-steps/s), 18 ms with 32 "
                 "sub-rollouts, for an LWPR model of 3 outputs x 15-24 fields over 4 inputs")
UNIT = "rollout-steps/s"
FLOPS_PER_FIELD = 360          # 16 sub + 136 FMA + 16 FMA + 16 FMA + 4 FMA (x2 flops per FMA)
FP32_LANES_PER_SM = 128
L2_BYTES = 126 * 2**20
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def profile_traffic(name: str):
    """Per-launch DRAM bytes recorded in a committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", f.read())
        return float(m.group(1)) if m else None
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]),
                                     float(parts[3].split()[0]) if parts[3][0].isdigit() else 0.0,
                                     parts[5], parts[6], parts[7], parts[8]))
                    except (ValueError, IndexError):
                        continue
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        power = [r[2] for r in rows]
        pmax = max(power)
        loaded = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in loaded for n, v in zip(names, r[3:]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(loaded), "power_w_max": pmax}


def workload(name: str, seed: int):
    from paper_1503_00330_b300 import workloads as W
    if name == "realtime":
        return W.realtime(seed), "realtime: K=8192 rollouts, T=100 steps, L=512 fields x 12 outputs, " \
                                 "16 cylinder obstacles, receding-horizon loop with warm-start shift"
    if name == "realtime_short":
        p = W.realtime(seed)
        p.T = 10
        p.u_nom = p.u_nom[:10].copy()
        return p, "realtime_short (profiling case): K=8192, T=10, L=512 x 12 outputs, 16 obstacles"
    if name == "precision_short":
        p = W.precision(seed)
        p.T = 5
        p.u_nom = p.u_nom[:5].copy()
        return p, "precision_short (profiling case): K=65536, T=5, L=2048 x 12 outputs, cond(D) logU[1,1e3]"
    if name == "small":
        return W.small(seed), "small: K=256, T=50, L=64 x 12 outputs, 4 obstacles"
    if name == "precision":
        return W.precision(seed), "precision: K=65536, T=100, L=2048 x 12 outputs, cond(D) logU[1,1e3]"
    if name == "subrollouts":
        # the paper's largest model-uncertainty setting (1000 rollouts x 32 sub-rollouts x 50 steps)
        # on the realtime model; a rollout-step here counts every sub-rollout step
        p = W.problem(1024, 50, 512, seed, n_obs=16, M=32)
        return p, "subrollouts: K=1024 rollouts x M=32 sub-rollouts, T=50, L=512 x 12 outputs, 16 obstacles"
    raise SystemExit(f"unknown workload {name}")


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo"
    dist.init_process_group(backend)
    return rank, ws, local, dist


def job_throughput(dist, units: float, seconds: float, device="cpu") -> float:
    """Whole-job rate of independent replicas: the units every rank processed,
    summed, over the slowest rank's time."""
    if dist is None:
        return units / seconds
    import torch
    u = torch.tensor([units], dtype=torch.float64, device=device)
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(t.item())


def reduce_max(dist, v: float, device):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(p, k_sample: int, k_single: int = 32):
    """FP64 oracle on one update of the workload's seed-0 inputs with the first
    k_sample / M rollouts (all host threads), and on k_single rollouts on one
    thread.  The sample's results are returned too: they are the reference the
    per-form errors are measured against (rollout k depends only on its own noise
    counters, so rollouts 0..k_sample-1 of the full-size launch are the sample's)."""
    from oracle import oracle as O
    O.build()
    k_sample = max(1, k_sample // max(p.M, 1))
    t0 = time.perf_counter()
    u, S0 = O.pi_update(p.model, p.cost, p.x0, p.u_nom, k_sample, p.T, p.lam, p.sigma_u, p.seed, M=p.M,
                        model_noise=p.model_noise)
    el = time.perf_counter() - t0
    cores = O.max_threads()
    k1 = max(min(k_single, k_sample), 1)
    O.set_threads(1)
    try:
        t1 = time.perf_counter()
        O.pi_update(p.model, p.cost, p.x0, p.u_nom, k1, p.T, p.lam, p.sigma_u, p.seed, M=p.M,
                    model_noise=p.model_noise)
        el1 = time.perf_counter() - t1
    finally:
        O.set_threads(cores)
    base = {"value": k_sample * p.T * p.M / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one update of {k_sample} of the {p.K} rollouts (T={p.T}, L={p.model.L}, M={p.M}; "
                      f"seed-0 inputs), {el:.2f} s",
            "single_thread": {"value": k1 * p.T * p.M / el1, "sample": f"{k1} rollouts on 1 thread, {el1:.2f} s"}}
    return base, {"K": k_sample, "u": u, "S0": S0}


def form_errors(p, form, ref, dev):
    """Error of each form against the FP64 oracle on the workload's seed-0 inputs (x0 = 0,
    u_nom = 0, seed = workload seed), on the same context kind the bench times:
      * costs S_{k,0} of rollouts 0..Ks-1 of the full-size launch (the bench's launch
        configuration), against the oracle's sample update of Ks rollouts;
      * u_out (per channel, max_t |du| / max_t |u_ref|) and every cost of a Ks-rollout
        update against the same oracle update.
    A rollout whose cost differs by at least half an obstacle step (w_obs dt) is counted as
    an indicator flip (the oracle decides the crash indicator on its FP64 state, the kernels
    on their FP32 state) and reported apart."""
    import torch
    from paper_1503_00330_b300.api import Controller
    Ks = ref["K"]
    ctl = Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, device=dev.index, precision=form)
    ctl.reserve(p.K, p.T)
    x0 = torch.as_tensor(p.x0, device=dev)
    un = torch.as_tensor(p.u_nom, device=dev)
    _, c_full = ctl.update(x0, un, p.K, p.T, p.lam, p.sigma_u, p.seed)
    u_s, c_s = ctl.update(x0, un, Ks, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    S0 = np.asarray(ref["S0"], np.float64)
    flip = 0.5 * float(p.cost.w_obs) * float(p.model.dt) / p.M
    out = {}
    for name, c in (("costs_full_launch", c_full.cpu().numpy()[:Ks]), ("costs_sample_update", c_s.cpu().numpy())):
        d = np.abs(c.astype(np.float64) - S0)
        ok = d < flip
        out[name] = {"rel_err_max": float(np.max(d[ok] / np.abs(S0[ok]))) if ok.any() else None,
                     "rollouts": int(Ks), "indicator_flips": int((~ok).sum())}
    uref = np.asarray(ref["u"], np.float64)
    eu = np.abs(u_s.cpu().numpy().astype(np.float64) - uref).max(0) / np.abs(uref).max(0)
    out["u_out_rel_err_per_channel"] = [float(e) for e in eu]
    out["u_out_rel_err_max"] = float(eu.max())
    out["reference"] = (f"FP64 oracle, one update of the first {Ks} rollouts (the CPU-baseline sample); "
                        f"costs also against rollouts 0..{Ks - 1} of the full K={p.K} launch")
    ctl.close()
    return out


def batched_cpu_baseline(probs, pick, n):
    """FP64 oracle on the first n rollouts of the controllers in `pick` of the batched
    workload (their seed-0 inputs), timed on all host threads; the results are the
    reference of the batched errors (rollout k of a controller depends only on its own
    noise counters)."""
    from oracle import oracle as O
    O.build()
    ref, steps, el = {}, 0, 0.0
    for i in pick:
        p = probs[i]
        t0 = time.perf_counter()
        r = O.rollouts(p.model, p.cost, p.x0, p.u_nom, n, p.T, p.sigma_u, p.seed, M=p.M, model_noise=p.model_noise)
        ref[i] = O.cost_to_go(r["cost"], r["phi"], float(p.model.dt))[:, 0]
        el += time.perf_counter() - t0
        steps += n * p.T * p.M
    return ({"value": steps / el, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
             "sample": "the first {} rollouts of controllers {} (K, T, L = {}), {:.2f} s".format(
                 n, list(pick), [(probs[i].K, probs[i].T, probs[i].model.L) for i in pick], el)}, ref)


def batched_errors(probs, costs, ref):
    """costs_out S_{k,0} of the sampled rollouts of each picked controller, from one batched
    update of the seed-0 inputs, against the oracle (relative, max over the sample)."""
    out = {}
    for i, S0 in ref.items():
        c = costs[i][:len(S0)]
        out[f"controller_{i}"] = {"costs_rel_err_max": float(np.max(np.abs(c - S0) / np.abs(S0))),
                                  "rollouts": int(len(S0)), "K": probs[i].K, "T": probs[i].T, "L": probs[i].model.L}
    out["costs_rel_err_max"] = max(v["costs_rel_err_max"] for v in out.values())
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    p, desc = workload(args.workload, 0)
    O.build()
    k_s = args.ref_sample
    u_nom = p.u_nom.astype(np.float64)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        u, _ = O.pi_update(p.model, p.cost, p.x0, u_nom, k_s, p.T, p.lam, p.sigma_u, p.seed + it, M=p.M,
                           model_noise=p.model_noise)
        el = time.perf_counter() - t0
        u_nom = np.concatenate([u[1:], u[-1:]], 0)
        if it >= args.warmup:
            times.append(el)
    total = sum(times)
    value = k_s * p.T * p.M * args.steps / total
    cores = O.max_threads()
    sample = f"each step: one update of {k_s} of the {p.K} rollouts (T={p.T}, L={p.model.L})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "K": p.K, "T": p.T, "L": p.model.L, "M": p.M,
                                            "sample_K": k_s},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Timed steps enqueued back to back before their stage times are read (at most the
# context's ring of stage-event sets, 64)
TIMING_CHUNK = 32
# Stated accuracy of each form against the FP64 oracle (u_out per channel and costs, relative)
ERROR_BOUND = {"fp32": 1e-5, "tc": 2e-3, "tc_fp16x2": 2e-3}
FORMS = ("fp32", "tc", "tc_fp16x2")
SPLIT_MODE = ["auto"]   # --split: launch of the FP32 rollout kernel (set in main)
TC_FIELDS_PER_TILE = 128                      # fields per tensor-core tile (MMA N)
# Issued MMA flops per field (2 per multiply-add): K step 0 of the exponent GEMM and the K=16
# prediction GEMM with 3 split products; the 128 quadratic features (K steps 1-8) with 3
# (tc) or 2 (tc_fp16x2); K step 9 (8 quadratic features, the constant, padding) with 3.
TC_MMA_FLOPS_PER_FIELD = {"tc": 2 * (3 * (16 + 16) + 3 * 128 + 3 * 16),
                          "tc_fp16x2": 2 * (3 * (16 + 16) + 2 * 128 + 3 * 16)}


def tensor_peak(peaks, clocks):
    """Dense bf16 tensor peak for a run with the given clock record: the seconds-long
    sustained figure when the run was held down by the power cap (sw_power_cap active and
    the median SM clock under load below 95 % of the maximum, as in the sustained GEMM
    loop), else the burst figure (the kernel ran at full clock, as the burst GEMM did)."""
    clocks = clocks or {}
    capped = "sw_power_cap" in (clocks.get("reasons") or [])
    mhz, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    held = capped and mhz is not None and mx and float(mhz) < 0.95 * float(mx)
    if held:
        return float(peaks.get("bf16_tflops_sustained", 1366.3)), \
            f"measured dense bf16 sustained (sw_power_cap, median SM clock {float(mhz):.0f} MHz under load)"
    note = "no power cap" if not capped else f"sw_power_cap flagged, median SM clock {float(mhz):.0f} MHz"
    return float(peaks.get("bf16_tflops", 1788.7)), f"measured dense bf16 burst ({note} in the run's clock record)"


def clock_scaled(peaks, clocks, achieved):
    """The burst tensor peak scaled to the run's median SM clock (the burst GEMM ran at the
    maximum clock), with the achieved rate's fraction of it.  A run that the power cap held
    well above the sustained loop's clock can exceed the sustained figure; this view shows
    how close it came to the tensor core's rate at the clock it actually ran at."""
    clocks = clocks or {}
    mhz, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2032.0)
    if mhz is None or not mx:
        return None
    peak = float(peaks.get("bf16_tflops", 1788.7)) * float(mhz) / float(mx)
    return {"peak": peak, "frac": achieved / peak, "sm_mhz": float(mhz),
            "basis": "measured dense bf16 burst x median SM clock / max SM clock"}


def fp32_launch(ctl, K):
    """(kernel name, ncu summary file stem) of the FP32 rollout launch for K rollouts."""
    plain, upc, ctas = ctl.split_plan(K)
    if upc and not plain:
        return (f"rollout_fp32_split_kernel (output-split launch: {ctas} CTAs x {upc} (block, output) units)",
                "rollout_fp32_split")
    if upc:
        return (f"rollout_fp32_kernel ({plain} CTAs, one per 64-slot block) + rollout_fp32_split_kernel "
                f"(the last partial wave: {ctas} CTAs x {upc} units)", "rollout_fp32")
    return f"rollout_fp32_kernel ({plain} CTAs, one per 64-slot block)", "rollout_fp32"


def form_roofline(precision, rollout_ms, K, T, M, L, dev, peaks, workload, clocks=None, launch=None):
    """Roofline of the rollout kernel from its per-launch CUDA-event times.
    launch: fp32_launch() of the FP32 form (kernel name, summary stem)."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    avg_s = statistics.mean(rollout_ms) / 1e3
    useful = float(K) * T * M * 12 * L * FLOPS_PER_FIELD
    if precision == "fp32":
        sm_max_mhz = float(peaks.get("sm_max_mhz", 2032.0))
        peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
        achieved = useful / avg_s / 1e12
        kname, stem = launch or ("rollout_fp32_kernel", "rollout_fp32")
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profile_traffic(f"{stem}_{workload}.md"), "kernel": kname,
                "peak_basis": f"FP32 FMA pipe: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} lanes x 2 flop "
                              f"x {sm_max_mhz:.0f} MHz (max SM clock)",
                "rollout_ms_per_launch": statistics.mean(rollout_ms)}
    L_pad = -(-L // TC_FIELDS_PER_TILE) * TC_FIELDS_PER_TILE
    per_field = TC_MMA_FLOPS_PER_FIELD[precision]
    issued = float(K) * T * M * 12 * L_pad * per_field
    peak, basis = tensor_peak(peaks, clocks)
    achieved = issued / avg_s / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": profile_traffic(f"rollout_tc_{workload}.md") if precision == "tc" else None,
            "kernel": "rollout_tc_kernel" + ("" if precision == "tc" else " (2 split products on the quadratic features)"),
            "peak_basis": basis + f"; fp16 has the same nominal rate; achieved counts the issued fp16 MMA "
                                  f"flops ({per_field} per field, fields padded to 128-field tiles)",
            "useful_tflops": useful / avg_s / 1e12, "useful_frac": useful / avg_s / 1e12 / peak,
            "useful_basis": f"{FLOPS_PER_FIELD} algorithmic flop per field evaluation (the FP32 form's count)",
            "at_run_clock": clock_scaled(peaks, clocks, achieved),
            "rollout_ms_per_launch": statistics.mean(rollout_ms)}


_PIPE_RATES = {}


def pipe_peaks(device: int) -> dict:
    """Measured FFMA2 and MUFU ex2 rates of the device (probed once per process)."""
    if device not in _PIPE_RATES:
        from paper_1503_00330_b300.api import pipe_rates
        _PIPE_RATES[device] = pipe_rates(device)
    return _PIPE_RATES[device]


def mufu_check(precision, rollout_ms, K, T, M, L, device):
    """The rollout kernel's secondary pipe: MUFU ex2 results per launch against the measured
    ex2 rate.  FP32 form: 3 per field pair and slot (the rescale and the two weights); tensor-core
    form: 1 per field evaluation (padded to 128-field tiles) and 1 per 16-field chunk (rescale)."""
    avg_s = statistics.mean(rollout_ms) / 1e3
    if precision == "fp32":
        per_slot_step = 12 * (-(-L // 2)) * 3
        binding = "FP32 FMA pipe"
    else:
        L_pad = -(-L // TC_FIELDS_PER_TILE) * TC_FIELDS_PER_TILE
        per_slot_step = 12 * L_pad * 17 / 16
        binding = "tensor pipe (MMA issue)"
    n = float(K) * T * M * per_slot_step
    rate = float(pipe_peaks(device)["ex2_per_s"])
    return {"pipe": "MUFU ex2", "achieved": n / avg_s, "peak": rate, "unit": "ex2/s", "frac": n / avg_s / rate,
            "ex2_per_launch": n, "binding_pipe": binding}


# FP64-pipe instructions per rollout-step in the scan (lane level): convert and
# FMA for the suffix sum, subtract, multiply and convert for the exponent.
SCAN_FP64_PER_ROLLOUT_STEP = 5
_FP64_RATE = {}


def fp64_peak(device: int) -> float:
    """Measured FP64 FMA lane results/s of the device (probed once per process)."""
    if device not in _FP64_RATE:
        from paper_1503_00330_b300.api import fp64_rate
        _FP64_RATE[device] = fp64_rate(device)
    return _FP64_RATE[device]


def reduction_rooflines(scan_ms, merge_ms, K, T, peaks, device=0):
    """Rooflines of the cost-to-go/LSE scan and of the merge.

    The scan is bound by B300's FP64 pipe (ncu: FP64 pipe busy ~62 % of active cycles, DRAM
    ~9 %): its roofline counts SCAN_FP64_PER_ROLLOUT_STEP FP64 instructions per rollout-step
    against the measured DFMA rate, with its bandwidth beside it.  The merge is a small,
    latency-bound launch; its bandwidth is given.  Bytes are algorithmic: the scan reads cost
    [T][K] f32 and eps [T][K] float4 and phi [K], writes costs_out [K] and the LSE partials
    [K/64][T][6] f64; the merge reads the partials and u_nom [T][4] and writes u_out [T][4].
    Their inputs were written by the rollout kernel just before (about 20 B per
    rollout-step), so they are mostly L2-resident: the bandwidth fraction is given against the
    measured HBM copy peak, and can exceed what DRAM alone would allow."""
    nblk = -(-K // 64)
    scan_b = K * T * 20 + K * 8 + nblk * T * 48
    merge_b = nblk * T * 48 + T * 32
    hbm = float(peaks.get("hbm_gbs", 6492.1))
    out = {}
    for name, ms, b in (("scan_lse_kernel", scan_ms, scan_b), ("lse_merge_kernel", merge_ms, merge_b)):
        avg = statistics.mean(ms)
        gbs = b / (avg / 1e3) / 1e9
        bw = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
              "bytes_per_launch": b, "ms_per_launch": avg,
              "data": "inputs written by the rollout kernel just before (L2-resident for this size)"}
        if name == "scan_lse_kernel":
            ops = SCAN_FP64_PER_ROLLOUT_STEP * K * T
            rate = fp64_peak(device)
            achieved = ops / (avg / 1e3)
            out[name] = {"bound": "fp64", "achieved": achieved / 1e9, "peak": rate / 1e9,
                         "unit": "G FP64 instr/s", "frac": achieved / rate, "fp64_instr_per_launch": ops,
                         "ms_per_launch": avg,
                         "peak_basis": "measured DFMA lane rate (pi_debug_fp64_rate); "
                                       f"{SCAN_FP64_PER_ROLLOUT_STEP} FP64 instructions per rollout-step",
                         "hbm_view": bw}
        else:
            out[name] = bw
    return out


def plant_step_roofline(plant_ms, L, peaks, precision):
    """The plant step of the receding-horizon loop (``pi_rh_advance``: rh_build_z, the
    clustered prediction kernel, rh_apply), timed with CUDA events on the launching
    stream.  Its algorithmic bytes are one read of the FP32 field-pair records of the 12
    outputs (1376 B per pair of fields; the second, re-centred pass re-reads them from
    shared memory when L <= 512, from L2 otherwise).  It is a small launch, bound by
    latency: the fraction is given against the measured HBM copy peak."""
    recs = 12 * ((L + 1) // 2) * 1376
    hbm = float(peaks.get("hbm_gbs", 6492.1))
    avg = statistics.mean(plant_ms)
    gbs = recs / (avg / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "bytes_per_launch": recs, "ms_per_launch": avg, "launches_per_step": 3,
            "kernel": "rh_build_z + predict_rows_kernel + rh_apply",
            "data": ("records last read by the rollout kernel (L2-resident)" if precision == "fp32" else
                     "records not read by the tensor-core rollout, so they come from DRAM after the L2 flush")}


def time_form(precision, p, args, dev):
    """The receding-horizon loop of `p` timed the same way with the other form."""
    import torch
    from paper_1503_00330_b300.api import Controller
    K, T, M, L = p.K, p.T, p.M, p.model.L
    ctl = Controller(p.model, p.cost, M=M, model_noise=p.model_noise, device=dev.index, precision=precision)
    launch = None
    if precision == "fp32":
        ctl.set_output_split(SPLIT_MODE[0])
        launch = fp32_launch(ctl, K)
    ctl.set_timing(True)
    ctl.reserve(K, T)
    x0 = torch.as_tensor(p.x0, device=dev).clone()
    ua = torch.as_tensor(p.u_nom, device=dev).clone()
    ub = torch.empty_like(ua)
    costs = torch.empty(K, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rollout_ms, step_ms, scan_ms, merge_ms, plant_ms = [], [], [], [], []
    for i in range(args.warmup):
        ctl.update(x0, ua, K, T, p.lam, p.sigma_u, p.seed + i, u_out=ub, costs_out=costs)
        ctl.rh_advance(x0, ub, ua)
    ctl.sync()
    sampler = ClockSampler(dev.index or 0)
    sampler.__enter__()
    for c0 in range(0, args.steps, TIMING_CHUNK):     # enqueued back to back, as in the headline loop
        c1 = min(args.steps, c0 + TIMING_CHUNK)
        evs = []
        for i in range(c0, c1):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctl.update(x0, ua, K, T, p.lam, p.sigma_u, p.seed + args.warmup + i, u_out=ub, costs_out=costs)
            pa.record(stream)
            ctl.rh_advance(x0, ub, ua)
            pb.record(stream)
            b.record(stream)
            evs.append((a, b, pa, pb))
        for i, (a, b, pa, pb) in zip(range(c0, c1), evs):
            st = ctl.stage_times(back=c1 - 1 - i)
            b.synchronize()
            rollout_ms.append(st[0])
            scan_ms.append(st[1])
            merge_ms.append(st[2])
            step_ms.append(a.elapsed_time(b))
            plant_ms.append(pa.elapsed_time(pb))
    sampler.__exit__(None, None, None)
    clk = sampler.summary()
    ctl.sync()
    ctl.close()
    total_s = sum(step_ms) / 1e3
    roof = form_roofline(precision, rollout_ms, K, T, M, L, dev, measured_peaks(), args.workload, clocks=clk,
                         launch=launch)
    roof["rollout_share_of_step"] = sum(rollout_ms) / sum(step_ms)
    roof["secondary"] = mufu_check(precision, rollout_ms, K, T, M, L, dev.index or 0)
    return {"value": K * T * M * args.steps / total_s, "ms_per_update": 1e3 * total_s / args.steps,
            "ms_per_update_stats": {"best": min(step_ms), "median": statistics.median(step_ms), "n": len(step_ms)},
            "roofline": roof, "reduction": {**reduction_rooflines(scan_ms, merge_ms, K, T, measured_peaks(), dev.index or 0),
                                            "plant_step": plant_step_roofline(plant_ms, L, measured_peaks(), precision)},
            "clocks": clk}


def time_updates(precision, p, steps, warmup, dev, workload):
    """Plain pi_update calls of `p` (no receding-horizon step), device-timed with CUDA events
    on the launching stream, L2 flushed outside each event window, clocks sampled."""
    import torch
    from paper_1503_00330_b300.api import Controller
    K, T, M, L = p.K, p.T, p.M, p.model.L
    ctl = Controller(p.model, p.cost, M=M, model_noise=p.model_noise, device=dev.index, precision=precision)
    launch = None
    if precision == "fp32":
        ctl.set_output_split(SPLIT_MODE[0])
        launch = fp32_launch(ctl, K)
    ctl.set_timing(True)
    ctl.reserve(K, T)
    x0 = torch.as_tensor(p.x0, device=dev).clone()
    un = torch.as_tensor(p.u_nom, device=dev).clone()
    u = torch.empty_like(un)
    costs = torch.empty(K, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for i in range(warmup):
        ctl.update(x0, un, K, T, p.lam, p.sigma_u, p.seed + i, u_out=u, costs_out=costs)
    ctl.sync()
    rollout_ms, step_ms, scan_ms, merge_ms = [], [], [], []
    launches0 = ctl.launch_count()
    with ClockSampler(dev.index or 0) as clocks:
        for c0 in range(0, steps, TIMING_CHUNK):       # enqueued back to back, as in the headline loop
            c1 = min(steps, c0 + TIMING_CHUNK)
            evs = []
            for i in range(c0, c1):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctl.update(x0, un, K, T, p.lam, p.sigma_u, p.seed + warmup + i, u_out=u, costs_out=costs)
                b.record(stream)
                evs.append((a, b))
            for i, (a, b) in zip(range(c0, c1), evs):
                st = ctl.stage_times(back=c1 - 1 - i)
                b.synchronize()
                rollout_ms.append(st[0])
                scan_ms.append(st[1])
                merge_ms.append(st[2])
                step_ms.append(a.elapsed_time(b))
    launches = ctl.launch_count() - launches0
    ctl.sync()
    ctl.close()
    clk = clocks.summary()
    total_s = sum(step_ms) / 1e3
    roof = form_roofline(precision, rollout_ms, K, T, M, L, dev, measured_peaks(), workload, clocks=clk,
                         launch=launch)
    roof["rollout_share_of_step"] = sum(rollout_ms) / sum(step_ms)
    roof["secondary"] = mufu_check(precision, rollout_ms, K, T, M, L, dev.index or 0)
    return {"value": K * T * M * steps / total_s, "ms_per_update": 1e3 * total_s / steps, "steps": steps,
            "warmup": warmup,
            "ms_per_update_stats": {"best": min(step_ms), "median": statistics.median(step_ms), "n": len(step_ms)},
            "gpu_launches": launches, "roofline": roof,
            "reduction": reduction_rooflines(scan_ms, merge_ms, K, T, measured_peaks(), dev.index or 0),
            "clocks": clk}


BATCHED_SCHEDULE = {"fp32": ("longest_first", 1), "tc": ("longest_first", 1), "tc_fp16x2": ("longest_first", 1)}


def batched_forms(probs, sched, order, steps, warmup, dev, pick=()):
    """Times one batched update of `probs` per form in `order` (schedule per form from
    `sched`), with CUDA events on the launching stream and L2 flushed between timed
    updates.  For the controllers in `pick`, also returns each form's costs_out of one
    update with the controllers' own seeds (the seed-0 inputs) for the error check."""
    import torch
    from paper_1503_00330_b300.api import Batch, Controller
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    forms, costs = {}, {}
    for form in order:
        ctls = [Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, precision=form) for p in probs]
        batch = Batch(ctls, [p.K for p in probs], [p.T for p in probs], precision=form,
                      x0=[p.x0 for p in probs], u_nom=[p.u_nom for p in probs])
        batch.set_schedule(sched[form][0])
        batch.set_tile(sched[form][1])
        lam = [p.lam for p in probs]
        su = [p.sigma_u for p in probs]
        for i in range(warmup):
            batch.update(lam, su, [p.seed + i for p in probs])
        batch.sync()
        ms = []
        launches0 = batch.launch_count()
        with ClockSampler(dev.index or 0) as clocks:
            for i in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                batch.update(lam, su, [p.seed + warmup + i for p in probs])
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        batch.sync()
        launches = batch.launch_count() - launches0
        if pick:
            _, c_b = batch.update(lam, su, [p.seed for p in probs])
            batch.sync()
            costs[form] = {i: c_b[i].cpu().numpy().astype(np.float64) for i in pick}
        rs = batch.rollout_steps()
        useful = sum(p.K * p.T * p.M * 12 * p.model.L for p in probs) * FLOPS_PER_FIELD
        entry = {"value": rs * steps / (sum(ms) / 1e3), "ms_per_update": statistics.mean(ms), "steps": steps,
                 "schedule": {"order": sched[form][0], "tile": sched[form][1]},
                 "gpu_launches": launches, "clocks": clocks.summary()}
        if form == "fp32":
            peak = torch.cuda.get_device_properties(dev).multi_processor_count * FP32_LANES_PER_SM * 2 * \
                float(measured_peaks().get("sm_max_mhz", 2032.0)) * 1e6 / 1e12
            ach = useful / (statistics.mean(ms) / 1e3) / 1e12
            kern = "rollout_fp32_batch_kernel" if sched[form][1] == 0 else "rollout_fp32_group_kernel"
            entry["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                                 "kernel": kern + " (time of the whole batched update)"}
        else:
            issued = sum(p.K * p.T * p.M * 12 * (-(-p.model.L // TC_FIELDS_PER_TILE) * TC_FIELDS_PER_TILE)
                         for p in probs) * TC_MMA_FLOPS_PER_FIELD[form]
            peak, basis = tensor_peak(measured_peaks(), entry["clocks"])
            ach = issued / (statistics.mean(ms) / 1e3) / 1e12
            uf = useful / (statistics.mean(ms) / 1e3) / 1e12
            entry["roofline"] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                 "frac": ach / peak, "useful_tflops": uf, "useful_frac": uf / peak,
                                 "peak_basis": basis,
                                 "at_run_clock": clock_scaled(measured_peaks(), entry["clocks"], ach),
                                 "kernel": ("rollout_tc_batch_kernel" if sched[form][1] == 0 else "rollout_tc_group_kernel")
                                           + " (time of the whole batched update)"}
        forms[form] = entry
        batch.close()
        for c in ctls:
            c.close()
    return forms, costs


def run_batched(args):
    """64 independent controllers (K ~ logU[1024, 32768], T ~ U{30..150},
    L ~ logU[128, 2048], own model/obstacles/seed each) updated by one
    batched launch under a CUDA graph; every form timed, each with the
    work-list order and (tensor cores) tile shape the autotuner picks."""
    import torch
    from paper_1503_00330_b300 import build
    from paper_1503_00330_b300 import workloads as W
    build.build()
    dev = torch.device("cuda", 0)
    probs = W.batched(64, seed=0)
    # schedule per form from the autotuner (JSON-cached by batch shape), unless fixed on the command line
    sched = {"fp32": ("longest_first", min(args.batch_tile, 1)), "tc": ("longest_first", args.batch_tile),
             "tc_fp16x2": ("longest_first", args.batch_tile)}
    tuned = None
    if args.batch_tile < 0:
        from paper_1503_00330_b300 import autotune
        tuned = autotune.tune(probs, reps=2)
        best = {}
        for key, ms in tuned["candidates"].items():   # "form/order/tile" -> ms per update
            f, o, t = key.split("/")
            if f not in best or ms < best[f][2]:
                best[f] = (o, int(t), ms)
        sched = {f: (o, t) for f, (o, t, _) in best.items()}
        sched["tc_fp16x2"] = sched["tc"]      # the same kernel with fewer MMAs: the tensor-core pick
    order = [args.precision] + ([] if args.no_compare else [f for f in FORMS if f != args.precision])
    forms, _ = batched_forms(probs, sched, order, args.steps, args.warmup, dev)
    main = forms[args.precision]
    rs_total = sum(p.K * p.T * p.M for p in probs)
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_update"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator)",
            "config": {"workload": "batched: 64 controllers, K ~ logU[1024, 32768], T ~ U{30..150}, "
                                   "L ~ logU[128, 2048], one persistent launch under a CUDA graph",
                       "controllers": len(probs), "rollout_steps_per_update": rs_total,
                       "precision": args.precision,
                       "schedule": "per form, from the autotuner" if tuned else "fixed on the command line",
                       "l2": "flushed between timed steps (256 MiB write outside the event window)"},
            "gpu_launches": main["gpu_launches"], "roofline": main["roofline"], "forms": forms,
            "autotune": None if tuned is None else {"best": {k: tuned[k] for k in ("form", "order", "tile", "ms")},
                                                    "cached": tuned["cached"], "candidates_ms": tuned["candidates"]},
            "clocks": main["clocks"]}
    print(json.dumps(line), flush=True)


SERVING_WORKLOAD = ("serving: 256 quadrotors, Poisson 50 Hz each, K ~ U{2048..16384}, T ~ U{50..120}, "
                    "shared LWPR model L=1024, continuous batching")


def serving_measure(precision, serve_seconds, sweep_loads, lanes, max_group, warmup):
    """256 simulated quadrotors over one shared LWPR model (L = 1024 fields per
    output): each issues update requests as a Poisson process with
    K ~ U{2048..16384}, T ~ U{50..120}; the continuous-batching server admits
    them by free lanes and pool memory.  A quadrotor whose previous plan has not
    come back skips its tick (the arrival is dropped).  Timed at the offered
    50 Hz (far above what one GPU serves at these sizes, so the server runs
    saturated), at half the capacity measured in that run (the latency of a
    loaded but stable server), and at the other loads of `sweep_loads`.
    Returns (at the offered rate, at half capacity, sweep points, capacity)."""
    import numpy as np
    import torch
    from paper_1503_00330_b300 import workloads as W
    from paper_1503_00330_b300.api import Controller, Server
    n_quad, L, lam = 256, 1024, 1.0
    model = W.make_lwpr(L, seed=4)
    cost = W.make_cost(16, seed=4)
    ctl = Controller(model, cost, precision=precision)
    srv = Server(ctl, n_quad, K_max=16384, T_max=120, max_inflight=lanes, max_group=max_group)
    rng = np.random.default_rng(5)
    for a in range(n_quad):
        srv.set_agent(a, rng.normal(0, 0.1, 12).astype(np.float32), None, seed=1000 + a)
    for i in range(warmup):                           # warm-up requests (one per agent 0..W-1)
        srv.submit(i, 4096, 100, lam, W.SIGMA_U, keep=False)
    srv.drain()
    srv.poll(1 << 16)
    L_pad = -(-L // TC_FIELDS_PER_TILE) * TC_FIELDS_PER_TILE

    def run(rate_hz, seconds, seed):
        trace = W.serving_requests(n_quad, rate_hz, seconds, seed=seed)
        st0 = srv.stats()
        with ClockSampler(0) as clocks:
            rec, dropped = srv.replay(trace, lam, W.SIGMA_U)
        st1 = srv.stats()
        t0 = int(rec["t_submit_ns"].min()) - int(trace[0][0] * 1e9)
        span = (int(rec["t_result_ns"].max()) - t0) / 1e9
        steps = float(np.sum(rec["K"].astype(np.float64) * rec["T"]))
        lat = (rec["t_result_ns"] - rec["t_submit_ns"]) / 1e6
        queue = (rec["t_launch_ns"] - rec["t_submit_ns"]) / 1e6
        useful = steps * 12 * L * FLOPS_PER_FIELD
        clk = clocks.summary()
        if precision != "fp32":
            issued = steps * 12 * L_pad * TC_MMA_FLOPS_PER_FIELD[precision]
            peak, basis = tensor_peak(measured_peaks(), clk)
            roof = {"bound": "tensor", "achieved": issued / span / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": issued / span / 1e12 / peak, "useful_tflops": useful / span / 1e12,
                    "useful_frac": useful / span / 1e12 / peak, "peak_basis": basis,
                    "at_run_clock": clock_scaled(measured_peaks(), clk, issued / span / 1e12),
                    "kernel": "rollout_tc_group_kernel (issued MMA flops over the whole serving span)"}
        else:
            peak = torch.cuda.get_device_properties(0).multi_processor_count * FP32_LANES_PER_SM * 2 * \
                float(measured_peaks().get("sm_max_mhz", 2032.0)) * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": useful / span / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": useful / span / 1e12 / peak,
                    "kernel": "rollout_fp32_group_kernel (useful flops over the whole serving span)"}
        return {"offered_hz_per_quad": rate_hz, "trace_s": seconds, "arrivals": len(trace), "served": int(len(rec)),
                "dropped": dropped, "span_s": span, "rollout_steps_per_s": steps / span,
                "requests_per_s": len(rec) / span,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "mean": float(lat.mean()), "max": float(lat.max())},
                "queue_ms": {"p50": float(np.percentile(queue, 50)), "p99": float(np.percentile(queue, 99))},
                "group_size": {"mean": float(rec["group_size"].mean()), "max": int(rec["group_size"].max())},
                "gpu_launches": int(st1["launches"] - st0["launches"]), "groups": int(st1["groups"] - st0["groups"]),
                "pool_peak_bytes": int(st1["pool_peak_bytes"]), "roofline": roof, "clocks": clk,
                "all_ok": bool(np.all(rec["status"] == 0))}

    full = run(50.0, serve_seconds, seed=1)
    cap = full["requests_per_s"]
    half_rate = 0.5 * cap / n_quad
    half = run(half_rate, max(serve_seconds, 160.0 / (0.5 * cap)), seed=2)
    sweep = []
    for i, frac in enumerate(sweep_loads):
        if frac == 0.5:
            pt = half
        else:
            pt = run(frac * cap / n_quad, max(serve_seconds, 120.0 / (frac * cap)), seed=3 + i)
        sweep.append({"load": frac, "offered_hz_per_quad": pt["offered_hz_per_quad"],
                      "requests_per_s": pt["requests_per_s"], "latency_ms": pt["latency_ms"],
                      "queue_ms": pt["queue_ms"], "group_size_mean": pt["group_size"]["mean"],
                      "rollout_steps_per_s": pt["rollout_steps_per_s"]})
    srv.close()
    ctl.close()
    return full, half, sweep, cap


def run_serving(args):
    """The serving workload (see serving_measure) as its own JSON line."""
    from paper_1503_00330_b300 import build
    build.build()
    full, half, sweep, cap = serving_measure(args.precision, args.serve_seconds, args.serve_sweep,
                                             args.serve_lanes, args.serve_group, args.warmup)
    line = {"metric": METRIC, "value": full["rollout_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": full["served"], "warmup": args.warmup, "ms_per_step": 1e3 / full["requests_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator; quadrotor-shaped LWPR model, Poisson request trace)",
            "config": {"workload": SERVING_WORKLOAD,
                       "precision": args.precision, "lanes": args.serve_lanes, "max_group": args.serve_group,
                       "step": "one served request (ms_per_step = 1 / served request rate)",
                       "l2": "inputs of a saturated group exceed L2 (each request's scratch ~K*T*20 bytes)"},
            "e2e": {"value": full["rollout_steps_per_s"], "unit": UNIT,
                    "note": "requests enter on the host and plans return to pinned host memory inside the span"},
            "gpu_launches": full["gpu_launches"], "roofline": full["roofline"],
            "latency_ms": full["latency_ms"], "at_offered_rate": full, "at_half_capacity": half,
            "load_sweep": {"capacity_requests_per_s": cap, "points": sweep},
            "clocks": full["clocks"]}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_1503_00330_b300 import build
    from paper_1503_00330_b300.api import Controller

    rank, ws, local, dist = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    p, desc = workload(args.workload, rank)          # replicas: rank-dependent seed
    K, T, M, L = p.K, p.T, p.M, p.model.L

    ctl = Controller(p.model, p.cost, M=M, model_noise=p.model_noise, device=local, precision=args.precision)
    launch = None
    if args.precision == "fp32":
        ctl.set_output_split(SPLIT_MODE[0])
        launch = fp32_launch(ctl, K)
    ctl.set_timing(True)
    ctl.reserve(K, T)
    x0 = torch.as_tensor(p.x0, device=dev).clone()
    ua = torch.as_tensor(p.u_nom, device=dev).clone()
    ub = torch.empty_like(ua)
    costs = torch.empty(K, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def rh_step(it, plant_ev=None):
        ctl.update(x0, ua, K, T, p.lam, p.sigma_u, p.seed + it, u_out=ub, costs_out=costs)
        if plant_ev is not None:
            plant_ev[0].record(stream)
        ctl.rh_advance(x0, ub, ua)                   # next warm start back into ua
        if plant_ev is not None:
            plant_ev[1].record(stream)

    for it in range(args.warmup):
        rh_step(it)
    ctl.sync()

    # ---- device-timed region -------------------------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    rollout_ms, step_ms, scan_ms, merge_ms = [], [], [], []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctl.launch_count()
    with ClockSampler(local) as clocks:
        # the steps of a chunk are enqueued back to back (no host sync between them, so
        # no host latency inside an event window); the context's ring of stage events
        # then gives each update's kernel times
        for c0 in range(0, args.steps, TIMING_CHUNK):
            c1 = min(args.steps, c0 + TIMING_CHUNK)
            for i in range(c0, c1):
                flush.zero_()                           # L2 flush, outside the event window
                ev[i][0].record(stream)
                rh_step(args.warmup + i, pev[i])
                ev[i][1].record(stream)
            for i in range(c0, c1):
                st = ctl.stage_times(back=c1 - 1 - i)
                rollout_ms.append(st[0])
                scan_ms.append(st[1])
                merge_ms.append(st[2])
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = ctl.launch_count() - launches0
    ctl.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    plant_ms = [a.elapsed_time(b) for a, b in pev]
    total_s = reduce_max(dist, sum(step_ms) / 1e3, dev)
    value = job_throughput(dist, K * T * M * args.steps, sum(step_ms) / 1e3, dev)

    # ---- end to end through the host-buffer entry point ----------------------
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory().numpy()
    hx0, hu = pin(p.x0), pin(p.u_nom)
    hout, hcost = pin(np.empty((T, 4), np.float32)), pin(np.empty(K, np.float32))
    e2e_times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ctl.update_host(hx0, hu, K, T, p.lam, p.sigma_u, p.seed + i, u_out=hout, costs_out=hcost)
        el = time.perf_counter() - t0
        hu[:-1] = hout[1:]
        hu[-1] = hout[-1]
        if i >= args.warmup:
            e2e_times.append(el)
    e2e_value = job_throughput(dist, K * T * M * args.steps, sum(e2e_times), dev)

    if rank != 0:
        dist.destroy_process_group()
        return

    peaks = measured_peaks()
    clk = clocks.summary()
    roofline = form_roofline(args.precision, rollout_ms, K, T, M, L, dev, peaks, args.workload, clocks=clk,
                             launch=launch)
    rates = pipe_peaks(local)   # measured pipe rates: context beside the unit-count FP32 peak
    roofline["rollout_share_of_step"] = sum(rollout_ms) / sum(step_ms)
    roofline["secondary"] = mufu_check(args.precision, rollout_ms, K, T, M, L, local)
    reduction = reduction_rooflines(scan_ms, merge_ms, K, T, peaks, local)
    reduction["plant_step"] = plant_step_roofline(plant_ms, L, peaks, args.precision)
    forms = {args.precision: {"value": value, "ms_per_update": 1e3 * total_s / args.steps,
                              "roofline": roofline, "reduction": reduction, "clocks": clk}}
    if not args.no_compare:
        for other in FORMS:
            if other != args.precision:
                forms[other] = time_form(other, p, args, dev)
    # the precision workload (K=65536, T=100, L=2048, conditioned D) in both forms, beside the headline
    prec = None
    if ws == 1 and args.workload == "realtime" and not args.no_precision:
        from paper_1503_00330_b300 import workloads as W
        pp = W.precision(0)
        prec = {"config": {"workload": "precision: K=65536 rollouts, T=100 steps, L=2048 fields x 12 outputs, "
                                       "cond(D_j) log-uniform in [1, 1e3], 16 obstacles; plain pi_update calls",
                           "K": pp.K, "T": pp.T, "L": pp.model.L, "M": pp.M,
                           "l2": "flushed between timed updates (256 MiB write outside the event window)"},
                "forms": {f: time_updates(f, pp, args.precision_steps, 3, dev, "precision") for f in FORMS}}
    # the batched workload (64 uneven controllers, one launch under a CUDA graph) in every form,
    # with the schedule the autotuner picks on it (longest first, one item per CTA)
    bat = None
    if ws == 1 and args.workload == "realtime" and not args.no_batched:
        from paper_1503_00330_b300 import workloads as W
        bprobs = W.batched(64, seed=0)
        by_L = max(range(len(bprobs)), key=lambda i: bprobs[i].model.L)
        by_K = max((i for i in range(len(bprobs)) if i != by_L), key=lambda i: bprobs[i].K)
        bpick = (by_L, by_K)
        bforms, bcosts = batched_forms(bprobs, BATCHED_SCHEDULE, FORMS, args.batched_steps, 3, dev, pick=bpick)
        bat = {"config": {"workload": "batched: 64 controllers, K ~ logU[1024, 32768], T ~ U{30..150}, "
                                      "L ~ logU[128, 2048], own model, obstacles and seed each; one launch under a "
                                      "CUDA graph", "controllers": len(bprobs),
                          "rollout_steps_per_update": sum(p.K * p.T * p.M for p in bprobs),
                          "schedule": "longest first, one item per CTA (the autotuner's pick on this workload)",
                          "l2": "flushed between timed updates (256 MiB write outside the event window)"},
               "forms": bforms}
    # the serving workload (256 quadrotors, continuous batching), tensor-core form
    srv_line = None
    if ws == 1 and args.workload == "realtime" and not args.no_serving:
        sfull, shalf, _, scap = serving_measure("tc", args.serve_seconds, [], args.serve_lanes, args.serve_group, 3)
        srv_line = {"config": {"workload": SERVING_WORKLOAD, "precision": "tc", "lanes": args.serve_lanes,
                               "max_group": args.serve_group},
                    "rollout_steps_per_s": sfull["rollout_steps_per_s"], "requests_per_s": sfull["requests_per_s"],
                    "latency_ms_at_offered_rate": sfull["latency_ms"],
                    "latency_ms_at_half_capacity": shalf["latency_ms"], "capacity_requests_per_s": scap,
                    "roofline": sfull["roofline"], "clocks": sfull["clocks"], "gpu_launches": sfull["gpu_launches"],
                    "all_ok": sfull["all_ok"] and shalf["all_ok"],
                    "error": "each served result equals the agent's updates run alone on the single-controller "
                             "path bitwise (tests/test_gpu_serve.py), so it carries that path's error"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator; quadrotor-shaped LWPR model and obstacle field)",
            "config": {"workload": desc, "K": K, "T": T, "L": L, "M": M, "precision": args.precision,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed between timed steps (256 MiB write outside the event window); "
                             "per-update working set ~21 MB"},
            "ms_per_update": 1e3 * total_s / args.steps,
            "ms_per_update_stats": {"best": min(step_ms), "median": statistics.median(step_ms),
                                    "n": len(step_ms), "note": "this rank's timed updates (CUDA events)"},
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": (12 + T * 4) * 4,
                    "d2h_bytes_per_step": (T * 4 + K) * 4},
            "roofline": roofline,
            "reduction_kernels": reduction,
            "measured_pipe_rates": {**rates, "dfma_per_s": fp64_peak(local),
                                    "note": "FFMA2 / MUFU ex2 / DFMA chains on every SM, event-timed; "
                                            "the FP32 roofline keeps the unit-count peak"},
            "forms": forms,
            "paper_context": PAPER_CONTEXT,
            "clocks": clk}
    if ws == 1 and not args.no_cpu_baseline:
        base, ref = cpu_baseline(p, args.cpu_sample)
        line["cpu_baseline"] = base
        for f in forms:
            forms[f]["error"] = {**form_errors(p, f, ref, dev), "tolerance_u_out": ERROR_BOUND[f],
                                 "tolerance_costs": ERROR_BOUND[f]}
        if prec is not None:
            pbase, pref = cpu_baseline(pp, args.precision_sample, k_single=8)
            prec["cpu_baseline"] = pbase
            for f in prec["forms"]:
                prec["forms"][f]["error"] = {**form_errors(pp, f, pref, dev), "tolerance_u_out": ERROR_BOUND[f],
                                             "tolerance_costs": ERROR_BOUND[f]}
        if bat is not None:
            bbase, bref = batched_cpu_baseline(bprobs, bpick, args.batched_sample)
            bat["cpu_baseline"] = bbase
            for f in bat["forms"]:
                bat["forms"][f]["error"] = {**batched_errors(bprobs, bcosts[f], bref),
                                            "tolerance_costs": ERROR_BOUND[f]}
    if prec is not None:
        line["precision_workload"] = prec
    if bat is not None:
        line["batched_workload"] = bat
    if srv_line is not None:
        line["serving_workload"] = srv_line
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["realtime", "realtime_short", "small", "precision", "precision_short", "batched",
                                                   "serving", "subrollouts"], default="realtime")
    ap.add_argument("--cpu-sample", type=int, default=2048,
                    help="rollouts in the CPU-baseline sample (also the error reference of each form)")
    ap.add_argument("--precision-sample", type=int, default=512,
                    help="rollouts in the precision workload's CPU-baseline / error-reference sample")
    ap.add_argument("--precision-steps", type=int, default=3,
                    help="timed updates of the precision workload (default line only)")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision workload in the default line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload in the default line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving workload in the default line")
    ap.add_argument("--batched-steps", type=int, default=3,
                    help="timed batched updates per form (default line only)")
    ap.add_argument("--batched-sample", type=int, default=32,
                    help="rollouts per sampled controller in the batched error reference")
    ap.add_argument("--ref-sample", type=int, default=64, help="rollouts per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=list(FORMS), default=None,
                    help="form of the headline line (the other forms are timed too and reported under 'forms'); "
                         "default fp32, except the serving workload, whose default is the tensor-core form")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other form")
    ap.add_argument("--split", choices=["auto", "off", "always"], default="auto",
                    help="launch of the FP32 rollout kernel (pi_set_output_split; same results bit for bit)")
    ap.add_argument("--batch-tile", type=int, default=-1,
                    help="batched: tile shape (0 persistent work list, 1 one item per CTA, 2..4 tensor-core "
                         "outputs split over CTAs; -1 = pick order and tile per form with the autotuner)")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="serving: trace length at the offered rate")
    ap.add_argument("--serve-lanes", type=int, default=2, help="serving: groups on the GPU at once")
    ap.add_argument("--serve-group", type=int, default=64, help="serving: most requests per group")
    ap.add_argument("--serve-sweep", type=float, nargs="*", default=[0.25, 0.5, 0.75, 0.9],
                    help="serving: offered loads (fractions of the measured capacity) for the latency sweep")
    args = ap.parse_args()
    SPLIT_MODE[0] = args.split
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.precision is None:
        args.precision = "tc" if args.workload == "serving" else "fp32"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

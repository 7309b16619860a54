"""Schedule autotuner for the batched (multi-controller) update.

For a set of controllers it times every candidate schedule of the batched
launch -- precision form (FP32 or tensor-core) x work-list order (controller
order, longest block first, round robin) x, for the tensor-core form, the
tile shape (persistent CTAs over the slot-block items, or one item per CTA,
or, with tensor cores, per pair of CTAs that split its outputs) -- on the device, keeps the
fastest, and stores it in a JSON cache keyed by the batch's shape signature
(per controller: K, T, L, M) and the device name, so later runs with the same
shapes skip the search.  Both forms meet the same accuracy target, so the
choice is by time alone.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import torch

from .api import Batch, Controller

DEFAULT_CACHE = os.environ.get("PI2RH_AUTOTUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "pi2rh", "autotune.json"))
ORDERS = ("as_given", "longest_first", "round_robin")
TC_TILES = (0, 1, 2)     # persistent work list; one item per CTA; outputs split over 2 CTAs
FP32_TILES = (0, 1)      # persistent work list; one item per CTA
VERSION = 3


def signature(problems, device: int = 0) -> str:
    shapes = sorted((p.K, p.T, p.model.L, p.M) for p in problems)
    name = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    blob = json.dumps({"v": VERSION, "device": name, "shapes": shapes})
    return hashlib.sha1(blob.encode()).hexdigest()


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, cache):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def time_batch(batch: Batch, problems, reps: int = 2, warmup: int = 1) -> float:
    """Mean device milliseconds of one batched update."""
    lam = [p.lam for p in problems]
    su = [p.sigma_u for p in problems]
    stream = torch.cuda.current_stream(batch.device)
    for i in range(warmup):
        batch.update(lam, su, [p.seed + i for p in problems])
    batch.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(reps):
        batch.update(lam, su, [p.seed + 100 + i for p in problems])
    b.record(stream)
    b.synchronize()
    batch.sync()
    return a.elapsed_time(b) / reps


def tune(problems, forms=("fp32", "tc"), orders=ORDERS, reps: int = 2, cache_path: str = DEFAULT_CACHE,
         use_cache: bool = True, device: int = 0, log=None, tc_tiles=TC_TILES) -> dict:
    """Returns {"form", "order", "tile", "ms", "candidates": {...}, "cached": bool}."""
    key = signature(problems, device)
    cache = _load(cache_path) if use_cache else {}
    if use_cache and key in cache:
        out = dict(cache[key])
        out["cached"] = True
        return out
    results = {}
    for form in forms:
        ctls = [Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, device=device, precision=form)
                for p in problems]
        batch = Batch(ctls, [p.K for p in problems], [p.T for p in problems], precision=form,
                      x0=[p.x0 for p in problems], u_nom=[p.u_nom for p in problems])
        for order in orders:
            batch.set_schedule(order)
            for tile in (FP32_TILES if form == "fp32" else tc_tiles):
                batch.set_tile(tile)
                t0 = time.perf_counter()
                ms = time_batch(batch, problems, reps=reps)
                results[f"{form}/{order}/{tile}"] = ms
                if log:
                    log(f"autotune {form}/{order}/tile {tile}: {ms:.2f} ms per update "
                        f"({time.perf_counter() - t0:.1f} s)")
        batch.close()
        for c in ctls:
            c.close()
    best = min(results, key=results.get)
    form, order, tile = best.split("/")
    out = {"form": form, "order": order, "tile": int(tile), "ms": results[best], "candidates": results}
    if use_cache:
        cache[key] = out
        _store(cache_path, cache)
    out = dict(out)
    out["cached"] = False
    return out

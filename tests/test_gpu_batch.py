"""Batched update (one persistent launch under a CUDA graph): every
controller's result must equal its own pi_update exactly (same kernels, same
per-slot arithmetic, same reduction order), across repeated updates, schedule
changes and both precision forms; plus the oracle for small controllers."""
import numpy as np
import pytest
import torch

from paper_1503_00330_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    build.build()


def _problems():
    spec = [(300, 20, 40, 1), (65, 7, 130, 2), (1000, 13, 9, 1), (128, 31, 257, 1), (1, 5, 3, 4)]
    out = []
    for i, (K, T, L, M) in enumerate(spec):
        p = W.problem(K, T, L, seed=50 + i, n_obs=3 + i, M=M)
        p.u_nom = np.random.default_rng(i).normal(0, 0.2, (T, 4)).astype(np.float32)
        p.x0 = np.random.default_rng(i + 9).normal(0, 0.1, 12).astype(np.float32)
        out.append(p)
    return out


@pytest.mark.parametrize("form", ["fp32", "tc", "tc_fp16x2"])
def test_batch_equals_single_updates(form):
    from paper_1503_00330_b300.api import Batch, Controller
    probs = _problems()
    ctls = [Controller(p.model, p.cost, M=p.M, precision=form) for p in probs]
    batch = Batch(ctls, [p.K for p in probs], [p.T for p in probs], precision=form,
                  x0=[p.x0 for p in probs], u_nom=[p.u_nom for p in probs])
    lam = [p.lam for p in probs]
    su = [p.sigma_u for p in probs]
    for rep, order in enumerate(["longest_first", "as_given", "round_robin"]):
        batch.set_schedule(order)
        seeds = [p.seed + 7 * rep for p in probs]
        u_b, c_b = batch.update(lam, su, seeds)
        batch.sync()
        for i, (p, c) in enumerate(zip(probs, ctls)):
            u, cs = c.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, seeds[i])
            c.sync()
            assert torch.equal(u_b[i], u), f"controller {i} u_out differs ({order})"
            assert torch.equal(c_b[i], cs), f"controller {i} costs differ ({order})"
    assert batch.launch_count() == 9


@pytest.mark.parametrize("form", ["fp32", "tc"])
def test_batch_against_oracle(oracle, form):
    from paper_1503_00330_b300.api import Batch, Controller
    probs = _problems()[:3]
    ctls = [Controller(p.model, p.cost, M=p.M, precision=form) for p in probs]
    batch = Batch(ctls, [p.K for p in probs], [p.T for p in probs], precision=form,
                  x0=[p.x0 for p in probs], u_nom=[p.u_nom for p in probs])
    u_b, c_b = batch.update([p.lam for p in probs], [p.sigma_u for p in probs], [p.seed for p in probs])
    batch.sync()
    for i, p in enumerate(probs):
        uref, cref = oracle.pi_update(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed, M=p.M)
        scale = np.maximum(np.abs(uref).max(0), np.sqrt(p.sigma_u.astype(np.float64) / p.K))
        eu = np.abs(u_b[i].cpu().numpy() - uref).max(0) / scale
        ec = np.max(np.abs(c_b[i].cpu().numpy() - cref) / cref)
        print(f"{form} controller {i}: u err {eu}, cost err {ec:.3g}")
        assert np.all(eu <= 1e-5) and ec <= 1e-5


def test_autotuner_picks_and_caches(tmp_path):
    from paper_1503_00330_b300 import autotune
    probs = _problems()[:3]
    cache = str(tmp_path / "tune.json")
    r1 = autotune.tune(probs, reps=1, cache_path=cache)
    assert r1["form"] in ("fp32", "tc") and r1["order"] in autotune.ORDERS and not r1["cached"]
    assert r1["tile"] in (autotune.TC_TILES if r1["form"] == "tc" else autotune.FP32_TILES)
    assert len(r1["candidates"]) == len(autotune.ORDERS) * (len(autotune.FP32_TILES) + len(autotune.TC_TILES))
    r2 = autotune.tune(probs, reps=1, cache_path=cache)
    assert r2["cached"] and (r2["form"], r2["order"], r2["tile"]) == (r1["form"], r1["order"], r1["tile"])


@pytest.mark.parametrize("split", [1, 2, 3, 4])
def test_batch_tile_shapes_equal_single_updates(split):
    """Every tensor-core tile shape of the batch gives each controller's own
    pi_update result bitwise (items per CTA, or outputs split over a cluster)."""
    from paper_1503_00330_b300.api import Batch, Controller, PiError
    probs = _problems()
    ctls = [Controller(p.model, p.cost, M=p.M, precision="tc") for p in probs]
    batch = Batch(ctls, [p.K for p in probs], [p.T for p in probs], precision="tc",
                  x0=[p.x0 for p in probs], u_nom=[p.u_nom for p in probs])
    batch.set_tile(split)
    seeds = [p.seed + 3 for p in probs]
    u_b, c_b = batch.update([p.lam for p in probs], [p.sigma_u for p in probs], seeds)
    batch.sync()
    for i, (p, c) in enumerate(zip(probs, ctls)):
        u, cs = c.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, seeds[i])
        c.sync()
        assert torch.equal(u_b[i], u) and torch.equal(c_b[i], cs), f"controller {i}, split {split}"
    with pytest.raises(PiError):
        batch.set_tile(5)
    fctl = [Controller(probs[0].model, probs[0].cost)]
    fb = Batch(fctl, [probs[0].K], [probs[0].T], precision="fp32")
    with pytest.raises(PiError):
        fb.set_tile(2)                    # FP32 items are not split over CTAs
    fb.close()


def test_fp32_batch_plain_launch_equals_single_updates():
    from paper_1503_00330_b300.api import Batch, Controller
    probs = _problems()
    ctls = [Controller(p.model, p.cost, M=p.M) for p in probs]
    batch = Batch(ctls, [p.K for p in probs], [p.T for p in probs], precision="fp32",
                  x0=[p.x0 for p in probs], u_nom=[p.u_nom for p in probs])
    batch.set_tile(1)
    seeds = [p.seed + 5 for p in probs]
    u_b, c_b = batch.update([p.lam for p in probs], [p.sigma_u for p in probs], seeds)
    batch.sync()
    for i, (p, c) in enumerate(zip(probs, ctls)):
        u, cs = c.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, seeds[i])
        c.sync()
        assert torch.equal(u_b[i], u) and torch.equal(c_b[i], cs), f"controller {i}"

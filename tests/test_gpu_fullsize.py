"""Parity at the benchmark's own sizes, and the cases where FP32 conditioning
of Eq. 1 limits the accuracy, through the C ABI against the FP64 oracle.

* Realtime update (K=8192, T=100, L=512, 16 obstacles, seed 0), launched as
  the benchmark launches it, in every form: u_out element-wise per channel and
  all 8192 costs S_{k,0} (Sec. 3.1, Eq. 2).  The oracle runs every rollout once
  for all forms.
* Precision shape (L=2048, T=100, cond(D_j) log-uniform in [1, 1e3]) at
  K=2048 in full, in every form.
* 64-controller batch at full size: S_{k,0} of the 32 first and 32 last
  rollouts of four controllers (the two largest L and the two largest K).

Obstacle indicator flips.  The oracle decides the crash indicator of Sec. 5 on
its FP64 state, the kernels on their FP32 state, so a rollout that grazes a
cylinder boundary can be inside at a step on one side only (a "flip": its
running cost jumps by w_obs).  Flips are counted from the per-step costs and
reported; a rollout with flips must differ from the oracle by exactly its
flips' cost (n * w_obs * dt, within the ordinary tolerance), and every other
rollout is held to the ordinary tolerance.

Tolerances: u_out max_t |du| / max_t |u_ref| per channel and |dS| / S, per
form: 1e-5 for FP32 and for the three-product tensor-core form (its split
products carry ~22 significand bits, so it is held to the FP32 bound, tighter
than the 2e-3 stated for the tensor-core form); 2e-3 for the two-product form
(tc_fp16x2), whose 128 quadratic terms per exponent each carry an fp16
rounding.  The damped cases have their own bounds (see there).
"""
import numpy as np
import pytest
import torch

from paper_1503_00330_b300 import workloads as W

pytestmark = pytest.mark.gpu

FORMS = ["fp32", "tc", "tc_fp16x2"]
U_TOL = {"fp32": 1e-5, "tc": 1e-5, "tc_fp16x2": 2e-3}
S_TOL = {"fp32": 1e-5, "tc": 1e-5, "tc_fp16x2": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    build.build()


def _ctrl(p, form):
    from paper_1503_00330_b300.api import Controller
    return Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, precision=form)


def _oracle_full(oracle, p):
    """Every rollout's per-step costs, perturbations and terminal cost, then the
    cost-to-go and Eq. 2 (the oracle's pi_update is exactly this composition)."""
    r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed, M=p.M,
                        model_noise=p.model_noise)
    S = oracle.cost_to_go(r["cost"], r["phi"], float(p.model.dt))
    u = oracle.weighted_update(S, r["eps"], p.u_nom, p.lam)
    return {"cost": r["cost"], "phi": r["phi"], "eps": r["eps"], "S0": S[:, 0].copy(), "u": u}


def _u_err(u, ref):
    u, ref = np.asarray(u, np.float64), np.asarray(ref, np.float64)
    return np.abs(u - ref).max(0) / np.abs(ref).max(0)


def _run_form(p, form, with_steps=True):
    """u_out, costs_out of one update as the benchmark launches it (scratch
    reserved first), and the per-step costs [K, T] of the same launch."""
    ctl = _ctrl(p, form)
    ctl.reserve(p.K, p.T)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    steps = None
    if with_steps:
        cost, _, _ = ctl.debug_rollout(p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed)
        steps = cost.cpu().numpy().T.astype(np.float64)
    ctl.sync()
    out = (u.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64), steps)
    ctl.close()
    return out


def _check_against_oracle(p, form, ref, u, c, steps, label):
    w_jump = float(p.cost.w_obs) * float(p.model.dt) / p.M
    # flips: steps whose cost differs from the oracle's by about w_obs
    dq = steps - ref["cost"]
    flip_steps = np.abs(dq) > 0.5 * float(p.cost.w_obs)
    n_flip = flip_steps.sum(1)
    signed = np.rint(dq / float(p.cost.w_obs)) * flip_steps
    flipped = n_flip > 0
    dS = c - ref["S0"]
    err = np.abs(dS) / ref["S0"]
    # a flipped rollout differs by exactly its flips' cost
    resid = np.abs(dS - signed.sum(1) * w_jump) / ref["S0"]
    eu = _u_err(u, ref["u"])
    print(f"{label} ({form}): u_out rel err per channel {np.array2string(eu, precision=3)}; "
          f"costs max rel err {err[~flipped].max():.3g} over {int((~flipped).sum())} rollouts; "
          f"indicator flips {int(n_flip.sum())} in {int(flipped.sum())} rollouts "
          f"(residual after the flips' cost {resid[flipped].max() if flipped.any() else 0.0:.3g})")
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(c))
    assert np.all(err[~flipped] <= S_TOL[form])
    assert np.all(resid[flipped] <= S_TOL[form])
    assert flipped.sum() <= max(2, p.K // 1000)
    assert np.all(eu <= U_TOL[form])


# ---------------------------------------------------------------------------
# realtime workload, full update
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def realtime_ref(oracle):
    p = W.realtime()
    return p, _oracle_full(oracle, p)


@pytest.mark.parametrize("form", FORMS)
def test_realtime_full_update(realtime_ref, form):
    """K=8192, T=100, L=512: every cost and u_out against the oracle."""
    p, ref = realtime_ref
    u, c, steps = _run_form(p, form)
    _check_against_oracle(p, form, ref, u, c, steps, "realtime K=8192 T=100 L=512")


# ---------------------------------------------------------------------------
# precision shape at K = 2048, full update
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def precision_ref(oracle):
    p = W.precision(K=2048)
    return p, _oracle_full(oracle, p)


@pytest.mark.parametrize("form", FORMS)
def test_precision_shape_full_update(precision_ref, form):
    """L=2048, T=100, cond(D_j) log-uniform in [1, 1e3], K=2048 in full."""
    p, ref = precision_ref
    u, c, steps = _run_form(p, form)
    _check_against_oracle(p, form, ref, u, c, steps, "precision shape K=2048 T=100 L=2048")


# ---------------------------------------------------------------------------
# damped model: FP32 conditioning of Eq. 1
# ---------------------------------------------------------------------------
def _damped_model(L, seed):
    """The synthetic model with each output's slope on its own state set to -3
    and the other slopes scaled by 0.3 (bounded over long horizons)."""
    m = W.make_lwpr(L, seed)
    beta = m.beta.astype(np.float64) * 0.3
    for o in range(beta.shape[0]):
        beta[o, :, o] = -3.0
    m.beta = np.ascontiguousarray(beta.astype(np.float32))
    return m


# cost-to-go error bounds of the damped cases (relative, per rollout)
DAMPED_S_BOUND = {"fp32": 5e-5, "tc": 2e-4, "tc_fp16x2": 2e-3}
# rollouts with indicator flips allowed in the damped cases: the two-product form's
# exponents carry ~1e-4 relative error per step, which over 600-2000 steps moves a
# grazing trajectory across a cylinder boundary at a different step (5 of 300
# rollouts over 2000 steps); their weight in Eq. 2 is bounded by the u_out check
DAMPED_FLIPS = {"fp32": lambda K: 2, "tc": lambda K: 2, "tc_fp16x2": lambda K: max(2, K // 50)}
TC_U_BOUND = 2e-3


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("K,T,L", [(40, 600, 7), (129, 257, 130), (300, 2000, 3)])
def test_damped_model_conditioning(oracle, form, K, T, L):
    """With the damped model the local predictions spread about ten times wider
    than the generator's, and receptive-field exponents q reach 50-100.  The
    FP32 rounding of an exponent, about q * 2^-24 absolute, is a relative error
    of the same size in its softmax weight (Eq. 1); the variance term of the
    cost inherits it at the wider spread, so the cost-to-go carries relative
    errors well above 1e-5 (bounded here by DAMPED_S_BOUND; the three-product
    tensor-core exponents carry ~22 significand bits, so four times the FP32
    bound; the two-product form is held to its stated 2e-3).

    u_out is then held to the first-order propagation of those errors through
    Eq. 2: P_k = softmax(-S_k / lambda) moves by P_k (|dS_k| + max |dS|) / lambda,
    so |du_c| <= 2 max_{k,i} |dS_{k,i}| max_k |eps_{k,c}| / lambda, where
    |dS_{k,i}| <= |dphi_k| + dt sum_j |dq_{k,j}| from the per-step errors.  The
    tensor-core forms are also held to their stated bound, 2e-3 per channel."""
    model = _damped_model(L, 2000 + K)
    p = W.problem(K, T, L, seed=2000 + K, n_obs=5, model=model)
    ref = _oracle_full(oracle, p)
    ctl = _ctrl(p, form)
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    cost, eps, phi = ctl.debug_rollout(p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed)
    ctl.sync()
    u, c = u.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)
    steps = cost.cpu().numpy().T.astype(np.float64)
    phi = phi.cpu().numpy().astype(np.float64)
    flipped = np.any(np.abs(steps - ref["cost"]) > 0.5 * float(p.cost.w_obs), axis=1)
    flips = int(flipped.sum())
    eS = (np.abs(c - ref["S0"]) / ref["S0"])[~flipped]
    dS_max = np.max(np.abs(phi - ref["phi"]) + float(p.model.dt) * np.abs(steps - ref["cost"]).sum(1))
    scale = np.abs(ref["u"]).max(0)
    bound = 2 * dS_max * np.abs(ref["eps"]).max((0, 1)) / p.lam / scale
    eu = _u_err(u, ref["u"])
    print(f"damped K={K} T={T} L={L} ({form}): u_out rel err {np.array2string(eu, precision=3)}, "
          f"first-order bound {np.array2string(bound, precision=3)}; S0 max rel err {eS.max():.3g}; "
          f"max |dS| {dS_max:.3g}; rollouts with indicator flips {flips}")
    assert flips <= DAMPED_FLIPS[form](K)
    assert eS.max() <= DAMPED_S_BOUND[form]
    assert np.all(eu <= bound + U_TOL[form])
    if form != "fp32":
        assert np.all(eu <= TC_U_BOUND)


# ---------------------------------------------------------------------------
# batched workload at full size, sampled
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def batched_ref(oracle):
    probs = W.batched(64, seed=0)
    by_L = sorted(range(len(probs)), key=lambda i: -probs[i].model.L)
    by_K = sorted(range(len(probs)), key=lambda i: -probs[i].K)
    pick = by_L[:2] + [i for i in by_K if i not in by_L[:2]][:2]
    refs = {}
    for i in pick:
        p = probs[i]
        ks, S0 = [], []
        for k0 in (0, p.K - 32):
            r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, 32, p.T, p.sigma_u, p.seed, k0=k0)
            S0.append(oracle.cost_to_go(r["cost"], r["phi"], float(p.model.dt))[:, 0])
            ks.append(np.arange(k0, k0 + 32))
        refs[i] = (np.concatenate(ks), np.concatenate(S0))
    return probs, refs


@pytest.mark.parametrize("form", FORMS)
def test_batched_workload_sampled(batched_ref, form):
    """64 controllers (K ~ logU[1024, 32768], T ~ U{30..150}, L ~ logU[128, 2048])
    in one batched launch: S_{k,0} of 64 edge rollouts of four controllers."""
    from paper_1503_00330_b300.api import Batch, Controller
    probs, refs = batched_ref
    ctls = [Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, precision=form) for p in probs]
    batch = Batch(ctls, [p.K for p in probs], [p.T for p in probs], precision=form,
                  x0=[p.x0 for p in probs], u_nom=[p.u_nom for p in probs])
    u_b, c_b = batch.update([p.lam for p in probs], [p.sigma_u for p in probs], [p.seed for p in probs])
    batch.sync()
    for i, (ks, S0) in refs.items():
        p = probs[i]
        c = c_b[i].cpu().numpy().astype(np.float64)
        err = np.abs(c[ks] - S0) / S0
        print(f"batched ({form}) controller {i} K={p.K} T={p.T} L={p.model.L}: S0 max rel err {err.max():.3g}")
        assert np.all(err <= S_TOL[form])
        assert np.all(np.isfinite(u_b[i].cpu().numpy()))
    batch.close()
    for c in ctls:
        c.close()


# ---------------------------------------------------------------------------
# FP32 with a split partial wave, sampled
# ---------------------------------------------------------------------------
def test_fp32_partial_wave_split_sampled(oracle):
    """The realtime model with one whole wave of 64-slot blocks plus ten more
    (K = 64 SMs + 640): the plain launch takes the whole wave, the output-split
    launch the last ten blocks.  S_{k,0} of 32 rollouts at each end (one side
    in each launch) against the oracle."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    p = W.realtime(0)
    p.K, p.T = 64 * nsm + 640, 40
    p.u_nom = p.u_nom[:p.T].copy()
    ctl = _ctrl(p, "fp32")
    plain, upc, ctas = ctl.split_plan(p.K)
    assert plain == nsm and upc == 1 and ctas == 120
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    c = c.cpu().numpy().astype(np.float64)
    for k0 in (0, p.K - 32):
        r = oracle.rollouts(p.model, p.cost, p.x0, p.u_nom, 32, p.T, p.sigma_u, p.seed, k0=k0)
        S0 = oracle.cost_to_go(r["cost"], r["phi"], float(p.model.dt))[:, 0]
        err = np.abs(c[k0:k0 + 32] - S0) / S0
        print(f"fp32 partial-wave split, rollouts {k0}..{k0 + 31}: S0 max rel err {err.max():.3g}")
        assert np.all(err <= S_TOL["fp32"])
    assert np.all(np.isfinite(u.cpu().numpy()))
    ctl.close()

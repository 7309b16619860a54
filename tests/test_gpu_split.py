"""Output-split launch of the FP32 rollout (pi_set_output_split).

With fewer 64-slot blocks than SMs, the split launch deals the (block, output)
units out to one co-resident CTA per SM, which exchange each step's state
through device memory; with more blocks than SMs, whole waves keep the plain
launch and only the last, partial wave is split.  Every output is still
evaluated by one CTA with the same records, order and merge (Sec. 2, Eq. 1),
so the update must equal the plain launch's bit for bit: u_out, costs, and
(through pi_debug_rollout) the per-step costs and perturbations.  The cases
cover one block, a ragged last block, sub-rollouts, mean-only noise, T = 1,
blocks spread over up to 12 CTAs (one output each), the realtime shape (128
blocks, 11 units per CTA) and a partial last wave after a whole one; the
oracle parity of the split path is covered by the end-to-end and full-size
tests, which run it in the default mode.  The failure test leaves the last
CTA out of the grid: the waits on it must give up, report PI_ERR_TIMEOUT and
leave the context usable."""
import numpy as np
import pytest
import torch

from paper_1503_00330_b300 import _lib
from paper_1503_00330_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    build.build()


def _problem(K, T, L, seed, M=1, noise="sampled"):
    p = W.problem(K, T, L, seed=seed, n_obs=5, M=M)
    p.model_noise = noise == "sampled"
    p.u_nom = np.random.default_rng(seed).normal(0, 0.2, (T, 4)).astype(np.float32)
    p.x0 = np.random.default_rng(seed + 1).normal(0, 0.1, 12).astype(np.float32)
    return p


# (K, T, L, M, noise): plan checked below
CASES = [
    (1, 6, 33, 1, "sampled"),          # one block, 12 CTAs of one output each
    (256, 20, 64, 1, "sampled"),       # 4 blocks, one output per CTA
    (1000, 15, 33, 1, "sampled"),      # ragged last block (1000 = 15 x 64 + 40)
    (300, 12, 40, 4, "sampled"),       # sub-rollouts: 1200 slots, 19 blocks
    (700, 9, 130, 1, "mean_only"),     # deterministic dynamics
    (129, 1, 17, 1, "sampled"),        # T = 1
    (8192, 6, 512, 1, "sampled"),      # realtime shape: 128 blocks, 11 units per CTA
    (-640, 5, 96, 1, "sampled"),       # one whole wave of blocks, then a partial wave of 10 (K = 64 SMs + 640)
    (1024, 4, 64, 32, "sampled"),      # the sub-rollout workload's shape: 512 blocks, 3 whole waves + a split tail
]


@pytest.mark.parametrize("K,T,L,M,noise", CASES)
def test_split_equals_plain_bitwise(K, T, L, M, noise):
    from paper_1503_00330_b300.api import Controller
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    if K < 0:
        K = 64 * nsm - K
    p = _problem(K, T, L, seed=K + T + L, M=M, noise=noise)
    ctl = Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, precision="fp32")
    ctl.set_output_split("always")
    plain, upc, ctas = ctl.split_plan(p.K)
    blocks = -(-p.K * p.M // 64)
    tail = blocks % nsm
    assert plain == blocks - tail and 0 < upc < 12 and ctas == -(-tail * 12 // upc) and ctas <= nsm
    outs = {}
    for mode in ("always", "off", "always"):
        ctl.set_output_split(mode)
        u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
        ctl.sync()
        outs.setdefault(mode, []).append((u.clone(), c.clone()))
    (u_s, c_s), (u_s2, c_s2) = outs["always"]
    u_p, c_p = outs["off"][0]
    print(f"K={K} T={T} L={L} M={M}: {plain} plain blocks + {ctas} CTAs x {upc} units")
    assert torch.equal(u_s, u_p) and torch.equal(c_s, c_p), "split launch differs from the plain launch"
    assert torch.equal(u_s2, u_s) and torch.equal(c_s2, c_s), "repeated split launch differs"
    ctl.close()


def test_split_rollout_stage_bitwise():
    """Per-step costs, perturbations and terminal costs of the rollout stage alone."""
    from paper_1503_00330_b300.api import Controller
    p = _problem(2000, 11, 96, seed=4, M=2)
    ctl = Controller(p.model, p.cost, M=p.M, precision="fp32")
    res = {}
    for mode in ("always", "off"):
        ctl.set_output_split(mode)
        res[mode] = [t.cpu().numpy() for t in ctl.debug_rollout(p.x0, p.u_nom, p.K, p.T, p.sigma_u, p.seed)]
        ctl.sync()
    for a, b in zip(res["always"], res["off"]):
        assert np.array_equal(a, b)
    ctl.close()


def test_auto_mode_plan():
    """Default mode: the realtime update (128 blocks) is split over all SMs in
    runs of 11 units; a launch that fills the SMs and a tiny model are not split."""
    from paper_1503_00330_b300.api import Controller
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    p = _problem(8, 2, 512, seed=1)
    ctl = Controller(p.model, p.cost, precision="fp32")
    plain, upc, ctas = ctl.split_plan(8192)
    assert plain == 0 and upc == -(-128 * 12 // nsm) and ctas == -(-128 * 12 // upc)
    assert ctl.split_plan(64 * nsm) == (nsm, 0, 0)                  # one whole wave: plain
    assert ctl.split_plan(64 * (nsm + 1)) == (nsm, 1, 12)           # + one block split 12 ways
    assert ctl.split_plan(64 * (2 * nsm - 1))[1] == 0                # a nearly full last wave: plain
    ctl.set_output_split("off")
    assert ctl.split_plan(8192) == (128, 0, 0)
    ctl.close()
    q = _problem(8, 2, 5, seed=1)   # 3 field pairs per output: (12 - 1) * 3 < 64
    ctl = Controller(q.model, q.cost, precision="fp32")
    assert ctl.split_plan(256) == (4, 0, 0)
    ctl.set_output_split("always")
    assert ctl.split_plan(256) == (0, 1, 48)
    ctl.close()


def test_split_peer_wait_times_out_and_context_recovers():
    from paper_1503_00330_b300.api import Controller
    p = _problem(640, 4, 64, seed=9)
    ctl = Controller(p.model, p.cost, precision="fp32")
    ctl.set_output_split("always")
    u_ref, c_ref = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    u_ref, c_ref = u_ref.clone(), c_ref.clone()
    lib = _lib.load()
    _lib.check(lib.pi_debug_split_drop_cta(ctl.handle, 1))
    ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    with pytest.raises(_lib.PiError) as ei:
        ctl.sync()
    assert ei.value.code == _lib.PI_ERR_TIMEOUT
    _lib.check(lib.pi_debug_split_drop_cta(ctl.handle, 0))
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    assert torch.equal(u, u_ref) and torch.equal(c, c_ref)
    ctl.close()


def test_refused_split_launch_falls_back_to_plain_blocks():
    """A cooperative launch the runtime refuses (fewer SMs open to the process
    than the device has) runs its blocks as plain blocks: same results."""
    from paper_1503_00330_b300.api import Controller
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    p = _problem(64 * nsm + 640, 4, 64, seed=12)
    ctl = Controller(p.model, p.cost, precision="fp32")
    ctl.set_output_split("off")
    u_ref, c_ref = (t.clone() for t in ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed))
    ctl.sync()
    ctl.set_output_split("always")
    lib = _lib.load()
    _lib.check(lib.pi_debug_split_drop_cta(ctl.handle, 2))
    n0 = ctl.launch_count()
    u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
    ctl.sync()
    assert ctl.launch_count() - n0 == 4   # plain whole wave + plain tail + scan + merge
    _lib.check(lib.pi_debug_split_drop_cta(ctl.handle, 0))
    assert torch.equal(u, u_ref) and torch.equal(c, c_ref)
    ctl.close()


def test_split_equals_plain_on_random_shapes():
    """Twelve seeded random shapes (K up to 3 waves of blocks, T, L, M, noise on
    or off): the split launch equals the plain one bit for bit wherever it runs."""
    from paper_1503_00330_b300.api import Controller
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rng = np.random.default_rng(2024)
    ran = 0
    for i in range(12):
        M = int(rng.choice([1, 1, 2, 4, 8]))
        K = int(rng.integers(1, 3 * 64 * nsm // M))
        T = int(rng.integers(1, 9))
        L = int(rng.integers(1, 200))
        p = _problem(K, T, L, seed=100 + i, M=M, noise="sampled" if rng.random() < 0.7 else "mean_only")
        ctl = Controller(p.model, p.cost, M=p.M, model_noise=p.model_noise, precision="fp32")
        ctl.set_output_split("always")
        plan = ctl.split_plan(p.K)
        res = []
        for mode in ("always", "off"):
            ctl.set_output_split(mode)
            u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
            ctl.sync()
            res.append((u.clone(), c.clone()))
        print(f"K={K} T={T} L={L} M={M}: plan {plan}")
        assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1]), f"shape {i} differs"
        ran += plan[1] > 0
        ctl.close()
    assert ran >= 6   # most shapes have a partial wave to split


def test_update_captured_in_a_graph_takes_the_plain_launch():
    """An FP32 update captured into a CUDA graph (here torch's) is launched
    plainly, so replays stay correct: each replay equals the eager update."""
    from paper_1503_00330_b300.api import Controller
    p = _problem(8192, 3, 64, seed=31)
    ctl = Controller(p.model, p.cost, precision="fp32")
    ctl.set_output_split("always")
    u_ref, c_ref = (t.clone() for t in ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed))
    ctl.sync()
    assert ctl.split_plan(p.K)[1] > 0            # eager: split
    x0 = torch.as_tensor(p.x0, device="cuda")
    un = torch.as_tensor(p.u_nom, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        ctl.reserve(p.K, p.T)            # the context moves to s (and its scratch is sized) before the capture
        with torch.cuda.graph(g, stream=s):
            u, c = ctl.update(x0, un, p.K, p.T, p.lam, p.sigma_u, p.seed)
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(u, u_ref) and torch.equal(c, c_ref)
    ctl.sync()
    ctl.close()


def test_concurrent_split_updates_on_two_streams():
    """Two contexts' split updates enqueued on two streams at once (each a
    cooperative grid over most SMs): both complete without a wait expiring and
    equal the same updates run one after the other."""
    from paper_1503_00330_b300.api import Controller
    p = _problem(8192, 12, 256, seed=41)
    ctls = [Controller(p.model, p.cost, precision="fp32") for _ in range(2)]
    for c in ctls:
        c.set_output_split("always")
    seeds = [p.seed, p.seed + 1]
    ref = []
    for c, sd in zip(ctls, seeds):
        u, cs = c.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, sd)
        c.sync()
        ref.append((u.clone(), cs.clone()))
    streams = [torch.cuda.Stream() for _ in range(2)]
    for s in streams:
        s.wait_stream(torch.cuda.current_stream())
    for rep in range(3):
        outs = []
        for c, s, sd in zip(ctls, streams, seeds):
            with torch.cuda.stream(s):
                outs.append(c.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, sd))
        for c in ctls:
            c.sync()            # raises PI_ERR_TIMEOUT if a wait between CTAs expired
        for (u, cs), (ur, cr) in zip(outs, ref):
            assert torch.equal(u, ur) and torch.equal(cs, cr)
    for c in ctls:
        c.close()


def test_split_equals_plain_with_the_papers_cost():
    """The Sec. 5 cost (Gaussian obstacle bumps, crash term, no variance or
    terminal term) through the split launch: bitwise the plain launch's."""
    from paper_1503_00330_b300.api import Controller
    p = W.problem(3000, 10, 80, seed=8, cost=W.paper_cost(n_obs=5, seed=8))
    p.u_nom = np.random.default_rng(8).normal(0, 0.2, (p.T, 4)).astype(np.float32)
    ctl = Controller(p.model, p.cost, precision="fp32")
    res = []
    for mode in ("always", "off"):
        ctl.set_output_split(mode)
        u, c = ctl.update(p.x0, p.u_nom, p.K, p.T, p.lam, p.sigma_u, p.seed)
        ctl.sync()
        res.append((u.clone(), c.clone()))
    assert ctl.split_plan(p.K)[1] == 0          # "off" now; "always" split it
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    ctl.close()

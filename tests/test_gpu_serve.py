"""Serving loop (continuous batching of receding-horizon updates of many
agents over one shared model).

Every served result must equal, bitwise, the same agent's updates run alone on
the single-controller path (pi_update with the agent's n-th seed, then
pi_rh_advance), whatever else is in the mix: the groups a request lands in,
the lanes, the memory-gated admission order.  Plus checkpoint/resume, a
measured-state override, the oracle for one served update, and a short
real-time trace replay."""
import numpy as np
import pytest
import torch

from paper_1503_00330_b300 import workloads as W

pytestmark = pytest.mark.gpu

LAM = 1.0
SU = W.SIGMA_U
# (K, T) of each agent: ragged K (a single rollout, non-multiples of 64 and 128) and T
AGENTS = [(300, 20), (65, 7), (1000, 13), (128, 31), (1, 5), (513, 24)]
T_MAX = 32
ROUNDS = 3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00330_b300 import build
    build.build()


def _controller(form):
    from paper_1503_00330_b300.api import Controller
    return Controller(W.make_lwpr(48, seed=7), W.make_cost(5, seed=7), precision=form)


def _agent_init(n):
    rng = np.random.default_rng(3)
    x0 = rng.normal(0, 0.1, (n, 12)).astype(np.float32)
    warm = rng.normal(0, 0.2, (n, T_MAX, 4)).astype(np.float32)
    seeds = [1000 + 17 * a for a in range(n)]
    return x0, warm, seeds


def _server(ctl, n, **kw):
    from paper_1503_00330_b300.api import Server
    srv = Server(ctl, n, K_max=1024, T_max=T_MAX, want_costs=True, **kw)
    x0, warm, seeds = _agent_init(n)
    for a in range(n):
        srv.set_agent(a, x0[a], warm[a], seeds[a])
    return srv


def _alone_sequence(ctl, a, rounds, x0=None, warm=None, first_round=0):
    """Agent a's updates on the single-controller path: (u_out, costs) per round, final x0."""
    from paper_1503_00330_b300.api import update_seed
    K, T = AGENTS[a]
    x0s, warms, seeds = _agent_init(len(AGENTS))
    x = torch.tensor(x0s[a] if x0 is None else x0, device="cuda")
    u_nom = torch.tensor((warms[a] if warm is None else warm)[:T], device="cuda")
    out = []
    for r in range(first_round, first_round + rounds):
        u, c = ctl.update(x, u_nom, K, T, LAM, SU, update_seed(seeds[a], r))
        u_next = torch.empty_like(u)
        ctl.rh_advance(x, u, u_next)
        ctl.sync()
        out.append((u.cpu().numpy(), c.cpu().numpy()))
        u_nom = u_next
    return out, x.cpu().numpy()


def _serve_all(srv, rounds, agents=None):
    """Submits `rounds` updates of every agent at once; returns {(agent, round): (u, costs, record)}."""
    agents = range(len(AGENTS)) if agents is None else agents
    tickets = {}
    for r in range(rounds):
        for a in agents:
            K, T = AGENTS[a]
            tickets[srv.submit(a, K, T, LAM, SU)] = (a, r)
    done = srv.wait(tickets)
    out = {}
    for t, (a, r) in tickets.items():
        assert done[t]["status"] == 0
        K, T = AGENTS[a]
        u, c = srv.result(t, T, K)
        out[(a, r)] = (u, c, done[t])
    return out


@pytest.mark.parametrize("form", ["fp32", "tc", "tc_fp16x2"])
def test_served_equals_alone_single_controller_path(form):
    ctl = _controller(form)
    srv = _server(ctl, len(AGENTS), max_inflight=3, max_group=4)
    got = _serve_all(srv, ROUNDS)
    srv.drain()
    st = srv.state_save()
    for a in range(len(AGENTS)):
        ref, x_end = _alone_sequence(ctl, a, ROUNDS)
        for r in range(ROUNDS):
            u, c, _ = got[(a, r)]
            assert np.array_equal(u, ref[r][0]), f"agent {a} round {r}: u_out differs"
            assert np.array_equal(c, ref[r][1]), f"agent {a} round {r}: costs differ"
        assert np.array_equal(st["x0"][a], x_end), f"agent {a}: advanced state differs"
        assert int(st["counter"][a]) == ROUNDS
    stats = srv.stats()
    assert stats["completed"] == stats["submitted"] == ROUNDS * len(AGENTS)
    assert stats["peak_group_size"] <= 4 and stats["launches"] == 7 * stats["groups"]
    srv.close()


@pytest.mark.parametrize("form", ["fp32", "tc"])
def test_alone_equals_mixed(form):
    ctl = _controller(form)
    mixed = _server(ctl, len(AGENTS), max_inflight=2, max_group=64)
    got_mixed = _serve_all(mixed, 2)
    mixed.close()
    for a in range(len(AGENTS)):
        alone = _server(ctl, len(AGENTS), max_inflight=1, max_group=1)
        got_alone = _serve_all(alone, 2, agents=[a])
        for r in range(2):
            assert got_alone[(a, r)][2]["group_size"] == 1
            assert np.array_equal(got_alone[(a, r)][0], got_mixed[(a, r)][0]), f"agent {a} round {r}"
            assert np.array_equal(got_alone[(a, r)][1], got_mixed[(a, r)][1]), f"agent {a} round {r}"
        alone.close()
    assert max(int(v[2]["group_size"]) for v in got_mixed.values()) > 1, "the mix never batched two requests"


def _req_bytes(K, T):
    a = lambda v: (v + 255) // 256 * 256  # noqa: E731
    nblk = (K + 63) // 64
    return a(K * T * 4) + a(K * T * 16) + a(K * 4) + a(nblk * T * 48) + a(T * 16 + K * 4)


def test_admission_by_memory():
    """A pool that holds only the two largest requests still serves everything, bitwise as alone."""
    ctl = _controller("fp32")
    biggest = sorted(_req_bytes(K, T) for K, T in AGENTS)[-2:]
    budget = sum(biggest)
    srv = _server(ctl, len(AGENTS), max_inflight=4, max_group=8, hbm_budget=budget)
    got = _serve_all(srv, 2)
    stats = srv.stats()
    assert stats["pool_bytes"] == budget and stats["pool_peak_bytes"] <= budget
    assert stats["memory_waits"] > 0
    for a in range(len(AGENTS)):
        ref, _ = _alone_sequence(ctl, a, 2)
        for r in range(2):
            assert np.array_equal(got[(a, r)][0], ref[r][0]) and np.array_equal(got[(a, r)][1], ref[r][1])
    with pytest.raises(Exception):
        srv.submit(0, 1024, T_MAX, LAM, SU)   # larger than the whole pool
    srv.close()


def test_checkpoint_resume():
    ctl = _controller("fp32")
    a_srv = _server(ctl, len(AGENTS))
    _serve_all(a_srv, 2)
    a_srv.drain()
    snap = a_srv.state_save()
    cont = _serve_all(a_srv, 2)
    a_srv.close()
    b_srv = _server(ctl, len(AGENTS))
    b_srv.state_load(snap)
    resumed = _serve_all(b_srv, 2)
    b_srv.close()
    for key in cont:
        assert np.array_equal(cont[key][0], resumed[key][0]) and np.array_equal(cont[key][1], resumed[key][1])


def test_measured_state_and_busy_agent():
    from paper_1503_00330_b300.api import PiError
    ctl = _controller("fp32")
    srv = _server(ctl, len(AGENTS))
    x_meas = np.linspace(-0.2, 0.2, 12).astype(np.float32)
    K, T = AGENTS[2]
    t = srv.submit(2, K, T, LAM, SU, x0=x_meas)
    with pytest.raises(PiError) as e:
        srv.set_agent(2, np.zeros(12, np.float32))   # the agent has a request outstanding
    assert e.value.code == 7
    srv.wait([t])
    u, c = srv.result(t, T, K)
    ref, _ = _alone_sequence(ctl, 2, 1, x0=x_meas)
    assert np.array_equal(u, ref[0][0]) and np.array_equal(c, ref[0][1])
    with pytest.raises(PiError):
        srv.submit(0, 2048, 5, LAM, SU)      # K > K_max
    with pytest.raises(PiError):
        srv.submit(0, 10, T_MAX + 1, LAM, SU)
    with pytest.raises(PiError):
        srv.submit(len(AGENTS), 10, 5, LAM, SU)
    srv.close()


@pytest.mark.parametrize("form", ["fp32", "tc", "tc_fp16x2"])
def test_served_update_against_oracle(oracle, form):
    from paper_1503_00330_b300.api import update_seed
    ctl = _controller(form)
    srv = _server(ctl, len(AGENTS))
    got = _serve_all(srv, 1)
    srv.close()
    x0s, warms, seeds = _agent_init(len(AGENTS))
    for a in (0, 2, 5):
        K, T = AGENTS[a]
        uref, cref = oracle.pi_update(ctl.model, ctl.cost, x0s[a], warms[a][:T], K, T, LAM, SU,
                                      update_seed(seeds[a], 0))
        scale = np.maximum(np.abs(uref).max(0), np.sqrt(SU.astype(np.float64) / K))
        eu = np.abs(got[(a, 0)][0] - uref).max(0) / scale
        ec = np.max(np.abs(got[(a, 0)][1] - cref) / cref)
        tol = 2e-3 if form == "tc_fp16x2" else 1e-5     # the two-product form's stated bound
        assert np.all(eu <= tol) and ec <= tol, (a, eu, ec)


def test_trace_replay():
    ctl = _controller("tc")
    n = 8
    from paper_1503_00330_b300.api import Server
    srv = Server(ctl, n, K_max=1024, T_max=T_MAX)
    g = np.random.default_rng(11)
    arrivals = []
    for a in range(n):
        t = g.exponential(1 / 50.0)
        while t < 0.3:
            arrivals.append((t, a, int(g.integers(64, 1025)), int(g.integers(5, T_MAX + 1))))
            t += g.exponential(1 / 50.0)
    arrivals.sort()
    rec, dropped = srv.replay(arrivals, LAM, SU)
    assert len(rec) + dropped == len(arrivals)
    assert np.all(rec["status"] == 0)
    assert np.all(rec["t_submit_ns"] <= rec["t_launch_ns"]) and np.all(rec["t_launch_ns"] <= rec["t_result_ns"])
    st = srv.stats()
    assert st["completed"] == len(rec)
    # each agent's counter advanced once per served request
    counts = np.bincount(rec["agent"], minlength=n)
    srv.drain()
    assert np.array_equal(srv.state_save()["counter"].astype(np.int64), counts)
    srv.close()


@pytest.mark.parametrize("split", ["1", "2", "3", "4"])
def test_served_equals_alone_for_each_group_split(monkeypatch, split):
    """Small groups run as one wave of clusters that split each block's outputs
    (split 1: the persistent batched kernel); every split serves the same bits."""
    monkeypatch.setenv("PI2RH_TC_SPLIT", split)
    ctl = _controller("tc")
    srv = _server(ctl, len(AGENTS), max_inflight=2, max_group=3)
    got = _serve_all(srv, 2)
    srv.close()
    for a in range(len(AGENTS)):
        ref, _ = _alone_sequence(ctl, a, 2)
        for r in range(2):
            assert np.array_equal(got[(a, r)][0], ref[r][0]), f"split {split}, agent {a} round {r}"
            assert np.array_equal(got[(a, r)][1], ref[r][1]), f"split {split}, agent {a} round {r}"


def test_cancelled_requests_leave_the_rest_unchanged():
    """Queued requests cancelled on the host never reach the GPU: every other
    request is served exactly as alone, and an agent whose request was cancelled
    continues its own sequence as if the request had never been made."""
    from paper_1503_00330_b300._lib import PI_ERR_CANCELLED, PiError
    ctl = _controller("fp32")
    srv = _server(ctl, len(AGENTS), max_inflight=1, max_group=1)   # a long queue
    tickets = {}
    for r in range(3):
        for a in range(len(AGENTS)):
            K, T = AGENTS[a]
            tickets[srv.submit(a, K, T, LAM, SU)] = (a, r)
    victims = [t for t, ar in tickets.items() if ar in ((2, 1), (5, 2))]
    cancelled = {t for t in victims if srv.cancel(t)}
    assert max(victims) in cancelled            # the last request submitted was still queued
    done = srv.wait(tickets)
    served = {a: [] for a in range(len(AGENTS))}
    for t in sorted(tickets):                   # ticket order is each agent's round order
        a, r = tickets[t]
        if t in cancelled:
            assert done[t]["status"] == PI_ERR_CANCELLED and done[t]["t_launch_ns"] == 0
            continue
        assert done[t]["status"] == 0
        K, T = AGENTS[a]
        served[a].append(srv.result(t, T, K))
    for a in range(len(AGENTS)):
        ref, _ = _alone_sequence(ctl, a, len(served[a]))
        for n, (u, c) in enumerate(served[a]):
            assert np.array_equal(u, ref[n][0]) and np.array_equal(c, ref[n][1]), f"agent {a} request {n}"
    assert srv.cancel(max(victims)) is False     # finished: nothing to cancel
    with pytest.raises(PiError):
        srv.cancel(10 ** 9)                     # never issued
    srv.drain()
    assert int(srv.state_save()["counter"][5]) == 2
    srv.close()


@pytest.mark.parametrize("form", ["tc", "tc_fp16x2"])
def test_served_at_full_size_sampled(oracle, form):
    """The serving workload's own sizes (one shared L = 1024 model, 16 obstacles,
    K up to 16384, T up to 120): three requests served in one mix; S_{k,0} of the
    32 first and 32 last rollouts of each against the oracle (rollout k depends only
    on its own noise counters, so a range is run alone)."""
    from paper_1503_00330_b300.api import Controller, Server, update_seed
    model, cost = W.make_lwpr(1024, seed=4), W.make_cost(16, seed=4)
    ctl = Controller(model, cost, precision=form)
    sizes = [(16384, 120), (2048, 50), (9001, 85)]
    srv = Server(ctl, len(sizes), K_max=16384, T_max=120, want_costs=True)
    rng = np.random.default_rng(11)
    x0 = rng.normal(0, 0.1, (len(sizes), 12)).astype(np.float32)
    warm = rng.normal(0, 0.2, (len(sizes), 120, 4)).astype(np.float32)
    seeds = [5000 + a for a in range(len(sizes))]
    for a in range(len(sizes)):
        srv.set_agent(a, x0[a], warm[a], seeds[a])
    tickets = {srv.submit(a, K, T, LAM, SU): a for a, (K, T) in enumerate(sizes)}
    done = srv.wait(tickets)
    tol = 2e-3 if form == "tc_fp16x2" else 1e-5
    for t, a in tickets.items():
        assert done[t]["status"] == 0
        K, T = sizes[a]
        _, c = srv.result(t, T, K)
        for k0 in (0, K - 32):
            r = oracle.rollouts(model, cost, x0[a], warm[a][:T], 32, T, SU, update_seed(seeds[a], 0), k0=k0)
            S0 = oracle.cost_to_go(r["cost"], r["phi"], float(model.dt))[:, 0]
            err = np.abs(c[k0:k0 + 32].astype(np.float64) - S0) / S0
            print(f"served {form} K={K} T={T} rollouts {k0}..{k0 + 31}: S0 max rel err {err.max():.3g}")
            assert np.all(err <= tol)
    srv.close()

"""Planning rules of the FP32 output-split launch, on the host alone
(pi_debug_split_plan_sizes: no context, no GPU).

For every size: the plain launch takes whole waves of 64-slot blocks and the
split launch the rest; a split happens only for a partial wave, with fewer
than 12 (block, output) units per CTA and at most one CTA per SM; the auto
mode also wants the work it saves to outweigh its two flag round trips per
step, (12 - units) * ceil(L / 2) >= 64; off never splits.  Spot values: the
realtime update (K = 8192 on 148 SMs) runs as 140 CTAs of 11 units, one
whole wave plus ten blocks as 148 plain CTAs and 120 of one unit."""
import ctypes

import pytest

from paper_1503_00330_b300 import _lib, build

OFF, AUTO, ALWAYS = _lib.PI_SPLIT_OFF, _lib.PI_SPLIT_AUTO, _lib.PI_SPLIT_ALWAYS


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def plan(lib, K, M, L, nsm, mode):
    pb, upc, ctas = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _lib.check(lib.pi_debug_split_plan_sizes(K, M, L, nsm, mode, ctypes.byref(pb), ctypes.byref(upc),
                                              ctypes.byref(ctas)))
    return pb.value, upc.value, ctas.value


def test_spot_values(lib):
    assert plan(lib, 8192, 1, 512, 148, AUTO) == (0, 11, 140)
    assert plan(lib, 64 * 148 + 640, 1, 96, 148, AUTO) == (148, 1, 120)
    assert plan(lib, 1024, 32, 512, 148, AUTO) == (444, 6, 136)
    assert plan(lib, 8192, 1, 512, 148, OFF) == (128, 0, 0)
    assert plan(lib, 9472, 1, 512, 148, AUTO) == (148, 0, 0)       # one whole wave: plain
    assert plan(lib, 256, 1, 5, 148, AUTO) == (4, 0, 0)            # (12 - 1) * 3 < 64
    assert plan(lib, 256, 1, 5, 148, ALWAYS) == (0, 1, 48)


@pytest.mark.parametrize("nsm", [1, 2, 7, 20, 132, 148, 160])
def test_invariants(lib, nsm):
    for K in list(range(1, 300, 7)) + [64 * nsm * w + d for w in (0, 1, 3) for d in (-64, -1, 1, 64, 640, 6400)]:
        if K < 1:
            continue
        for M in (1, 4, 32):
            blocks = -(-K * M // 64)
            for L in (1, 9, 64, 512):
                P = (L + 1) // 2
                for mode in (OFF, AUTO, ALWAYS):
                    pb, upc, ctas = plan(lib, K, M, L, nsm, mode)
                    tail = blocks % nsm
                    if upc == 0:
                        assert pb == blocks and ctas == 0
                        if mode != OFF and tail and -(-tail * 12 // nsm) < 12:
                            assert mode == AUTO and (12 - -(-tail * 12 // nsm)) * P < 64
                        continue
                    assert mode != OFF
                    assert pb == blocks - tail and tail > 0 and pb % nsm == 0
                    assert upc == -(-tail * 12 // nsm) and 0 < upc < 12
                    assert ctas == -(-tail * 12 // upc) and ctas <= nsm
                    if mode == AUTO:
                        assert (12 - upc) * P >= 64


def test_rejects_bad_sizes(lib):
    out = [ctypes.c_int() for _ in range(3)]
    for args in ((0, 1, 8, 148, AUTO), (8, 0, 8, 148, AUTO), (8, 1, 0, 148, AUTO), (8, 1, 8, 0, AUTO), (8, 1, 8, 148, 7)):
        assert lib.pi_debug_split_plan_sizes(*args, *[ctypes.byref(o) for o in out]) == _lib.PI_ERR_INVALID_ARG


def partition(lib, blocks, upc):
    """Per CTA: list of segments (block, o0, o1, owned, parts_or_index) from the kernel's own plan."""
    units = blocks * 12
    ctas = -(-units // upc)
    out = []
    seg = (ctypes.c_int * 10)()
    n = ctypes.c_int()
    for c in range(ctas):
        _lib.check(lib.pi_debug_split_partition(blocks, upc, c, seg, ctypes.byref(n)))
        out.append([tuple(seg[5 * i:5 * i + 5]) for i in range(n.value)])
    assert lib.pi_debug_split_partition(blocks, upc, ctas, seg, ctypes.byref(n)) == _lib.PI_ERR_INVALID_ARG
    return out


def simulate(parts, blocks, T=3):
    """Runs the split kernel's flag protocol (publish / wait ready, done / wait
    done) over T steps under a round-robin schedule; True when every CTA finishes."""
    ready = {}
    done = {}
    progs = []
    for segs in parts:
        ev = []
        own = [s for s in segs if s[3]]
        if own:
            ev.append(("pub", own[0][0], 1))
        for t in range(T):
            for b, o0, o1, owned, idx in segs:
                if not owned:
                    ev += [("wait_ready", b, t + 1), ("done", b, idx, t + 1)]
            if own:
                b, _, _, _, nparts = own[0]
                ev += [("wait_done", b, p, t + 1) for p in range(nparts)]
                if t + 1 < T:
                    ev.append(("pub", b, t + 2))
        progs.append(ev)
    pc = [0] * len(progs)
    moved = True
    while moved:
        moved = False
        for c, ev in enumerate(progs):
            while pc[c] < len(ev):
                e = ev[pc[c]]
                if e[0] == "pub":
                    ready[e[1]] = e[2]
                elif e[0] == "done":
                    done[(e[1], e[2])] = e[3]
                elif e[0] == "wait_ready" and ready.get(e[1], 0) < e[2]:
                    break
                elif e[0] == "wait_done" and done.get((e[1], e[2]), 0) < e[3]:
                    break
                pc[c] += 1
                moved = True
    return all(pc[c] == len(ev) for c, ev in enumerate(progs))


@pytest.mark.parametrize("nsm", [2, 7, 20, 148, 160])
def test_kernel_partition_covers_every_unit_once_and_cannot_deadlock(lib, nsm):
    for blocks in range(1, nsm + 1):
        upc = -(-blocks * 12 // nsm)
        if upc >= 12:
            continue
        parts = partition(lib, blocks, upc)
        seen = {}
        owners = {}
        nonowner_idx = {}
        for c, segs in enumerate(parts):
            assert 1 <= len(segs) <= 2 and sum(s[3] for s in segs) <= 1
            assert len(segs) == 1 or not segs[0][3], "the non-owned segment comes first"
            for b, o0, o1, owned, idx in segs:
                assert 0 <= b < blocks and 0 <= o0 < o1 <= 12
                for o in range(o0, o1):
                    assert (b, o) not in seen
                    seen[(b, o)] = c
                if owned:
                    assert o1 == 12 and o0 > 0
                    owners[b] = (c, idx)
                else:
                    nonowner_idx.setdefault(b, []).append(idx)
        assert len(seen) == blocks * 12
        for b in range(blocks):
            c, nparts = owners[b]
            assert sorted(nonowner_idx.get(b, [])) == list(range(nparts)) and 1 <= nparts <= 11
        assert simulate(parts, blocks), f"flag protocol cannot finish for {blocks} blocks on {nsm} SMs"

"""Host logic of the serving engine, without a GPU: the pool allocator that
gates admission by memory, checked against a brute-force first-fit model of
the same pool (one byte-map over the whole capacity)."""
import numpy as np
import pytest

from paper_1503_00330_b300.api import PiError, debug_pool


def _unit(n):
    return (max(n, 1) + 255) // 256 * 256


class _BruteFirstFit:
    """Byte-map first fit: lowest offset whose run of free units is long enough."""

    def __init__(self, cap):
        self.free = np.ones(cap // 256, bool)

    def alloc(self, n):
        u = _unit(n) // 256
        run = 0
        for i, f in enumerate(self.free):
            run = run + 1 if f else 0
            if run == u:
                s = i - u + 1
                self.free[s:i + 1] = False
                return s * 256
        return -1

    def release(self, off, n):
        self.free[off // 256: (off + _unit(n)) // 256] = True

    def extents(self):
        f = self.free.astype(np.int8)
        return int(np.sum(np.diff(np.concatenate([[0], f])) == 1))


@pytest.mark.parametrize("seed", range(6))
def test_pool_matches_brute_force_first_fit(seed):
    g = np.random.default_rng(seed)
    cap = 64 * 1024 + 100                 # the pool keeps whole 256-byte units only
    bf = _BruteFirstFit(cap & ~255)
    ops, expect, live = [], [], []        # live: indices of successful allocations not yet freed
    for _ in range(400):
        if live and g.random() < 0.45:
            j = live.pop(int(g.integers(len(live))))
            bf.release(expect[j], ops[j][1])
            ops.append(("free", j))
            expect.append(expect[j])
            expect[j] = -2
        else:
            n = int(g.integers(1, 9000))
            o = bf.alloc(n)
            ops.append(("alloc", n))
            expect.append(o)
            if o >= 0:
                live.append(len(ops) - 1)
    assert -1 in expect                   # the sequence exercised "does not fit"
    off, ext = debug_pool(cap, ops)
    assert list(off) == expect
    assert ext == bf.extents()


def test_pool_alignment_and_no_overlap():
    g = np.random.default_rng(9)
    sizes = [int(s) for s in g.integers(1, 5000, 50)]
    off, _ = debug_pool(1 << 20, [("alloc", s) for s in sizes])
    spans = sorted((o, o + _unit(s)) for o, s in zip(off, sizes) if o >= 0)
    assert all(o % 256 == 0 for o, _ in spans)
    assert all(a_end <= b_start for (_, a_end), (b_start, _) in zip(spans, spans[1:]))
    assert spans[-1][1] <= 1 << 20


def test_pool_coalesces_back_to_one_extent():
    cap = 256 * 100
    ops = [("alloc", 256 * 10)] * 10
    order = [3, 7, 0, 9, 1, 5, 2, 8, 4, 6]
    ops += [("free", i) for i in order]
    ops.append(("alloc", cap))
    off, ext = debug_pool(cap, ops)
    assert list(off[:10]) == [-2] * 10                        # every allocation was freed
    assert list(off[10:20]) == [256 * 10 * i for i in order]  # ... from where it had been placed
    assert off[-1] == 0 and ext == 0      # the whole pool is one block again, then fully taken


def test_pool_first_fit_reuses_lowest_hole_and_reports_no_fit():
    cap = 256 * 16
    ops = [("alloc", 256 * 4)] * 4 + [("free", 1), ("free", 2), ("alloc", 256 * 2), ("alloc", 256 * 9),
                                      ("alloc", 256 * 6)]
    off, ext = debug_pool(cap, ops)
    assert off[6] == 256 * 4           # lowest hole
    assert off[7] == -1                # 9 units never fit in the 6 free units
    assert off[8] == 256 * 6           # the rest of the merged hole
    assert ext == 0


def test_pool_rejects_bad_frees():
    with pytest.raises(PiError):
        debug_pool(4096, [("free", 0)])
    with pytest.raises(PiError):
        debug_pool(4096, [("alloc", 100), ("free", 0), ("free", 0)])

"""The CPU oracle against what the paper and the mathematics fix (CPU only)."""
import numpy as np
import pytest

import oracle
import _pins


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("check", _pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(orc, check):
    assert check(orc) == []


def test_invariants_medium(orc):
    """Exactly k outputs; all of them <= the rank-k pair; the others > it;
    #{pairs < kth} = k - 1 (Section 4 problem statement)."""
    g = np.random.Generator(np.random.Philox(11))
    n = 20000
    keys = (g.integers(0, 300, size=n)).astype(np.uint32)
    perm = orc.sort_order(keys, "u32")
    for k in (1, 2, 999, 10000, n):
        sel, kth = orc.select(keys, "u32", k)
        assert sel.size == k and np.unique(sel).size == k
        kv = (int(keys[kth]), kth)
        pairs_sel = {(int(keys[i]), int(i)) for i in sel}
        assert max(pairs_sel) == kv
        mask = np.ones(n, bool)
        mask[sel] = False
        rest = np.nonzero(mask)[0]
        assert all((int(keys[i]), int(i)) > kv for i in rest[:2000])
        below = np.sum((keys < kv[0]) | ((keys == kv[0]) & (np.arange(n) < kv[1])))
        assert below == k - 1
        assert np.array_equal(np.sort(sel), np.sort(perm[:k]))


def test_runs_invariants(orc):
    g = np.random.Generator(np.random.Philox(12))
    p = 50
    lens = g.integers(0, 400, size=p)
    off = np.zeros(p + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    keys = g.integers(0, 100, size=int(off[-1]), dtype=np.uint64)
    for r in range(p):
        keys[int(off[r]):int(off[r + 1])].sort()
    total = int(off[-1])
    for k in (1, 17, total // 2, total):
        split, kr, kp = orc.select_runs(keys, off, k)
        assert int(split.sum()) == k
        assert np.all(split <= lens.astype(np.uint64))
        # rank-k pair is the last selected element of its run
        assert split[kr] == kp + 1
        kv = (int(keys[int(off[kr]) + kp]), kr, kp)
        for r in range(p):
            c = int(split[r])
            if c > 0:   # last selected of run r is <= kth
                assert (int(keys[int(off[r]) + c - 1]), r, c - 1) <= kv
            if c < lens[r]:  # first unselected of run r is > kth
                assert (int(keys[int(off[r]) + c]), r, c) > kv


def test_rejects_bad_arguments(orc):
    keys = np.arange(10, dtype=np.uint32)
    with pytest.raises(ValueError):
        orc.select(keys, "u32", 0)
    with pytest.raises(ValueError):
        orc.select(keys, "u32", 11)
    with pytest.raises(ValueError):
        orc.select_runs(np.arange(4, dtype=np.uint64), np.array([0, 2, 4], np.uint64), 5)

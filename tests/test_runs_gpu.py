"""topk_select_sorted_runs on the GPU against the CPU oracle (bit-exact).

Multisequence selection (Section 4.2, Appendix A): split positions per run
and the rank-k object, ties ordered by (run, position).  Small cases cover
empty runs, single runs, heavy ties and every k class; the full
configuration (1024 runs of 2^U(10,20) sorted u64 keys) is checked by the
properties that fix the answer uniquely.
"""
import numpy as np
import pytest

import oracle
from paper_1502_03942_gb300 import workloads as wl

from _gpu import bits_of, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03942_gb300 as tk
    return tk


@pytest.fixture(scope="module")
def ctx(tk):
    c = tk.Context(0)
    yield c
    c.close()


def make_runs(p, maxlen, seed, alphabet=None):
    g = np.random.Generator(np.random.Philox(seed))
    lens = g.integers(0, maxlen + 1, size=p)
    if lens.sum() == 0:
        lens[0] = 1
    off = np.zeros(p + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    if alphabet:
        keys = (g.integers(0, alphabet, size=int(off[-1])) * 1000003).astype(np.uint64)
    else:
        keys = g.integers(0, np.iinfo(np.uint64).max, size=int(off[-1]), dtype=np.uint64, endpoint=True)
    for r in range(p):
        keys[int(off[r]):int(off[r + 1])].sort()
    return keys, off


def run_and_check(tk, ctx, keys, off, k, params=None):
    d_keys = to_device(keys, "u64")
    d_off = to_device(off, "u64")
    split, kk, kr, kp = tk.topk_select_sorted_runs(ctx, d_keys, d_off, k, params=params)
    want_split, want_run, want_pos = oracle.select_runs(keys, off, k)
    assert np.array_equal(bits_of(split)[: off.size - 1], want_split), "splits differ"
    assert int(bits_of(kr)[0]) == want_run and int(bits_of(kp)[0]) == want_pos, "rank-k object differs"
    assert int(bits_of(kk)[0]) == int(keys[int(off[want_run]) + want_pos])


@pytest.mark.parametrize("p,maxlen,alphabet", [(1, 5000, None), (3, 40, 4), (17, 3000, None),
                                               (64, 2000, 10), (300, 700, None), (1024, 300, 50)])
def test_runs_small(tk, ctx, p, maxlen, alphabet):
    keys, off = make_runs(p, maxlen, seed=p * 7 + maxlen, alphabet=alphabet)
    total = int(off[-1])
    for k in sorted({1, 2, total // 3 + 1, total // 2, max(1, total - 1), total}):
        run_and_check(tk, ctx, keys, off, k)


def test_runs_pivot_count_does_not_change_result(tk, ctx):
    keys, off = make_runs(200, 5000, seed=5)
    total = int(off[-1])
    for d in (1, 2, 8, 256):
        run_and_check(tk, ctx, keys, off, total // 2 + 17, params=tk.make_params(sample_size=d))


def test_runs_bad_k_and_unsorted(tk, ctx):
    import torch
    keys, off = make_runs(10, 100, seed=9)
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    with pytest.raises(tk.TopkError) as e:
        tk.topk_select_sorted_runs(ctx, d_keys, d_off, int(off[-1]) + 1)
    assert e.value.status == tk.TOPK_EINVAL
    bad = keys.copy()
    r0, r1 = int(off[3]), int(off[4])
    if r1 - r0 >= 2:
        bad[r0], bad[r1 - 1] = bad[r1 - 1], bad[r0]
    with pytest.raises(tk.TopkError) as e:
        tk.topk_select_sorted_runs(ctx, to_device(bad, "u64"), d_off, 5,
                                   params=tk.make_params(flags=tk.TOPK_FLAG_CHECK_SORTED))
    assert e.value.status == tk.TOPK_EINVAL


@pytest.mark.parametrize("kind", ["one", "2^16", "half"])
def test_runs_config_full_size(tk, ctx, kind):
    """1024 sorted u64 runs of 2^U(10,20) keys: properties that fix the answer."""
    keys, off = wl.sorted_runs(1024, 10, 20, seed=3)
    total = int(off[-1])
    k = {"one": 1, "2^16": 1 << 16, "half": total // 2}[kind]
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    split, kk, kr, kp = tk.topk_select_sorted_runs(ctx, d_keys, d_off, k)
    split = bits_of(split).astype(np.int64)
    lens = np.diff(off).astype(np.int64)
    kr, kp, kk = int(bits_of(kr)[0]), int(bits_of(kp)[0]), int(bits_of(kk)[0])
    assert split.sum() == k and np.all(split >= 0) and np.all(split <= lens)
    g_k = int(off[kr]) + kp
    assert kk == int(keys[g_k]) and split[kr] == kp + 1
    # last selected of every run <= (kk, g_k) < first unselected, on (key, global index)
    starts = off[:-1].astype(np.int64)
    has_sel = split > 0
    last_g = starts + split - 1
    lk = keys[last_g[has_sel]]
    assert np.all((lk < kk) | ((lk == kk) & (last_g[has_sel] <= g_k)))
    has_rest = split < lens
    first_g = starts + split
    fk = keys[first_g[has_rest]]
    assert np.all((fk > kk) | ((fk == kk) & (first_g[has_rest] > g_k)))


def run_flexible_and_check(tk, ctx, keys, off, kmin, kmax, params=None):
    """The k returned lies in [kmin, kmax] (kmax clamped to the total) and the
    selection equals the oracle's for that k."""
    d_keys = to_device(keys, "u64")
    d_off = to_device(off, "u64")
    split, kk, kr, kp, kout = tk.topk_select_sorted_runs_flexible(ctx, d_keys, d_off, kmin, kmax, params=params)
    k = int(bits_of(kout)[0])
    assert kmin <= k <= min(kmax, int(off[-1])), (kmin, kmax, k)
    want_split, want_run, want_pos = oracle.select_runs(keys, off, k)
    assert np.array_equal(bits_of(split)[: off.size - 1], want_split), "splits differ"
    assert int(bits_of(split)[: off.size - 1].sum()) == k
    assert int(bits_of(kr)[0]) == want_run and int(bits_of(kp)[0]) == want_pos, "rank-k object differs"
    assert int(bits_of(kk)[0]) == int(keys[int(off[want_run]) + want_pos])
    return k


@pytest.mark.parametrize("p,maxlen", [(1, 50000), (7, 20000), (300, 3000), (1024, 40000)])
def test_flexible_ranges(tk, ctx, p, maxlen):
    keys, off = make_runs(p, maxlen, seed=81 + p)
    total = int(off[-1])
    ranges = [(1, 1), (1, 10), (100, 200), (total // 3, total // 3 + total // 20), (total // 2, total // 2),
              (total - 10, total + 1000), (5000, 5000 + 5000 // 64), (1, total)]
    for kmin, kmax in ranges:
        kmin = max(1, min(kmin, total))
        run_flexible_and_check(tk, ctx, keys, off, kmin, max(kmin, kmax))


def test_flexible_ties_and_seeds(tk, ctx):
    """Heavy ties; several seeds and trial counts: the k may differ, the
    selection for it never does."""
    keys, off = make_runs(64, 5000, seed=91, alphabet=5)
    total = int(off[-1])
    ks = set()
    for seed, d in ((1, 64), (2, 64), (3, 8), (4, 256)):
        p = tk.make_params(seed=seed, sample_size=d)
        ks.add(run_flexible_and_check(tk, ctx, keys, off, total // 4, total // 4 + total // 10, params=p))
    assert ks


def test_flexible_rejects_bad_ranges(tk, ctx):
    keys, off = make_runs(4, 100, seed=92)
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    for kmin, kmax in ((0, 5), (6, 5)):
        with pytest.raises(tk.TopkError) as e:
            tk.topk_select_sorted_runs_flexible(ctx, d_keys, d_off, kmin, kmax)
        assert e.value.status == tk.TOPK_EINVAL


def test_flexible_full_configuration(tk, ctx):
    """1024 runs of 2^U(10,20) sorted u64 keys, k within 10% above 2^16 and
    above total/2: in range, and the splits are the k smallest for the k
    chosen (the properties that fix the answer uniquely)."""
    keys, off = wl.sorted_runs(1024, 10, 20, seed=3)
    total = int(off[-1])
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    lens = np.diff(off).astype(np.int64)
    starts = off[:-1].astype(np.int64)
    for kmin in (1 << 16, total // 2):
        kmax = kmin + kmin // 10
        split, kk, kr, kp, kout = tk.topk_select_sorted_runs_flexible(ctx, d_keys, d_off, kmin, kmax)
        k = int(bits_of(kout)[0])
        assert kmin <= k <= kmax
        split = bits_of(split).astype(np.int64)
        kr, kp, kk = int(bits_of(kr)[0]), int(bits_of(kp)[0]), int(bits_of(kk)[0])
        assert split.sum() == k and np.all(split >= 0) and np.all(split <= lens)
        g_k = int(off[kr]) + kp
        assert kk == int(keys[g_k]) and split[kr] == kp + 1
        has_sel = split > 0
        last_g = starts + split - 1
        lk = keys[last_g[has_sel]]
        assert np.all((lk < kk) | ((lk == kk) & (last_g[has_sel] <= g_k)))
        has_rest = split < lens
        first_g = starts + split
        fk = keys[first_g[has_rest]]
        assert np.all((fk > kk) | ((fk == kk) & (first_g[has_rest] > g_k)))


# ---- bulk deleteMin* over sorted runs with cursors (Section 5) ----

def pop_and_check(tk, ctx, keys, off, d_keys, d_off, d_cur, cursor, k, params=None):
    kk, kr, kp = tk.topk_runs_delete_min(ctx, d_keys, d_off, d_cur, k, params=params)
    want, wr, wp = oracle.runs_delete_min(keys, off, cursor, k)
    assert np.array_equal(bits_of(d_cur), want), "cursors differ"
    assert (int(bits_of(kr)[0]), int(bits_of(kp)[0])) == (wr, wp), "largest deleted object differs"
    assert int(bits_of(kk)[0]) == int(keys[int(off[wr]) + wp])
    return want


@pytest.mark.parametrize("p,maxlen,alphabet", [(1, 20000, None), (5, 3000, 3), (64, 2000, None),
                                               (700, 400, 20), (1024, 3000, None)])
def test_delete_min_sequence(tk, ctx, p, maxlen, alphabet):
    """Pops of random sizes from empty cursors until the queue is empty; each
    pop against the oracle's deleteMin*."""
    keys, off = make_runs(p, maxlen, seed=101 + p, alphabet=alphabet)
    total = int(off[-1])
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    cursor = np.zeros(p, np.uint64)
    d_cur = to_device(cursor, "u64")
    g = np.random.Generator(np.random.Philox(p))
    left = total
    sizes = [1, 2, 1000]
    while left > 0:
        k = sizes.pop(0) if sizes else int(g.integers(1, max(2, total // 5)))
        k = min(k, left)
        cursor = pop_and_check(tk, ctx, keys, off, d_keys, d_off, d_cur, cursor, k)
        left -= k
    assert np.array_equal(cursor, np.diff(off))


def test_delete_min_from_given_cursors(tk, ctx):
    """Arbitrary starting cursors, some at 0, some at the run's end; the
    composition of two pops equals one pop of their sum."""
    keys, off = make_runs(300, 2000, seed=111, alphabet=50)
    lens = np.diff(off)
    g = np.random.Generator(np.random.Philox(7))
    cursor = np.array([int(g.integers(0, l + 1)) for l in lens], np.uint64)
    cursor[:10] = 0
    cursor[10:20] = lens[10:20]
    remain = int((lens - cursor).sum())
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    for k1, k2 in ((1, 1), (remain // 3, remain // 5), (remain - 1, 1)):
        d_cur = to_device(cursor, "u64")
        c1 = pop_and_check(tk, ctx, keys, off, d_keys, d_off, d_cur, cursor, k1)
        c2 = pop_and_check(tk, ctx, keys, off, d_keys, d_off, d_cur, c1, k2)
        d_once = to_device(cursor, "u64")
        tk.topk_runs_delete_min(ctx, d_keys, d_off, d_once, k1 + k2)
        assert np.array_equal(bits_of(d_once), c2)


def test_delete_min_rejects(tk, ctx):
    keys, off = make_runs(8, 100, seed=112)
    lens = np.diff(off)
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    cursor = lens.copy()
    cursor[0] = 0
    with pytest.raises(tk.TopkError) as e:  # more than remain
        tk.topk_runs_delete_min(ctx, d_keys, d_off, to_device(cursor, "u64"), int(lens[0]) + 1)
    assert e.value.status == tk.TOPK_EINVAL
    bad = np.zeros(8, np.uint64)
    bad[3] = lens[3] + 1  # cursor past its run
    with pytest.raises(tk.TopkError) as e:
        tk.topk_runs_delete_min(ctx, d_keys, d_off, to_device(bad, "u64"), 1)
    assert e.value.status == tk.TOPK_EINVAL
    # the context stays usable
    d_cur = to_device(np.zeros(8, np.uint64), "u64")
    pop_and_check(tk, ctx, keys, off, d_keys, d_off, d_cur, np.zeros(8, np.uint64), 5)


def test_delete_min_flexible_sequence(tk, ctx):
    """Flexible pops: each k in its range, the cursors those of the oracle's
    deleteMin* for that k; clamped at the end of the queue."""
    keys, off = make_runs(200, 5000, seed=113)
    total = int(off[-1])
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    cursor = np.zeros(200, np.uint64)
    d_cur = to_device(cursor, "u64")
    left = total
    step = total // 7
    while left > 0:
        kmin = min(step, left)
        kmax = kmin + step // 8
        kk, kr, kp, kout = tk.topk_runs_delete_min_flexible(ctx, d_keys, d_off, d_cur, kmin, kmax)
        k = int(bits_of(kout)[0])
        assert kmin <= k <= min(kmax, left)
        want, wr, wp = oracle.runs_delete_min(keys, off, cursor, k)
        assert np.array_equal(bits_of(d_cur), want)
        assert (int(bits_of(kr)[0]), int(bits_of(kp)[0])) == (wr, wp)
        cursor = want
        left -= k
    assert np.array_equal(cursor, np.diff(off))


def test_delete_min_full_configuration(tk, ctx):
    """1024 runs of 2^U(10,20) sorted u64 keys: three pops of 2^16 leave the
    cursors of one selection of 3 * 2^16, and every run's last deleted
    object is below the largest deleted, its first remaining one above."""
    keys, off = wl.sorted_runs(1024, 10, 20, seed=3)
    d_keys, d_off = to_device(keys, "u64"), to_device(off, "u64")
    import torch
    d_cur = torch.zeros(1024, dtype=torch.uint64, device="cuda")
    for _ in range(3):
        kk, kr, kp = tk.topk_runs_delete_min(ctx, d_keys, d_off, d_cur, 1 << 16)
    split, _, _, _ = tk.topk_select_sorted_runs(ctx, d_keys, d_off, 3 << 16)
    cur = bits_of(d_cur).astype(np.int64)
    assert np.array_equal(cur, bits_of(split).astype(np.int64))
    lens = np.diff(off).astype(np.int64)
    starts = off[:-1].astype(np.int64)
    kr, kp, kk = int(bits_of(kr)[0]), int(bits_of(kp)[0]), int(bits_of(kk)[0])
    g_k = int(off[kr]) + kp
    assert cur.sum() == 3 << 16 and kk == int(keys[g_k]) and cur[kr] == kp + 1
    has = cur > 0
    lk = keys[(starts + cur - 1)[has]]
    assert np.all((lk < kk) | ((lk == kk) & ((starts + cur - 1)[has] <= g_k)))
    rest = cur < lens
    fk = keys[(starts + cur)[rest]]
    assert np.all((fk > kk) | ((fk == kk) & ((starts + cur)[rest] > g_k)))

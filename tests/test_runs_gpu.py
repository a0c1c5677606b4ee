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

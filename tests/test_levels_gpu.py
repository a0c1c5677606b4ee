"""The grid levels of topk_select at every size class (GPU): three launches
per grid level (sample, pivots, pass) and the finish, the number of grid
levels predicted on the host from the pivot-rank rule.

Each case checks the launch count (counted by the context's measurement
hooks: 3 per level plus the finish) and that the result is the oracle's, bit
for bit, including forced pivot failures and candidate overflows, the k
largest, the rank-k-only call, an unaligned input and heavy ties.
"""
import numpy as np
import pytest

import oracle
from paper_1502_03942_gb300 import workloads as wl

from _gpu import bits_of, check_against_oracle, to_device

pytestmark = pytest.mark.gpu

SMALL_MAX = 1 << 22  # sizes up to here: one or two grid levels at small k


@pytest.fixture(scope="module")
def tk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03942_gb300 as tk
    return tk


@pytest.fixture(scope="module")
def ctx(tk):
    c = tk.Context(0)
    c.profile(True)
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def keys_for(name, n, seed):
    g = np.random.Generator(np.random.Philox(seed))
    if name in ("u32", "i32"):
        return wl.uniform_u32(n, seed)
    if name == "f32":
        return wl.normal_f32(n, seed).view(np.uint32)
    if name == "bf16":
        return g.integers(0, 1 << 16, size=n, dtype=np.uint32).astype(np.uint16)
    return wl.uniform_u64(n, seed)


def launches_of(ctx, run):
    ctx.profile_read(reset=True)
    out = run()
    return out, ctx.profile_read(reset=True)["launches"]


# (key type, n, k): sizes from just above the one-block range to 2^22, ragged
# and power-of-two; k from 2 to n - 1 (one grid level or several)
CASES = [
    ("u32", 16385, 2),
    ("u32", 16385, 8192),
    ("u32", 1 << 20, 1000),
    ("u32", 1 << 20, 1 << 19),
    ("u32", SMALL_MAX, 4000),
    ("u32", SMALL_MAX, SMALL_MAX - 1),
    ("i32", 300007, 777),
    ("i32", 300007, 100002),
    ("f32", (1 << 21) + 3, 100),
    ("f32", SMALL_MAX, 3000),
    ("f32", SMALL_MAX, SMALL_MAX // 2),
    ("bf16", SMALL_MAX, 5000),
    ("bf16", 999_999, 2),
    ("bf16", 999_999, 499_999),
    ("u64", 1_000_003, 50),
    ("u64", 1_000_003, 333_334),
    ("u64", SMALL_MAX, 100),
]


@pytest.mark.parametrize("name,n,k", CASES)
def test_levels_exact(tk, ctx, orc, name, n, k):
    keys = keys_for(name, n, seed=n % 9973 + k)
    d = to_device(keys, name)
    out, launches = launches_of(ctx, lambda: tk.topk_select(ctx, d, k))
    assert launches > 1 and (launches - 1) % 3 == 0
    check_against_oracle(keys, name, k, out, orc)
    # a second call on the same context (counters and sample reused)
    out, launches2 = launches_of(ctx, lambda: tk.topk_select(ctx, d, k))
    assert launches2 == launches
    check_against_oracle(keys, name, k, out, orc)


@pytest.mark.parametrize("name,n", [("u32", SMALL_MAX + 1), ("f32", (1 << 24) + 5), ("u64", (1 << 23) + 3)])
def test_grid_levels_large(tk, ctx, orc, name, n):
    """Larger inputs, every k class: three launches per grid level (sample,
    pivots, pass), then the finish."""
    keys = keys_for(name, n, seed=5)
    d = to_device(keys, name)
    for k in (2, 100, 1 << 16, n // 3, n // 2, n - 1):
        out, launches = launches_of(ctx, lambda: tk.topk_select(ctx, d, k))
        assert launches > 1 and (launches - 1) % 3 == 0
        check_against_oracle(keys, name, k, out, orc)


def test_large_forced_failures_and_overflows(tk, ctx, orc):
    """A margin far too narrow misses rank k and candidate buffers of T pairs
    overflow, on an input above 2^22 keys; the results stay exact."""
    n = SMALL_MAX + 12345
    keys = keys_for("u32", n, seed=6)
    d = to_device(keys, "u32")
    failures = overflows = 0
    for k in (17, 5000, n // 3, n - 5):
        p = tk.make_params(delta_factor=0.25, flags=tk.TOPK_FLAG_RAW_DELTA)
        out = tk.topk_select(ctx, d, k, params=p)
        check_against_oracle(keys, "u32", k, out, orc)
        failures += ctx.last_stats()["pivot_failures"]
    for k in (n // 2, n // 5):
        p = tk.make_params(flags=tk.TOPK_FLAG_TINY_CAND)
        out = tk.topk_select(ctx, d, k, params=p)
        check_against_oracle(keys, "u32", k, out, orc)
        overflows += ctx.last_stats()["overflows"]
    assert failures > 0 and overflows > 0


def test_forced_pivot_failures_at_the_limit(tk, ctx, orc):
    """A margin far too narrow (z = 0.25, used as given) misses rank k; the
    levels that follow must still find the exact set."""
    n = SMALL_MAX
    keys = keys_for("u32", n, seed=7)
    d = to_device(keys, "u32")
    failures = 0
    for k in (17, 900, 3000, n // 2):
        p = tk.make_params(delta_factor=0.25, flags=tk.TOPK_FLAG_RAW_DELTA)
        out = tk.topk_select(ctx, d, k, params=p)
        check_against_oracle(keys, "u32", k, out, orc)
        failures += ctx.last_stats()["pivot_failures"]
    assert failures > 0, "the narrow margin should have missed rank k at least once"


@pytest.mark.parametrize("name", ["f32", "u64"])
def test_largest_and_kth(tk, ctx, orc, name):
    n = 1 << 21
    k = 64
    keys = keys_for(name, n, seed=8)
    d = to_device(keys, name)
    p = tk.make_params(flags=tk.TOPK_FLAG_LARGEST)
    ok, oi, kk, ki = tk.topk_select(ctx, d, k, params=p)
    want_sel, want_kth = orc.select_largest(keys, name, k)
    got = bits_of(oi)
    assert np.array_equal(np.sort(got), np.sort(want_sel))
    assert np.array_equal(bits_of(ok), keys[got])
    assert int(bits_of(ki)[0]) == want_kth and int(bits_of(kk)[0]) == int(keys[want_kth])
    kk, ki = tk.topk_select_kth(ctx, d, k)
    _, want = orc.select(keys, name, k)
    assert int(bits_of(ki)[0]) == want and int(bits_of(kk)[0]) == int(keys[want])


def test_unaligned_and_ties(tk, ctx, orc):
    """An input that starts 4 bytes past a 16-byte boundary, and one of seven
    distinct values (ties split by position)."""
    n = (1 << 20) + 1
    keys = keys_for("f32", n, seed=9)
    d = to_device(keys, "f32")
    sub = d[1:]
    assert sub.data_ptr() % 16 == 4
    out = tk.topk_select(ctx, sub, 500)
    check_against_oracle(keys[1:].copy(), "f32", 500, out, orc)
    g = np.random.Generator(np.random.Philox(10))
    ties = (np.array([0.0, -0.0, 1.0, -1.0, 2.5, np.inf, -np.inf], np.float32)[g.integers(0, 7, size=n)]
            ).view(np.uint32)
    d = to_device(ties, "f32")
    for k in (2, 1000):
        out = tk.topk_select(ctx, d, k)
        check_against_oracle(ties, "f32", k, out, orc)

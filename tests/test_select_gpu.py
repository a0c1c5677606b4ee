"""topk_select on the GPU against the CPU oracle, element by element.

Sizes span the one-block path (n <= 16384), the in-block recursion
(16384 < n <= 65536) and the grid path with several levels, with ragged tails;
every key type; ties, IEEE specials, unaligned inputs, forced pivot failures
and forced candidate-buffer overflows.  Results must be bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1502_03942_gb300 import workloads as wl

from _gpu import bits_of, check_against_oracle, to_device

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


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def keys_for(name, n, seed, kind="uniform"):
    g = np.random.Generator(np.random.Philox(seed))
    if kind == "ties":
        vals = g.integers(0, 7, size=n)
        if name == "f32":
            return (np.array([0.0, -0.0, 1.0, -1.0, 2.5, np.inf, -np.inf], np.float32)[vals]).view(np.uint32)
        if name == "bf16":
            return np.array([0x0000, 0x8000, 0x3F80, 0xBF80, 0x4020, 0x7F80, 0xFF80], np.uint16)[vals]
        if name == "u64":
            return (vals.astype(np.uint64) * np.uint64(0x1234_5678_9ABC))
        return vals.astype(np.uint32) * np.uint32(0x2345_6789 // 7)
    if name in ("u32", "i32"):
        return wl.uniform_u32(n, seed)
    if name == "f32":
        return wl.normal_f32(n, seed).view(np.uint32)
    if name == "bf16":
        return g.integers(0, 1 << 16, size=n, dtype=np.uint32).astype(np.uint16)
    if name == "u64":
        return wl.uniform_u64(n, seed)
    raise ValueError(name)


def ks_for(n):
    ks = {1, 2, 3, n // 3 + 1, n // 2, n - 1, n}
    if n > 2000:
        ks |= {1000, 1024}
    return sorted(k for k in ks if 1 <= k <= n)


def test_config_plain_single_selection(tk, ctx, orc):
    """n = 2^20 uniform u32 keys from seed 1, k = 1000, p = 64 partitions."""
    n, k = 1 << 20, 1000
    keys = wl.uniform_u32(n, seed=1)
    d = to_device(keys, "u32")
    out = tk.topk_select(ctx, d, k, params=tk.make_params(partitions=64))
    check_against_oracle(keys, "u32", k, out, orc)


@pytest.mark.parametrize("name", ["u32", "i32", "f32", "bf16", "u64"])
@pytest.mark.parametrize("n", [1, 2, 7, 4095, 4096, 16385, 70001, 300007])
def test_sizes_and_ks(tk, ctx, orc, name, n):
    keys = keys_for(name, n, seed=n)
    d = to_device(keys, name)
    for k in ks_for(n):
        out = tk.topk_select(ctx, d, k)
        check_against_oracle(keys, name, k, out, orc)


@pytest.mark.parametrize("name", ["u32", "f32", "bf16", "u64"])
@pytest.mark.parametrize("n", [5000, 200003])
def test_heavy_ties_and_specials(tk, ctx, orc, name, n):
    keys = keys_for(name, n, seed=7, kind="ties")
    d = to_device(keys, name)
    for k in ks_for(n):
        out = tk.topk_select(ctx, d, k)
        check_against_oracle(keys, name, k, out, orc)


def test_nan_payloads_and_signed_zero(tk, ctx, orc):
    golden = np.array([0xFFFFFFFF, 0xFFC00001, 0xFF800001, 0xFF800000, 0x80000000, 0x00000000,
                       0x00000001, 0x7F800000, 0x7F800001, 0x7FFFFFFF], np.uint32)
    g = np.random.Generator(np.random.Philox(3))
    keys = golden[g.integers(0, golden.size, size=100_000)]
    d = to_device(keys, "f32")
    for k in (1, 5, 10_000, 50_000, 99_999, 100_000):
        out = tk.topk_select(ctx, d, k)
        check_against_oracle(keys, "f32", k, out, orc)


def test_zipf_heavy_ties(tk, ctx, orc):
    n = 1 << 21
    keys = wl.zipf_f32(n, seed=5).view(np.uint32)
    d = to_device(keys, "f32")
    for k in (1024, 1 << 17, n // 2):
        out = tk.topk_select(ctx, d, k)
        check_against_oracle(keys, "f32", k, out, orc)


@pytest.mark.parametrize("name", ["u32", "f32", "bf16", "u64"])
def test_unaligned_input(tk, ctx, orc, name):
    n = 100_003
    keys = keys_for(name, n + 1, seed=9)
    d = to_device(keys, name)[1:]          # one element off a 16-byte boundary
    for k in (1, 999, n // 2, n):
        out = tk.topk_select(ctx, d, k)
        check_against_oracle(keys[1:], name, k, out, orc)


@pytest.mark.parametrize("name", ["u32", "f32", "bf16", "u64"])
@pytest.mark.parametrize("order", ["ascending", "front", "descending"])
def test_clustered_hits(tk, ctx, orc, name, order):
    """Inputs whose selected elements sit together (sorted, or the smallest
    keys moved to the front): whole tiles are hits of the sparse pass, so its
    per-warp queues fill in one tile (for 64-bit keys beyond half a tile)."""
    n = 1 << 20
    keys = keys_for(name, n, seed=13)
    by_rank = orc.sort_order(keys, name)
    if order == "ascending":
        keys = keys[by_rank]
    elif order == "descending":
        keys = keys[by_rank[::-1]]
    else:
        small = np.zeros(n, bool)
        small[by_rank[:40000]] = True
        keys = np.concatenate([keys[small], keys[~small]])
    d = to_device(keys, name)
    for k in (1000, 5000, 30000):
        out = tk.topk_select(ctx, d, k)
        check_against_oracle(keys, name, k, out, orc)


def test_forced_pivot_failures_stay_exact(tk, ctx, orc):
    n = 1 << 20
    keys = wl.uniform_u32(n, seed=11)
    d = to_device(keys, "u32")
    failures = 0
    for k in (17, 5000, n // 3, n - 5):
        p = tk.make_params(delta_factor=0.25, flags=tk.TOPK_FLAG_RAW_DELTA)
        out = tk.topk_select(ctx, d, k, params=p)
        check_against_oracle(keys, "u32", k, out, orc)
        failures += ctx.last_stats()["pivot_failures"]
    assert failures > 0, "the narrow margin should have missed rank k at least once"


def test_forced_candidate_overflow_stays_exact(tk, ctx, orc):
    n = 1 << 20
    keys = wl.normal_f32(n, seed=12).view(np.uint32)
    d = to_device(keys, "f32")
    overflows = 0
    for k in (n // 2, n // 5):
        p = tk.make_params(flags=tk.TOPK_FLAG_TINY_CAND)
        out = tk.topk_select(ctx, d, k, params=p)
        check_against_oracle(keys, "f32", k, out, orc)
        overflows += ctx.last_stats()["overflows"]
    assert overflows > 0


def test_result_independent_of_tuning(tk, ctx, orc):
    """Partitions, seed, sample size and margin change the path, not the result."""
    n, k = 500_000, 12_345
    keys = wl.uniform_u32(n, seed=13)
    d = to_device(keys, "u32")
    for p in (tk.make_params(partitions=1), tk.make_params(partitions=64, seed=99),
              tk.make_params(sample_size=1024, delta_factor=2.0),
              tk.make_params(finish_threshold=512)):
        out = tk.topk_select(ctx, d, k, params=p)
        check_against_oracle(keys, "u32", k, out, orc)


def test_rejects_bad_arguments(tk, ctx):
    import torch
    d = torch.zeros(10, dtype=torch.float32, device="cuda")
    for k in (0, 11):
        with pytest.raises(tk.TopkError) as e:
            tk.topk_select(ctx, d, k)
        assert e.value.status == tk.TOPK_EINVAL


def test_philox_known_answers(tk):
    """Salmon et al. (SC'11) Philox4x32-10 known-answer vectors."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        vals = [int(x, 16) for x in line]
        ctr, key, want = vals[0:4], vals[4:6], vals[6:10]
        got = bits_of(tk.topk_debug_philox(ctr, key, 1))
        assert [int(x) for x in got] == want


# ---- the k largest (TOPK_FLAG_LARGEST) ----

def check_largest(keys_bits, name, k, out, orc):
    ok, oi, kk, ki = out
    got_idx = bits_of(oi)
    want_sel, want_kth = orc.select_largest(keys_bits, name, k)
    assert got_idx.size == k
    assert np.array_equal(np.sort(got_idx), np.sort(want_sel)), "selected set differs"
    assert np.array_equal(bits_of(ok), keys_bits[got_idx]), "output keys are not the input keys"
    assert int(bits_of(ki)[0]) == want_kth, "rank-k position differs"
    assert int(bits_of(kk)[0]) == int(keys_bits[want_kth]), "rank-k key differs"


@pytest.mark.parametrize("name", ["u32", "i32", "f32", "bf16", "u64"])
@pytest.mark.parametrize("n", [1, 7, 4096, 70001, 300007])
def test_largest_sizes_and_ks(tk, ctx, orc, name, n):
    keys = keys_for(name, n, seed=n + 11)
    d = to_device(keys, name)
    p = tk.make_params(flags=tk.TOPK_FLAG_LARGEST)
    for k in ks_for(n):
        check_largest(keys, name, k, tk.topk_select(ctx, d, k, params=p), orc)


@pytest.mark.parametrize("name", ["u32", "f32", "bf16", "u64"])
def test_largest_heavy_ties_and_specials(tk, ctx, orc, name):
    keys = keys_for(name, 200003, seed=13, kind="ties")
    d = to_device(keys, name)
    p = tk.make_params(flags=tk.TOPK_FLAG_LARGEST)
    for k in ks_for(200003):
        check_largest(keys, name, k, tk.topk_select(ctx, d, k, params=p), orc)

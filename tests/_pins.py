"""Checks that pin the CPU oracle to things other than itself.

Each check returns a list of failure strings (empty = pass), so the same
checks run both against the real oracle (tests/test_oracle_pins.py) and
against deliberately broken copies of it (tests/test_oracle_mutants.py), which
must fail at least one of them.

What pins the oracle (none of it re-types the oracle's comparator):
  * brute-force rank counting, rank_i = #{j : (v_j, j) < (v_i, i)}, with the
    value order taken from Python's own int / float comparison (paper,
    Section 2: unique order by (value, position));
  * exhaustive small inputs over 3-letter alphabets, which force ties;
  * special cases that are library routines: k = 1 is min(), k = n is a
    stable sort, integer selection is numpy's stable argsort, heapq.nsmallest;
  * IEEE 754 totalOrder on a hand-written fixture (tests/golden) and on all
    2^16 bf16 patterns, via a float-semantics order key;
  * multisequence selection against heapq.merge of the runs (Appendix A).
"""
from __future__ import annotations

import heapq
import itertools
import math
import os
import struct

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ------------------------------------------------------------- value orders

def f32_value_key(bits: int):
    """Sort key for a binary32 pattern under totalOrder, built on Python float
    semantics (not on bit tricks): NaNs by sign then payload, numbers by value,
    and -0 before +0."""
    bits &= 0xFFFFFFFF
    f = struct.unpack("<f", struct.pack("<I", bits))[0]
    neg = bits >> 31
    if math.isnan(f):
        payload = bits & 0x7FFFFF
        return (0, -payload, 0) if neg else (2, payload, 0)
    return (1, f, 0 if math.copysign(1.0, f) < 0 else 1)


def bf16_value_key(bits: int):
    return f32_value_key((bits & 0xFFFF) << 16)


def i32_value_key(bits: int):
    bits &= 0xFFFFFFFF
    return bits - (1 << 32) if bits >> 31 else bits


def uint_value_key(bits: int):
    return int(bits)


VALUE_KEY = {"u32": uint_value_key, "u64": uint_value_key, "i32": i32_value_key,
             "f32": f32_value_key, "bf16": bf16_value_key}
STORE = {"u32": np.uint32, "i32": np.uint32, "f32": np.uint32, "bf16": np.uint16,
         "u64": np.uint64}


def brute_force_ranks(keys, dtype):
    vk = VALUE_KEY[dtype]
    pairs = [(vk(int(x)), i) for i, x in enumerate(keys)]
    return [sum(1 for q in pairs if q < p) for p in pairs]


def expected_by_brute_force(keys, dtype, k):
    ranks = brute_force_ranks(keys, dtype)
    order = sorted(range(len(keys)), key=lambda i: ranks[i])
    return order[:k], order[k - 1]


# ------------------------------------------------------------------ checks

def random_bits(g, dtype, n):
    """n keys drawn from a small pool per type, so that ties, -0/+0, NaNs and
    the signed/unsigned difference all occur."""
    if dtype in ("f32", "bf16"):
        pool = [0x00000000, 0x80000000, 0x3F800000, 0xBF800000, 0x7F800000,
                0xFF800000, 0x7FC00000, 0xFFC00000, 0x00000001, 0x80000001]
        if dtype == "bf16":
            pool = [p >> 16 for p in pool] + [0x0001, 0x8001]
        return np.array(g.choice(pool, size=n), dtype=STORE[dtype])
    if dtype == "u64":
        pool = [0, 1, 1 << 32, (1 << 63) - 1, 1 << 63, (1 << 64) - 1]
        return np.array([pool[i] for i in g.integers(0, len(pool), size=n)], dtype=np.uint64)
    # the same pool for u32 and i32: the two orders differ on it
    pool = [0, 1, 2, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
    return np.array(g.choice(pool, size=n), dtype=np.uint32)


def check_brute_force(orc, seed=0, sizes=(1, 2, 3, 5, 8, 13, 31, 64)):
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for dtype in ("u32", "i32", "f32", "bf16", "u64"):
        for n in sizes:
            keys = random_bits(g, dtype, n)
            for k in range(1, n + 1):
                want_sel, want_kth = expected_by_brute_force(keys, dtype, k)
                sel, kth = orc.select(keys, dtype, k)
                if list(sel) != want_sel or kth != want_kth:
                    fails.append(f"brute force {dtype} n={n} k={k}")
                    break
    return fails


def check_exhaustive_ties(orc, max_n=7):
    alphabets = {
        "u32": [0, 1, 0xFFFFFFFF],
        "i32": [0xFFFFFFFF, 0, 1],            # -1, 0, 1: differs from unsigned order
        "f32": [0x80000000, 0x00000000, 0xFFC00000],  # -0, +0, -NaN
        "bf16": [0x8000, 0x0000, 0x7FC0],     # -0, +0, +NaN
    }
    fails = []
    for dtype, alpha in alphabets.items():
        for n in range(1, max_n + 1):
            for combo in itertools.product(alpha, repeat=n):
                keys = np.array(combo, dtype=STORE[dtype])
                perm = list(orc.sort_order(keys, dtype))
                ranks = brute_force_ranks(keys, dtype)
                want = sorted(range(n), key=lambda i: ranks[i])
                if perm != want:
                    fails.append(f"exhaustive {dtype} {combo}")
                    break
    return fails


def check_library_special_cases(orc, seed=1):
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for dtype in ("u32", "i32", "u64"):
        n = 5000
        if dtype == "u64":
            keys = g.integers(0, 1000, size=n, dtype=np.uint64) * np.uint64(1 << 50)
        else:
            keys = g.integers(0, 1000, size=n, dtype=np.uint64).astype(np.uint32) * np.uint32(4194301)
        vk = VALUE_KEY[dtype]
        as_int = [vk(int(x)) for x in keys]
        # k = 1: min over pairs
        sel, kth = orc.select(keys, dtype, 1)
        mn = min(zip(as_int, range(n)))
        if kth != mn[1] or list(sel) != [mn[1]]:
            fails.append(f"k=1 vs min {dtype}")
        # k = n: Python's stable sort by value
        stable = sorted(range(n), key=lambda i: as_int[i])
        sel, kth = orc.select(keys, dtype, n)
        if list(sel) != stable or kth != stable[-1]:
            fails.append(f"k=n vs stable sort {dtype}")
        # numpy stable argsort on the signed/unsigned values
        typed = keys.view(np.int32) if dtype == "i32" else keys
        ref = np.argsort(typed, kind="stable")
        for k in (1, 7, 100, 2500, n):
            sel, kth = orc.select(keys, dtype, k)
            if not np.array_equal(sel, ref[:k]) or kth != ref[k - 1]:
                fails.append(f"numpy stable argsort {dtype} k={k}")
        # heapq.nsmallest on (value, position)
        for k in (3, 50):
            want = [i for _, i in heapq.nsmallest(k, zip(as_int, range(n)))]
            sel, _ = orc.select(keys, dtype, k)
            if list(sel) != want:
                fails.append(f"heapq.nsmallest {dtype} k={k}")
    # float without NaN and without -0: numpy's stable argsort is totalOrder
    x = g.standard_normal(4000).astype(np.float32)
    x[::7] = x[3]                          # ties
    x[x == 0] = 1.0
    ref = np.argsort(x, kind="stable")
    for k in (1, 10, 2000, 4000):
        sel, kth = orc.select(x.view(np.uint32), "f32", k)
        if not np.array_equal(sel, ref[:k]) or kth != ref[k - 1]:
            fails.append(f"numpy stable argsort f32 k={k}")
    return fails


def load_golden_f32_order():
    out = []
    with open(os.path.join(GOLDEN, "f32_total_order.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append(int(line, 16))
    return out


def check_total_order_fixture(orc, seed=2):
    fails = []
    golden = load_golden_f32_order()
    g = np.random.Generator(np.random.Philox(seed))
    for trial in range(5):
        shuffled = np.array(golden, dtype=np.uint32)[g.permutation(len(golden))]
        perm = orc.sort_order(shuffled, "f32")
        if [int(v) for v in shuffled[perm]] != golden:
            fails.append("f32 totalOrder fixture")
            break
    # the fixture also agrees with the float-semantics key (self-consistency)
    if sorted(golden, key=f32_value_key) != golden:
        fails.append("fixture vs float key")
    return fails


def check_bf16_exhaustive(orc):
    allbits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    perm = orc.sort_order(allbits, "bf16")
    want = sorted(range(1 << 16), key=lambda b: (bf16_value_key(b), b))
    return [] if list(perm) == want else ["bf16 exhaustive totalOrder"]


def merged_runs_reference(keys, off, k):
    runs = []
    for r in range(len(off) - 1):
        a, b = int(off[r]), int(off[r + 1])
        runs.append([(int(keys[a + j]), r, j) for j in range(b - a)])
    merged = list(itertools.islice(heapq.merge(*runs), k))
    split = [0] * (len(off) - 1)
    for _, r, _j in merged:
        split[r] += 1
    return split, merged[-1][1], merged[-1][2]


def check_runs_vs_merge(orc, seed=3):
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for trial in range(40):
        p = int(g.integers(1, 9))
        lens = g.integers(0, 12, size=p)
        if lens.sum() == 0:
            lens[0] = 1
        off = np.zeros(p + 1, np.uint64)
        off[1:] = np.cumsum(lens)
        keys = (g.integers(0, 5, size=int(off[-1])) * 3).astype(np.uint64)
        for r in range(p):
            keys[int(off[r]):int(off[r + 1])].sort()
        total = int(off[-1])
        for k in range(1, total + 1):
            split, kr, kp = orc.select_runs(keys, off, k)
            ws, wr, wp = merged_runs_reference(keys, off, k)
            if list(split) != ws or (kr, kp) != (wr, wp):
                fails.append(f"runs vs heapq.merge trial={trial} k={k}")
                return fails
    return fails


def check_delete_min_vs_heap(orc, seed=5):
    """Bulk deleteMin* (Section 5) against a textbook binary-heap priority
    queue (heapq): the queue holds (key, run, position) of every object at or
    after its run's cursor; k pops give the deleted objects.  Sequences of
    bulk deletions from random cursors down to an empty queue."""
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for trial in range(30):
        p = int(g.integers(1, 7))
        lens = g.integers(0, 10, size=p)
        if lens.sum() == 0:
            lens[0] = 1
        off = np.zeros(p + 1, np.uint64)
        off[1:] = np.cumsum(lens)
        keys = (g.integers(0, 4, size=int(off[-1])) * 5).astype(np.uint64)
        for r in range(p):
            keys[int(off[r]):int(off[r + 1])].sort()
        cursor = np.array([int(g.integers(0, l + 1)) for l in lens], np.uint64)
        heap = []
        for r in range(p):
            for j in range(int(cursor[r]), int(lens[r])):
                heapq.heappush(heap, (int(keys[int(off[r]) + j]), r, j))
        while heap:
            k = int(g.integers(1, len(heap) + 1))
            popped = [heapq.heappop(heap) for _ in range(k)]
            want = cursor.copy()
            for _, r, _j in popped:
                want[r] += 1
            cursor, kr, kp = orc.runs_delete_min(keys, off, cursor, k)
            if list(cursor) != list(want) or (kr, kp) != popped[-1][1:]:
                fails.append(f"deleteMin* vs heapq trial={trial} k={k}")
                return fails
    return fails


def check_largest_brute_force(orc, seed=8):
    """The k largest against brute force (values descending by Python's own
    int/float order, equal values by ascending position) for every key type,
    and against the k smallest of the complemented u32 / u64 keys."""
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for dtype in ("u32", "i32", "f32", "bf16", "u64"):
        vk = VALUE_KEY[dtype]
        for n in (1, 2, 5, 13, 40):
            bits = random_bits(g, dtype, n)
            order = sorted(range(n), key=lambda i: (_neg(vk(int(bits[i]))), i))
            for k in sorted({1, n // 2 + 1, n}):
                sel, kth = orc.select_largest(bits, dtype, k)
                if list(sel) != order[:k] or kth != order[k - 1]:
                    fails.append(f"largest {dtype} n={n} k={k}")
    for dtype, top in (("u32", 0xFFFFFFFF), ("u64", 0xFFFFFFFFFFFFFFFF)):
        store = np.uint32 if dtype == "u32" else np.uint64
        bits = g.integers(0, 8, size=500).astype(store)
        comp = (np.array(top, dtype=store) - bits).astype(store)
        for k in (1, 100, 500):
            sel, kth = orc.select_largest(bits, dtype, k)
            want, wkth = orc.select(comp, dtype, k)
            if list(sel) != list(want) or kth != wkth:
                fails.append(f"largest vs complemented smallest {dtype} k={k}")
    return fails


def _neg(v):
    """Reverses a value key's order (a float or int, or a NaN's tuple key)."""
    if isinstance(v, tuple):
        return tuple(-x if isinstance(x, (int, float)) else x for x in v)
    return -v


# ---- top-k most frequent objects (Section 7) ----

def load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def check_philox_kat(orc):
    """The oracle's Philox4x32-10 against the published known-answer vectors."""
    return [f"philox KAT {i}" for i, (c, k, want) in enumerate(load_kat())
            if list(orc.philox(c, k)) != want]


def load_pac_example():
    ex = {"pes": []}
    with open(os.path.join(GOLDEN, "pac_worked_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            if key.startswith("pe "):
                ex["pes"].append("".join(val.split()))
            elif key in ("rho",):
                ex[key] = float(val)
            elif key in ("k", "kstar"):
                ex[key] = int(val)
            else:
                w = val.split()
                ex[key] = [(w[i], int(w[i + 1])) for i in range(0, len(w), 2)]
    return ex


def check_pac_worked_example(orc):
    """The paper's worked example: PAC's estimates (sample count / rho,
    rounded), EC's candidates with their exact counts and EC's result."""
    fails = []
    ex = load_pac_example()
    text = "".join(ex["pes"])
    objects = np.array([ord(ch.upper()) for ch in text], np.uint32)
    mask = np.array([1 if ch.islower() else 0 for ch in text], np.uint8)
    name = lambda o: chr(int(o))
    # sample counts of every sampled object (k = all distinct sampled)
    d = len(ex["sample_counts"])
    o, c, m = orc.frequent(objects, mask, d)
    if sorted(zip(map(name, o), map(int, c))) != sorted(ex["sample_counts"]) or m != int(mask.sum()):
        fails.append("worked example: sample counts")
    o, c, _ = orc.frequent(objects, mask, ex["k"])
    est = [(name(a), int(round(int(b) / ex["rho"]))) for a, b in zip(o, c)]
    if sorted(est) != sorted(ex["pac_estimated"]):
        fails.append(f"worked example: PAC estimates {est}")
    o, c, _ = orc.frequent(objects, mask, ex["kstar"], kstar=ex["kstar"], exact=True)
    if sorted(zip(map(name, o), map(int, c))) != sorted(ex["ec_candidates"]):
        fails.append("worked example: EC candidates")
    o, c, _ = orc.frequent(objects, mask, ex["k"], kstar=ex["kstar"], exact=True)
    got = list(zip(map(name, o), map(int, c)))
    if got != ex["ec_result"] or sorted(got) != sorted(ex["exact"]):
        fails.append(f"worked example: EC result {got}")
    return fails


def check_frequent_vs_counter(orc, seed=6):
    """PAC and EC against collections.Counter over the sampled (PAC) or all
    (EC) objects, most frequent first, equal counts by the smaller object."""
    import collections
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for trial in range(25):
        n = int(g.integers(1, 3000))
        objects = ((g.integers(0, int(g.integers(1, 60)), size=n).astype(np.uint64) * 2654435761)
                   % (1 << 32)).astype(np.uint32)
        mask = (g.random(n) < g.uniform(0.05, 1.0)).astype(np.uint8)
        sampled = collections.Counter(int(x) for x, s in zip(objects, mask) if s)
        ranked = sorted(sampled.items(), key=lambda t: (-t[1], t[0]))
        if not ranked:
            continue
        k = int(g.integers(1, len(ranked) + 1))
        o, c, _ = orc.frequent(objects, mask, k)
        if list(zip(map(int, o), map(int, c))) != ranked[:k]:
            fails.append(f"PAC vs Counter trial={trial}")
            return fails
        kstar = int(g.integers(k, len(ranked) + 1))
        full = collections.Counter(int(x) for x in objects)
        cand = sorted(((x, full[x]) for x, _ in ranked[:kstar]), key=lambda t: (-t[1], t[0]))
        o, c, _ = orc.frequent(objects, mask, k, kstar=kstar, exact=True)
        if list(zip(map(int, o), map(int, c))) != cand[:k]:
            fails.append(f"EC vs Counter trial={trial}")
            return fails
    return fails


def check_bernoulli_decisions(orc, seed=7):
    """Element i is sampled iff word i % 4 of Philox at counter (i / 4, 0,
    stream, 0) is below the threshold; the sampled fraction is within six
    standard deviations of rho; rho = 1 samples everything, 0 nothing."""
    fails = []
    n = 1 << 16
    for rho in (0.074, 0.5):
        thr = orc.sample_threshold(rho)
        if thr != int(rho * 2 ** 32):
            fails.append(f"threshold {rho}")
        mask = orc.bernoulli_sample(n, 0x1234_5678_9ABC_DEF0, thr)
        frac = mask.mean()
        if abs(frac - rho) > 6 * (rho * (1 - rho) / n) ** 0.5:
            fails.append(f"sampled fraction {frac} for rho {rho}")
        for i in (0, 1, 2, 3, 4, 7, 12345, n - 1):
            j = i // 4
            w = orc.philox([j & 0xFFFFFFFF, j >> 32, 0x53414D50, 0], [0x9ABCDEF0, 0x12345678])[i % 4]
            if int(mask[i]) != int(int(w) < thr):
                fails.append(f"decision of element {i}")
    if orc.bernoulli_sample(1000, 5, orc.sample_threshold(1.0)).min() != 1:
        fails.append("rho = 1")
    if orc.bernoulli_sample(1000, 5, orc.sample_threshold(0.0)).max() != 0:
        fails.append("rho = 0")
    return fails


def check_frequent_plan(orc):
    """Sample sizes against the closed forms the paper states: PAC's
    8 ln(2k/delta) / eps^2 where the second term of equation sampleSize
    dominates, EC's 2 ln(n/delta) / (eps^2 k) with k* = k on one PE; rho
    is clamped to 1."""
    import math
    fails = []
    n, k, eps, delta = 1 << 40, 32, 3e-4, 1e-4
    rho, ks = orc.frequent_plan(n, k, eps, delta)
    if ks != k or abs(rho * n / (8 / eps ** 2 * math.log(2 * k / delta)) - 1) > 1e-12:
        fails.append("PAC closed form")
    rho, ks = orc.frequent_plan(1 << 28, k, eps, delta, exact=True)
    if ks != k or abs(rho * (1 << 28) / (2 / (eps ** 2 * k) * math.log((1 << 28) / delta)) - 1) > 1e-12:
        fails.append("EC closed form")
    if orc.frequent_plan(1 << 28, k, eps, delta)[0] != 1.0:
        fails.append("PAC rho clamp")
    rho_big_p, ks_big_p = orc.frequent_plan(1 << 40, k, 1e-6, 1e-8, pes=1024, exact=True)
    if not ks_big_p > k:
        fails.append("EC k* grows with p")
    # hand-evaluated closed forms (tests/golden/frequent_plan_values.txt):
    # EC with p > 1 (so k* > k) and PAC where the first term of equation
    # sampleSize is the larger one
    for alg, n, kk, e, d, p, want_ks, want_rn in load_plan_values():
        rho, ks = orc.frequent_plan(n, kk, e, d, pes=p, exact=(alg == "EC"))
        if ks != want_ks or abs(rho * n / want_rn - 1) > 1e-12:
            fails.append(f"{alg} plan n={n} k={kk} p={p}: k*={ks} rho*n={rho * n}")
    return fails


def load_plan_values():
    rows = []
    for line in open(os.path.join(GOLDEN, "frequent_plan_values.txt")):
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        alg, n, k, eps, delta, p, ks, rn = line
        rows.append((alg, int(n), int(k), float(eps), float(delta), int(p), int(ks), float(rn)))
    return rows


def check_batched_rows(orc, seed=4):
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    lens = g.integers(1, 40, size=9)
    off = np.zeros(10, np.uint64)
    off[1:] = np.cumsum(lens)
    keys = g.integers(0, 6, size=int(off[-1])).astype(np.uint32)
    ks = np.array([int(g.integers(1, l + 1)) for l in lens], np.uint32)
    sel, out_off, kth = orc.select_batched(keys, off, ks, "u32")
    for i in range(9):
        row = keys[int(off[i]):int(off[i + 1])]
        want_sel, want_kth = expected_by_brute_force(row, "u32", int(ks[i]))
        got = list(sel[int(out_off[i]):int(out_off[i + 1])])
        if got != want_sel or kth[i] != want_kth:
            fails.append(f"batched row {i}")
    return fails


def check_pairs_before(orc, seed=9):
    """The one-pass rank count against brute force with Python's own value
    order, both directions, on inputs full of ties: the pair of rank r has
    r - 1 pairs before it (Section 2 order on (value, position))."""
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for dtype in ("u32", "i32", "f32", "bf16", "u64"):
        for n in (1, 2, 9, 40):
            keys = random_bits(g, dtype, n)
            vk = VALUE_KEY[dtype]
            for pos in range(n):
                asc = sum(1 for j in range(n)
                          if (vk(int(keys[j])), j) < (vk(int(keys[pos])), pos))
                desc = sum(1 for j in range(n)
                           if (_neg(vk(int(keys[j]))), j) < (_neg(vk(int(keys[pos]))), pos))
                if orc.pairs_before(keys, dtype, pos) != asc:
                    fails.append(f"pairs_before {dtype} n={n} pos={pos}")
                    break
                if orc.pairs_before(keys, dtype, pos, descending=True) != desc:
                    fails.append(f"pairs_before descending {dtype} n={n} pos={pos}")
                    break
    return fails


def check_selection_checker(orc, seed=10):
    """The sort-free checker accepts the brute-force answer (Python's own
    value order) in both directions and rejects answers with one planted
    error each: an unselected position swapped in, a repeated position, the
    rank-k position moved by one, an output key not the input key."""
    fails = []
    g = np.random.Generator(np.random.Philox(seed))
    for dtype in ("u32", "i32", "f32", "bf16", "u64"):
        for n in (2, 9, 40):
            keys = random_bits(g, dtype, n)
            vk = VALUE_KEY[dtype]
            for desc in (False, True):
                f = (lambda v: _neg(v)) if desc else (lambda v: v)
                order = sorted(range(n), key=lambda i: (f(vk(int(keys[i]))), i))
                for k in (1, n // 2, n - 1):
                    if k < 1:
                        continue
                    sel = np.array(order[:k], np.uint32)
                    kth = order[k - 1]
                    good = orc.check_selection(keys, dtype, k, sel, kth, keys[sel], keys[kth:kth + 1],
                                               descending=desc)
                    if good != 0:
                        fails.append(f"checker rejects the answer {dtype} n={n} k={k} desc={desc}: {good}")
                        continue
                    bad = sel.copy()
                    if k >= 2:
                        bad[0] = order[k]  # an unselected pair in place of a selected one
                        if orc.check_selection(keys, dtype, k, bad, kth, descending=desc) == 0:
                            fails.append(f"checker takes a swapped-in position {dtype} n={n} k={k}")
                        bad = sel.copy()
                        bad[1] = bad[0]
                        if orc.check_selection(keys, dtype, k, bad, kth, descending=desc) != 2:
                            fails.append(f"checker takes a repeated position {dtype} n={n} k={k}")
                    if orc.check_selection(keys, dtype, k, sel, order[k], descending=desc) != 1:
                        fails.append(f"checker takes the rank-(k+1) pair as rank k {dtype} n={n} k={k}")
                    wrong = keys[sel].copy()
                    wrong[-1] ^= 1
                    if orc.check_selection(keys, dtype, k, sel, kth, wrong, descending=desc) != 4:
                        fails.append(f"checker takes a wrong output key {dtype} n={n} k={k}")
    return fails


ALL_CHECKS = [check_brute_force, check_exhaustive_ties, check_library_special_cases,
              check_total_order_fixture, check_bf16_exhaustive, check_runs_vs_merge,
              check_batched_rows, check_delete_min_vs_heap, check_philox_kat,
              check_pac_worked_example, check_frequent_vs_counter, check_bernoulli_decisions,
              check_frequent_plan, check_largest_brute_force, check_pairs_before,
              check_selection_checker]

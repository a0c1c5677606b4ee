"""topk_frequent on the GPU against the CPU oracle (bit-exact).

Top-k most frequent objects (Section 7): Algorithm PAC (the k most
frequently sampled objects with their sample counts) and Algorithm EC (the k
most frequent of the k* most frequently sampled, with exact counts).  Both
sides draw the same Bernoulli sample: Philox4x32-10 decisions defined
element by element, implemented separately in the oracle and the kernels.
The result is unique (count, then the smaller object), so the comparison is
exact: the same objects, the same counts, the same sample size.
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


def ranked(o, c):
    return sorted(zip(map(int, o), map(int, c)), key=lambda t: (-t[1], t[0]))


def run_and_check(tk, ctx, objects, k, rho, exact, kstar=0, seed=0x5EED, d_obj=None):
    fp = tk.make_freq_params(k, algorithm=tk.TOPK_FREQ_EC if exact else tk.TOPK_FREQ_PAC, rho=rho,
                             kstar=kstar if exact else 0, seed=seed)
    if d_obj is None:
        d_obj = to_device(objects, "u32")
    oo, oc, ss = tk.topk_frequent(ctx, d_obj, fp)
    mask = oracle.bernoulli_sample(objects.size, seed, oracle.sample_threshold(rho))
    wo, wc, wss = oracle.frequent(objects, mask, k, kstar=kstar if exact else 0, exact=exact)
    assert int(bits_of(ss)[0]) == wss, "sample size differs"
    assert ranked(bits_of(oo), bits_of(oc)) == ranked(wo, wc), "objects or counts differ"


def distinct_sampled(objects, rho, seed):
    mask = oracle.bernoulli_sample(objects.size, seed, oracle.sample_threshold(rho))
    return np.unique(objects[mask.astype(bool)]).size


@pytest.mark.parametrize("n", [1, 7, 1000, 65539, 1 << 20])
@pytest.mark.parametrize("kind", ["zipf", "negbin", "few"])
def test_pac_and_ec_small(tk, ctx, n, kind):
    if kind == "zipf":
        obj = wl.zipf_objects(n, seed=n)
    elif kind == "negbin":
        obj = wl.negbin_objects(n, seed=n + 1)
    else:
        # five objects including the largest (its table word differs from an
        # empty slot only in the count half)
        alphabet = np.array([0xFFFFFFFF, 0xFFFFFFFE, 0, 1, 12345], np.uint32)
        obj = alphabet[wl.rng(n + 2).integers(0, 5, size=n)]
    for rho in (1.0, 0.3, 0.074):
        d = distinct_sampled(obj, rho, seed=0x5EED)
        if d == 0:
            continue
        for k in sorted({1, min(d, 5), min(d, 32), d}):
            run_and_check(tk, ctx, obj, k, rho, exact=False)
            kstar = min(d, 2 * k, 4096)  # the recount takes k* <= 4096
            if k <= kstar:
                run_and_check(tk, ctx, obj, k, rho, exact=True, kstar=kstar)
        if d >= 4096:
            run_and_check(tk, ctx, obj, 100, rho, exact=True, kstar=4096)


def test_seeds_and_unaligned_input(tk, ctx):
    """Other seeds draw other samples (same on both sides); an input that is
    not 16-byte aligned takes the scalar load path."""
    import torch
    obj = wl.zipf_objects((1 << 18) + 5, seed=44)
    buf = torch.zeros(obj.size + 1, dtype=torch.int32, device="cuda").view(torch.uint32)
    buf[1:] = to_device(obj, "u32")
    for seed in (1, 2, 0xFFFFFFFFFFFFFFFF):
        run_and_check(tk, ctx, obj, 32, 0.05, exact=False, seed=seed)
        run_and_check(tk, ctx, obj, 32, 0.05, exact=True, kstar=64, seed=seed, d_obj=buf[1:])


def test_planned_rate(tk, ctx):
    """rho and k* from eps and delta: the library's plan is the oracle's, and
    the run with it matches the oracle run with that rho."""
    obj = wl.zipf_objects(1 << 20, seed=45)
    for alg, eps, delta in ((tk.TOPK_FREQ_EC, 3e-3, 1e-4), (tk.TOPK_FREQ_PAC, 1e-2, 1e-3)):
        fp = tk.make_freq_params(8, algorithm=alg, epsilon=eps, delta=delta, seed=9)
        rho, kstar = tk.topk_frequent_plan(obj.size, fp)
        want_rho, want_kstar = oracle.frequent_plan(obj.size, 8, eps, delta, exact=alg == tk.TOPK_FREQ_EC)
        assert kstar == want_kstar and rho == pytest.approx(want_rho, rel=1e-14)
        oo, oc, ss = tk.topk_frequent(ctx, to_device(obj, "u32"), fp)
        mask = oracle.bernoulli_sample(obj.size, 9, oracle.sample_threshold(rho))
        wo, wc, wss = oracle.frequent(obj, mask, 8, kstar=kstar, exact=alg == tk.TOPK_FREQ_EC)
        assert int(bits_of(ss)[0]) == wss
        assert ranked(bits_of(oo), bits_of(oc)) == ranked(wo, wc)


def test_errors(tk, ctx):
    obj = (np.arange(1000, dtype=np.uint32) % 10).astype(np.uint32)
    d_obj = to_device(obj, "u32")
    # more objects asked for than were sampled (10 distinct)
    for exact, k, kstar in ((False, 11, 0), (True, 5, 11)):
        fp = tk.make_freq_params(k, algorithm=tk.TOPK_FREQ_EC if exact else tk.TOPK_FREQ_PAC, rho=1.0,
                                 kstar=kstar)
        with pytest.raises(tk.TopkError) as e:
            tk.topk_frequent(ctx, d_obj, fp)
        assert e.value.status == tk.TOPK_EINVAL
    # argument errors: k* < k, k* above the recount's limit, rho > 1
    for fp in (tk.make_freq_params(5, rho=1.0, kstar=4), tk.make_freq_params(5, rho=1.0, kstar=5000),
               tk.make_freq_params(5, algorithm=tk.TOPK_FREQ_PAC, rho=1.5)):
        with pytest.raises(tk.TopkError) as e:
            tk.topk_frequent(ctx, d_obj, fp)
        assert e.value.status == tk.TOPK_EINVAL
    # a table too small for the distinct sampled objects
    many = to_device(np.arange(1 << 14, dtype=np.uint32), "u32")
    fp = tk.make_freq_params(4, algorithm=tk.TOPK_FREQ_PAC, rho=1.0, max_distinct=1000)
    with pytest.raises(tk.TopkError) as e:
        tk.topk_frequent(ctx, many, fp)
    assert e.value.status == tk.TOPK_ENOMEM
    # the context stays usable
    run_and_check(tk, ctx, obj, 3, 1.0, exact=False)


def test_paper_configuration_2e26(tk, ctx):
    """n = 2^26 Zipf objects (s = 1, 2^20 values), k = 32, eps = 3e-4,
    delta = 1e-4 (Section 10.2): EC with its planned rate and PAC with a
    sampled rate, against the oracle."""
    n = 1 << 26
    obj = wl.zipf_objects(n, seed=46)
    fp = tk.make_freq_params(32, algorithm=tk.TOPK_FREQ_EC, epsilon=3e-4, delta=1e-4, seed=11)
    rho, kstar = tk.topk_frequent_plan(n, fp)
    assert kstar == 32 and 0 < rho < 1
    run_and_check(tk, ctx, obj, 32, rho, exact=True, kstar=32, seed=11)
    run_and_check(tk, ctx, obj, 32, 0.02, exact=False, seed=12)


def test_full_size_exact_counting(tk, ctx):
    """n = 2^28 Zipf objects drawn on the device, PAC with rho = 1 (what
    equation sampleSize gives on one GPU for eps = 3e-4): the counts
    returned are the objects' exact counts and no other object is more
    frequent (torch.unique as the checker); EC's exact counts likewise."""
    import torch
    n = 1 << 28
    d_obj = wl.device_zipf_objects(n, seed=47)
    fp = tk.make_freq_params(32, algorithm=tk.TOPK_FREQ_PAC, epsilon=3e-4, delta=1e-4, seed=13)
    rho, _ = tk.topk_frequent_plan(n, fp)
    assert rho == 1.0
    oo, oc, ss = tk.topk_frequent(ctx, d_obj, fp)
    assert int(bits_of(ss)[0]) == n
    got = ranked(bits_of(oo), bits_of(oc))
    vals, counts = torch.unique(d_obj.view(torch.int32), return_counts=True)
    vals = vals.cpu().numpy().view(np.uint32)
    counts = counts.cpu().numpy()
    order = sorted(range(vals.size), key=lambda i: (-int(counts[i]), int(vals[i])))[:32]
    assert got == [(int(vals[i]), int(counts[i])) for i in order]
    fp = tk.make_freq_params(32, algorithm=tk.TOPK_FREQ_EC, epsilon=3e-4, delta=1e-4, seed=13)
    oo, oc, ss = tk.topk_frequent(ctx, d_obj, fp)
    lookup = dict(zip(map(int, vals), map(int, counts)))
    for o, c in zip(bits_of(oo), bits_of(oc)):
        assert lookup[int(o)] == int(c)

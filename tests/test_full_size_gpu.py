"""topk_select at the benchmark's full size, checked against the oracle.

n = 2^28 float32 keys, the three datasets the benchmark times (U(0,1),
N(0,1), Zipf s = 1.2 over 10^4 values, drawn on the device exactly as the
benchmark draws them), k in {1, 1024, 2^20, n/2}, p = 148 partitions, the
same launch configuration the benchmark times.  A full sort of 2^28 pairs
takes minutes on the host, so each answer goes through the oracle's
sort-free checker (``oracle.check_selection``), which holds it to the
definition of the k smallest pairs (Section 2 order on (value, position);
Section 4 problem statement):

  * the rank-k pair has exactly k - 1 pairs before it (one pass over n);
  * the k positions are distinct (bitmap);
  * no selected pair comes after the rank-k pair;
  * every output key has the bits of the input key at its position.

k distinct pairs, none after the one with k - 1 pairs before it, can only be
the k smallest, so this is the exact answer, element for element.  On the
Zipf data, k = 1024 and 2^20 fall inside the run of the smallest value
(about 21% of n equal keys) and k = n/2 inside another run, so the position
tie-break decides every one of them.  The same holds for the k largest.
"""
import numpy as np
import pytest

import oracle
from paper_1502_03942_gb300 import workloads as wl

from _gpu import bits_of

pytestmark = pytest.mark.gpu

N = 1 << 28
KS = (1, 1024, 1 << 20, N // 2)


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


def _check(orc, host_bits, k, out, descending=False):
    ok, oi, kk, ki = out
    code = orc.check_selection(host_bits, "f32", k, bits_of(oi), int(bits_of(ki)[0]),
                               out_keys=bits_of(ok), kth_key=bits_of(kk), descending=descending)
    assert code == 0, {1: "the rank-k pair has the wrong rank", 2: "a position repeats",
                       3: "a selected pair lies beyond the rank-k pair",
                       4: "an output key is not the input key"}.get(code, code)


@pytest.mark.parametrize("ds", ["uniform", "normal", "zipf"])
def test_headline_selection_full_size(tk, ctx, orc, ds):
    import torch
    d = wl.device_f32_dataset(ds, N, seed=2)  # the benchmark's rank-0 inputs
    host_bits = d.view(torch.int32).cpu().numpy().view(np.uint32)
    params = tk.make_params(partitions=148)
    for k in KS:
        out = tk.topk_select(ctx, d, k, params=params)
        _check(orc, host_bits, k, out)
        del out
    del d
    torch.cuda.empty_cache()


def test_largest_full_size(tk, ctx, orc):
    """The 1024 and the n/2 largest of 2^28 N(0,1) keys, and of the Zipf keys
    (heavy ties: equal keys taken by the smaller position)."""
    import torch
    p = tk.make_params(partitions=148, flags=tk.TOPK_FLAG_LARGEST)
    for ds, seed in (("normal", 31), ("zipf", 32)):
        d = wl.device_f32_dataset(ds, N, seed=seed)
        host_bits = d.view(torch.int32).cpu().numpy().view(np.uint32)
        for k in (1024, N // 2):
            out = tk.topk_select(ctx, d, k, params=p)
            _check(orc, host_bits, k, out, descending=True)
            del out
        del d
        torch.cuda.empty_cache()

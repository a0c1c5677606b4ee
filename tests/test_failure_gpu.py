"""Failure detection on the GPU without a fault: a bounded device wait that
nothing completes expires, the context latches TOPK_ETIMEOUT, the host reads
it, and the same context then runs a selection correctly."""
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


def test_wait_expires_and_context_recovers(tk):
    import time
    ctx = tk.Context(0)
    t0 = time.perf_counter()
    tk.topk_debug_wait_timeout(ctx, 2000)  # 2 ms
    assert ctx.sync() == tk.TOPK_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert ctx.sync() == tk.TOPK_OK  # reported once, then cleared
    bits = wl.uniform_u32(100000, 71)
    ok, oi, kk, ki = tk.topk_select(ctx, to_device(bits, "u32"), 777)
    want_sel, want_kth = oracle.select(bits, "u32", 777)
    assert np.array_equal(np.sort(bits_of(oi)), np.sort(want_sel))
    assert int(bits_of(ki)[0]) == want_kth
    ctx.close()


def test_wait_limit_checked(tk):
    ctx = tk.Context(0)
    for bad in (0, 2_000_000):
        with pytest.raises(tk.TopkError) as e:
            tk.topk_debug_wait_timeout(ctx, bad)
        assert e.value.status == tk.TOPK_EINVAL
    ctx.close()

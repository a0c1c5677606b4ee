"""topk_select_kth (the rank-k key alone) and the entry points that refuse
the largest-k flag, against the CPU oracle."""
import pytest

import oracle

from _gpu import bits_of, to_device
from test_select_gpu import keys_for

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


@pytest.mark.parametrize("name", ["u32", "f32", "bf16", "u64"])
def test_kth_only(tk, ctx, orc, name):
    """topk_select_kth: the rank-k key and position of the k smallest and of
    the k largest, as the oracle's."""
    n = 100003
    keys = keys_for(name, n, seed=17, kind="ties" if name != "u64" else "uniform")
    d = to_device(keys, name)
    for k in (1, 1000, n // 2, n):
        kk, ki = tk.topk_select_kth(ctx, d, k)
        _, want = orc.select(keys, name, k)
        assert int(bits_of(ki)[0]) == want and int(bits_of(kk)[0]) == int(keys[want])
        kk, ki = tk.topk_select_kth(ctx, d, k, params=tk.make_params(flags=tk.TOPK_FLAG_LARGEST))
        _, want = orc.select_largest(keys, name, k)
        assert int(bits_of(ki)[0]) == want and int(bits_of(kk)[0]) == int(keys[want])


def test_largest_flag_refused_where_unsupported(tk, ctx):
    """Batched selection, its tuner and the sorted-runs calls select the k
    smallest only; they refuse the largest-k flag instead of ignoring it."""
    import torch
    p = tk.make_params(flags=tk.TOPK_FLAG_LARGEST)
    keys = torch.randn(1000, device="cuda")
    row_off = torch.tensor([0, 500, 1000], dtype=torch.int64, device="cuda").view(torch.uint64)
    row_k = torch.tensor([3, 4], dtype=torch.int32, device="cuda").view(torch.uint32)
    with pytest.raises(tk.TopkError) as e:
        tk.topk_select_batched(ctx, keys, row_off, row_k, params=p)
    assert e.value.status == tk.TOPK_EINVAL
    runs = torch.arange(1000, dtype=torch.int64, device="cuda").view(torch.uint64)
    with pytest.raises(tk.TopkError) as e:
        tk.topk_select_sorted_runs(ctx, runs, row_off, 10, params=p)
    assert e.value.status == tk.TOPK_EINVAL

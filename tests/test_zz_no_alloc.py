"""The allocation-free selection entry point against topk_select (GPU).

topk_select_noalloc serves callers that cannot allocate device memory when
they call (for instance while a CUDA graph is being captured, or from inside
another allocator's callbacks): its scratch is a fixed device array.  This
test calls it through the C ABI, twice in a row on different inputs, and
requires bit-identical results to the context-based entry point.  The file
name sorts last so that a run stopping at the first failure has run every
other test first; it also runs alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1502_03942_gb300 import workloads as wl

from _gpu import bits_of, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03942_gb300 as tk
    return tk, tk.load_library()


def _outputs(torch, keys, k):
    return (torch.empty(k, dtype=keys.dtype, device="cuda"),
            torch.empty(k, dtype=torch.uint32, device="cuda"),
            torch.empty(1, dtype=keys.dtype, device="cuda"),
            torch.empty(1, dtype=torch.uint32, device="cuda"))


def _call_noalloc(tk, clib, keys, k, out, status, stream):
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    return clib.topk_select_noalloc(p(keys), keys.numel(), k, tk.dtype_code(keys), p(out[0]), p(out[1]),
                                    p(out[2]), p(out[3]), p(status), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_topk_select_twice(lib):
    import torch
    tk, clib = lib
    ctx = tk.Context(0)
    stream = torch.cuda.current_stream()
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    cases = [
        (wl.uniform_u32(1_000_003, seed=21), "u32", 777),
        (wl.normal_f32(tk.NOALLOC_MAX_N, seed=22).view(np.uint32), "f32", tk.NOALLOC_MAX_N // 2),
    ]
    for bits, name, k in cases:  # two calls in a row share the scratch array
        keys = to_device(bits, name)
        out = _outputs(torch, keys, k)
        assert _call_noalloc(tk, clib, keys, k, out, status, stream) == tk.TOPK_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        ref = tk.topk_select(ctx, keys, k)
        got_idx, ref_idx = bits_of(out[1]), bits_of(ref[1])
        order, rorder = np.argsort(got_idx), np.argsort(ref_idx)
        assert np.array_equal(got_idx[order], ref_idx[rorder])
        assert np.array_equal(bits_of(out[0])[order], bits_of(ref[0])[rorder])
        assert np.array_equal(bits_of(out[2]), bits_of(ref[2]))
        assert np.array_equal(bits_of(out[3]), bits_of(ref[3]))
    ctx.close()


def test_noalloc_rejects_oversize(lib):
    import torch
    tk, clib = lib
    keys = torch.zeros(tk.NOALLOC_MAX_N + 1, dtype=torch.float32, device="cuda")
    out = _outputs(torch, keys, 4)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call_noalloc(tk, clib, keys, 4, out, status, torch.cuda.current_stream()) == tk.TOPK_EINVAL

"""The allocation-free selection entry point (GPU), through the C ABI.

Some callers of this library cannot allocate device memory at the moment
they call it: code running inside another framework's allocator or
memory-pool callbacks (allocating there would re-enter that allocator),
latency-critical loops that cannot accept the device-wide synchronisation
that cudaMalloc / cudaFree may cause, and programs that fix their device
memory when they start.  topk_select_noalloc serves them: its scratch is a
fixed array in device memory, so it accepts at most 2^22 keys.

Each case makes two calls in a row on the same stream, without waiting in
between, so the second reuses the scratch array the first just left; both
results must be bit-identical to the context-based entry point topk_select
and to the CPU oracle, for every key type and for k = 1, a small k, n/2 and
n.  This file is named to be collected after every other test file, so a run
that stops at the first failure has run all other tests before it; its
tests set up everything they use, so they also pass run on their own in a
fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1502_03942_gb300 import workloads as wl

from _gpu import bits_of, to_device

pytestmark = pytest.mark.gpu

MAX_N = 1 << 22  # the entry point's size limit (include/topk.h)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03942_gb300 as tk
    assert tk.NOALLOC_MAX_N == MAX_N
    return tk, tk.load_library()


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def _outputs(torch, keys, k):
    return (torch.empty(k, dtype=keys.dtype, device="cuda"),
            torch.empty(k, dtype=torch.uint32, device="cuda"),
            torch.empty(1, dtype=keys.dtype, device="cuda"),
            torch.empty(1, dtype=torch.uint32, device="cuda"))


def _call_noalloc(tk, clib, keys, k, out, status, stream):
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    return clib.topk_select_noalloc(p(keys), keys.numel(), k, tk.dtype_code(keys), p(out[0]), p(out[1]),
                                    p(out[2]), p(out[3]), p(status), ctypes.c_void_p(stream.cuda_stream))


def _bits_for(name, n, seed):
    if name in ("u32", "i32"):
        return wl.uniform_u32(n, seed)
    if name == "f32":
        return wl.normal_f32(n, seed).view(np.uint32)
    if name == "bf16":  # Zipf-tied bf16 keys: the position tie-break decides most of k
        return wl.zipf_bf16_bits(n, seed)
    return wl.uniform_u64(n, seed)


CASES = {"u32": 1_000_003, "i32": 300_007, "f32": MAX_N, "bf16": 2_000_001, "u64": MAX_N}


def _same(got, ref):
    """Bit-identical result sets (output order is unspecified)."""
    gi, ri = bits_of(got[1]), bits_of(ref[1])
    go, ro = np.argsort(gi), np.argsort(ri)
    return (np.array_equal(gi[go], ri[ro]) and np.array_equal(bits_of(got[0])[go], bits_of(ref[0])[ro])
            and np.array_equal(bits_of(got[2]), bits_of(ref[2]))
            and np.array_equal(bits_of(got[3]), bits_of(ref[3])))


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_matches_topk_select_and_oracle(lib, orc, name):
    import torch
    tk, clib = lib
    ctx = tk.Context(0)
    stream = torch.cuda.current_stream()
    n = CASES[name]
    inputs = [_bits_for(name, n, seed) for seed in (21, 22)]
    perms = [orc.sort_order(b, name) for b in inputs]  # one full sort answers every k
    keys = [to_device(b, name) for b in inputs]
    for k in (1, 777, n // 2, n):
        outs = [_outputs(torch, d, k) for d in keys]
        status = [torch.full((1,), 7, dtype=torch.int32, device="cuda") for _ in keys]
        for d, out, stw in zip(keys, outs, status):  # two calls in a row, one scratch array
            assert _call_noalloc(tk, clib, d, k, out, stw, stream) == tk.TOPK_OK
        torch.cuda.synchronize()
        for b, perm, d, out, stw in zip(inputs, perms, keys, outs, status):
            assert int(stw.item()) == 0
            ref = tk.topk_select(ctx, d, k)
            assert _same(out, ref), f"{name} n={n} k={k}: differs from topk_select"
            got_idx = bits_of(out[1])
            assert np.array_equal(np.sort(got_idx), np.sort(perm[:k])), "selected set differs from the oracle"
            assert np.array_equal(bits_of(out[0]), b[got_idx]), "output keys are not the input keys"
            assert int(bits_of(out[3])[0]) == int(perm[k - 1]), "rank-k position differs from the oracle"
            assert int(bits_of(out[2])[0]) == int(b[perm[k - 1]])
    ctx.close()


def test_noalloc_rejects_oversize_and_foreign_memory(lib):
    import torch
    tk, clib = lib
    stream = torch.cuda.current_stream()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    keys = torch.zeros(MAX_N + 1, dtype=torch.float32, device="cuda")
    assert _call_noalloc(tk, clib, keys, 4, _outputs(torch, keys, 4), status, stream) == tk.TOPK_EINVAL
    # keys in host memory are not memory of the current device: refused before any launch
    host = torch.zeros(1000, dtype=torch.float32, pin_memory=True)
    small = torch.zeros(1000, dtype=torch.float32, device="cuda")
    assert _call_noalloc(tk, clib, host, 4, _outputs(torch, small, 4), status, stream) == tk.TOPK_EINVAL
    torch.cuda.synchronize()

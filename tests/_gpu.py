"""Helpers shared by the GPU tests: moving key bits between numpy and torch
without any value conversion, and comparing library results with the oracle."""
from __future__ import annotations

import numpy as np

NP_BITS = {"u32": np.uint32, "i32": np.uint32, "f32": np.uint32, "bf16": np.uint16, "u64": np.uint64}
NP_SIGNED = {np.uint16: np.int16, np.uint32: np.int32, np.uint64: np.int64}


def torch_dtype(name):
    import torch
    return {"u32": torch.uint32, "i32": torch.int32, "f32": torch.float32,
            "bf16": torch.bfloat16, "u64": torch.uint64}[name]


def to_device(bits: np.ndarray, name: str):
    """Key bit patterns (unsigned numpy array) -> CUDA tensor of the key dtype."""
    import torch
    store = NP_BITS[name]
    b = np.ascontiguousarray(bits, dtype=store)
    t = torch.from_numpy(b.view(NP_SIGNED[store])).cuda()
    return t.view(torch_dtype(name))


def bits_of(t) -> np.ndarray:
    """CUDA tensor -> its raw bits as an unsigned numpy array."""
    import torch
    size = t.element_size()
    signed = {2: torch.int16, 4: torch.int32, 8: torch.int64}[size]
    unsigned = {2: np.uint16, 4: np.uint32, 8: np.uint64}[size]
    return t.view(signed).cpu().numpy().view(unsigned)


def check_against_oracle(keys_bits, name, k, out, orc):
    """Exact comparison of one topk_select result with the oracle."""
    ok, oi, kk, ki = out
    got_idx = bits_of(oi)
    got_keys = bits_of(ok)
    want_sel, want_kth = orc.select(keys_bits, name, k)
    assert got_idx.size == k
    assert np.array_equal(np.sort(got_idx), np.sort(want_sel)), "selected set differs"
    assert np.array_equal(got_keys, keys_bits[got_idx]), "output keys are not the input keys"
    assert int(bits_of(ki)[0]) == want_kth, "rank-k position differs"
    assert int(bits_of(kk)[0]) == int(keys_bits[want_kth]), "rank-k key differs"

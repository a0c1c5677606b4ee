"""CPU oracle for exact k-smallest selection — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it, and
it shares no code with the CUDA path.

The C file next to this one (``oracle.c``) states what is computed: all n pairs
(key, position) sorted once under the key type's value order (integers by
value, floats by IEEE 754 totalOrder), first k taken (paper, Section 2 for the
(value, position) tie-break, Section 4 for the problem, Appendix A for the
multisequence split positions, Section 5 for deleteMin* over runs with
cursors).  For the top-k most frequent objects (Section 7) it follows the
algorithms' steps on one PE: Bernoulli sample decisions from Philox4x32-10
(written from its published definition), counting by sort-and-run-length,
the k (PAC) or k* (EC, then an exact recount) most frequent.  This module
only loads that library and moves numpy arrays in and out of it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH, build as _build

DTYPE_CODES = {"u32": 0, "i32": 1, "f32": 2, "bf16": 3, "u64": 4}
NP_STORAGE = {"u32": np.uint32, "i32": np.uint32, "f32": np.uint32,
              "bf16": np.uint16, "u64": np.uint64}


def _bits(keys: np.ndarray, dtype: str) -> np.ndarray:
    """Raw key bits as a contiguous unsigned array of the key's width."""
    store = NP_STORAGE[dtype]
    a = np.ascontiguousarray(keys)
    if a.dtype.itemsize != np.dtype(store).itemsize:
        raise ValueError(f"{dtype} keys need {np.dtype(store).itemsize}-byte items")
    return a.view(store)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Oracle:
    """The oracle library at ``path`` with numpy-level entry points."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        vp = ctypes.c_void_p
        lib.oracle_key_cmp.argtypes = [i32, u64, u64]
        lib.oracle_key_cmp.restype = i32
        lib.oracle_sort_order.argtypes = [vp, u64, i32, vp]
        lib.oracle_sort_order.restype = i32
        lib.oracle_select.argtypes = [vp, u64, i32, u64, vp, vp]
        lib.oracle_select.restype = i32
        lib.oracle_select_largest.argtypes = [vp, u64, i32, u64, vp, vp]
        lib.oracle_select_largest.restype = i32
        lib.oracle_pairs_before.argtypes = [vp, u64, i32, u64, i32, vp]
        lib.oracle_pairs_before.restype = i32
        lib.oracle_check_selection.argtypes = [vp, u64, i32, u64, i32, vp, vp, u64, vp]
        lib.oracle_check_selection.restype = i32
        lib.oracle_select_runs.argtypes = [vp, vp, u32, u64, vp, vp, vp]
        lib.oracle_select_runs.restype = i32
        lib.oracle_runs_delete_min.argtypes = [vp, vp, u32, vp, u64, vp, vp]
        lib.oracle_runs_delete_min.restype = i32
        lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_sample_threshold.argtypes = [ctypes.c_double]
        lib.oracle_sample_threshold.restype = u64
        lib.oracle_bernoulli_sample.argtypes = [u64, u64, u64, vp]
        lib.oracle_bernoulli_sample.restype = i32
        lib.oracle_frequent.argtypes = [vp, u64, vp, u32, u32, i32, vp, vp, vp]
        lib.oracle_frequent.restype = i32
        lib.oracle_frequent_plan.argtypes = [u64, u32, ctypes.c_double, ctypes.c_double, u32, i32, vp, vp]
        lib.oracle_frequent_plan.restype = i32
        lib.oracle_select_batched.argtypes = [vp, vp, vp, u32, i32, vp, vp, vp]
        lib.oracle_select_batched.restype = i32
        self.lib = lib
        self.path = path

    def key_cmp(self, dtype: str, a: int, b: int) -> int:
        """-1/0/+1 comparison of two raw key bit patterns."""
        return self.lib.oracle_key_cmp(DTYPE_CODES[dtype], int(a), int(b))

    def sort_order(self, keys: np.ndarray, dtype: str) -> np.ndarray:
        """Permutation listing positions in ascending (key, position) order."""
        k = _bits(keys, dtype)
        perm = np.empty(k.size, np.uint32)
        if self.lib.oracle_sort_order(_ptr(k), k.size, DTYPE_CODES[dtype], _ptr(perm)) != 0:
            raise ValueError("oracle_sort_order rejected its arguments")
        return perm

    def select(self, keys: np.ndarray, dtype: str, k: int):
        """(sel_idx ascending by pair order, kth_idx) of the k smallest pairs."""
        a = _bits(keys, dtype)
        sel = np.empty(max(int(k), 1), np.uint32)
        kth = np.zeros(1, np.uint32)
        if self.lib.oracle_select(_ptr(a), a.size, DTYPE_CODES[dtype], int(k),
                                  _ptr(sel), _ptr(kth)) != 0:
            raise ValueError("oracle_select rejected its arguments")
        return sel[: int(k)], int(kth[0])

    def select_largest(self, keys: np.ndarray, dtype: str, k: int):
        """(sel_idx in descending value order, kth_idx) of the k largest;
        equal values by ascending position."""
        a = _bits(keys, dtype)
        sel = np.empty(max(int(k), 1), np.uint32)
        kth = np.zeros(1, np.uint32)
        if self.lib.oracle_select_largest(_ptr(a), a.size, DTYPE_CODES[dtype], int(k), _ptr(sel),
                                          _ptr(kth)) != 0:
            raise ValueError("oracle_select_largest rejected its arguments")
        return sel[: int(k)], int(kth[0])

    def pairs_before(self, keys: np.ndarray, dtype: str, pos: int, descending: bool = False) -> int:
        """Number of pairs preceding (keys[pos], pos) in the ascending (or,
        with ``descending``, the descending) value order, ties by position."""
        a = _bits(keys, dtype)
        c = np.zeros(1, np.uint64)
        if self.lib.oracle_pairs_before(_ptr(a), a.size, DTYPE_CODES[dtype], int(pos),
                                        1 if descending else 0, _ptr(c)) != 0:
            raise ValueError("oracle_pairs_before rejected its arguments")
        return int(c[0])

    def check_selection(self, keys: np.ndarray, dtype: str, k: int, sel_idx: np.ndarray, kth: int,
                        out_keys: np.ndarray | None = None, kth_key: np.ndarray | None = None,
                        descending: bool = False) -> int:
        """0 if (sel_idx, out_keys, kth, kth_key) is exactly the k smallest
        (largest) pairs with their input keys; else the code of the first
        failed condition (see oracle.h)."""
        a = _bits(keys, dtype)
        sel = np.ascontiguousarray(sel_idx, dtype=np.uint32)
        if sel.size != int(k):
            return 2
        ok = _ptr(_bits(out_keys, dtype)) if out_keys is not None else None
        kk = _ptr(_bits(kth_key, dtype)) if kth_key is not None else None
        keep = (out_keys, kth_key)  # alive during the call
        r = self.lib.oracle_check_selection(_ptr(a), a.size, DTYPE_CODES[dtype], int(k),
                                            1 if descending else 0, _ptr(sel), ok, int(kth), kk)
        del keep
        if r < 0:
            raise ValueError("oracle_check_selection rejected its arguments")
        return int(r)

    def select_runs(self, keys: np.ndarray, run_off: np.ndarray, k: int):
        """(split[p], kth_run, kth_pos) for multisequence selection of rank k."""
        a = _bits(keys, "u64")
        off = np.ascontiguousarray(run_off, dtype=np.uint64)
        p = off.size - 1
        split = np.zeros(p, np.uint64)
        kr = np.zeros(1, np.uint32)
        kp = np.zeros(1, np.uint64)
        if self.lib.oracle_select_runs(_ptr(a), _ptr(off), p, int(k), _ptr(split),
                                       _ptr(kr), _ptr(kp)) != 0:
            raise ValueError("oracle_select_runs rejected its arguments")
        return split, int(kr[0]), int(kp[0])

    def runs_delete_min(self, keys: np.ndarray, run_off: np.ndarray, cursor: np.ndarray, k: int):
        """(new cursor[p], kth_run, kth_pos) after deleting the k smallest
        objects at or after the cursors (Section 5, deleteMin*)."""
        a = _bits(keys, "u64")
        off = np.ascontiguousarray(run_off, dtype=np.uint64)
        p = off.size - 1
        cur = np.array(cursor, dtype=np.uint64, copy=True)
        kr = np.zeros(1, np.uint32)
        kp = np.zeros(1, np.uint64)
        if self.lib.oracle_runs_delete_min(_ptr(a), _ptr(off), p, _ptr(cur), int(k), _ptr(kr),
                                           _ptr(kp)) != 0:
            raise ValueError("oracle_runs_delete_min rejected its arguments")
        return cur, int(kr[0]), int(kp[0])

    # ---- top-k most frequent objects (Section 7) ----

    def philox(self, ctr, key):
        c = np.ascontiguousarray(ctr, dtype=np.uint32)
        kk = np.ascontiguousarray(key, dtype=np.uint32)
        out = np.zeros(4, np.uint32)
        self.lib.oracle_philox4x32_10(_ptr(c), _ptr(kk), _ptr(out))
        return out

    def sample_threshold(self, rho: float) -> int:
        return int(self.lib.oracle_sample_threshold(float(rho)))

    def bernoulli_sample(self, n: int, seed: int, threshold: int) -> np.ndarray:
        """mask[n] uint8: 1 where element i is sampled (Section 7.1)."""
        mask = np.zeros(max(n, 1), np.uint8)
        if self.lib.oracle_bernoulli_sample(int(n), int(seed), int(threshold), _ptr(mask)) != 0:
            raise ValueError("oracle_bernoulli_sample rejected its arguments")
        return mask[:n]

    def frequent(self, objects: np.ndarray, mask: np.ndarray, k: int, kstar: int = 0,
                 exact: bool = False):
        """(objects[k], counts[k], sample_size): Algorithm PAC (sample counts)
        or EC (exact counts of the k most frequent of k* candidates), most
        frequent first, equal counts by the smaller object."""
        obj = np.ascontiguousarray(objects, dtype=np.uint32)
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        out_obj = np.zeros(k, np.uint32)
        out_cnt = np.zeros(k, np.uint64)
        ss = np.zeros(1, np.uint64)
        if self.lib.oracle_frequent(_ptr(obj), obj.size, _ptr(m), int(k), int(kstar), int(bool(exact)),
                                    _ptr(out_obj), _ptr(out_cnt), _ptr(ss)) != 0:
            raise ValueError("oracle_frequent rejected its arguments")
        return out_obj, out_cnt, int(ss[0])

    def frequent_plan(self, n: int, k: int, eps: float, delta: float, pes: int = 1,
                      exact: bool = False):
        """(rho, kstar) from the accuracy targets (Sections 7.1, 7.2)."""
        rho = np.zeros(1, np.float64)
        ks = np.zeros(1, np.uint32)
        if self.lib.oracle_frequent_plan(int(n), int(k), float(eps), float(delta), int(pes),
                                         int(bool(exact)), _ptr(rho), _ptr(ks)) != 0:
            raise ValueError("oracle_frequent_plan rejected its arguments")
        return float(rho[0]), int(ks[0])

    def select_batched(self, keys: np.ndarray, row_off: np.ndarray, row_k: np.ndarray,
                       dtype: str):
        """(sel_idx concatenated per row, out_off, kth_idx[rows]); indices row-local."""
        a = _bits(keys, dtype)
        off = np.ascontiguousarray(row_off, dtype=np.uint64)
        rk = np.ascontiguousarray(row_k, dtype=np.uint32)
        rows = rk.size
        out_off = np.zeros(rows + 1, np.uint64)
        out_off[1:] = np.cumsum(rk.astype(np.uint64))
        sel = np.empty(max(int(out_off[-1]), 1), np.uint32)
        kth = np.zeros(max(rows, 1), np.uint32)
        if self.lib.oracle_select_batched(_ptr(a), _ptr(off), _ptr(rk), rows,
                                          DTYPE_CODES[dtype], _ptr(out_off), _ptr(sel),
                                          _ptr(kth)) != 0:
            raise ValueError("oracle_select_batched rejected its arguments")
        return sel[: int(out_off[-1])], out_off, kth[:rows]


class CpuBaselines:
    """The benchmark's timed CPU baselines (``cpu_baselines.cpp``): threaded
    sort-and-take and one-core std::nth_element over float32 keys."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        lib.cpu_sort_chunks_f32.argtypes = [vp, u64, i32, vp]
        lib.cpu_sort_chunks_f32.restype = i32
        lib.cpu_take_k.argtypes = [vp, u64, i32, u64, vp, vp]
        lib.cpu_take_k.restype = i32
        lib.cpu_nth_element_f32.argtypes = [vp, u64, u64, vp, vp]
        lib.cpu_nth_element_f32.restype = i32
        self.lib = lib

    def sort_chunks(self, bits: np.ndarray, threads: int, work: np.ndarray):
        b = np.ascontiguousarray(bits, dtype=np.uint32)
        if self.lib.cpu_sort_chunks_f32(_ptr(b), b.size, int(threads), _ptr(work)) != 0:
            raise ValueError("cpu_sort_chunks_f32 rejected its arguments")

    def take_k(self, work: np.ndarray, threads: int, k: int, sel: np.ndarray) -> int:
        kth = np.zeros(1, np.uint32)
        if self.lib.cpu_take_k(_ptr(work), work.size, int(threads), int(k), _ptr(sel), _ptr(kth)) != 0:
            raise ValueError("cpu_take_k rejected its arguments")
        return int(kth[0])

    def nth_element(self, bits: np.ndarray, k: int, work: np.ndarray) -> int:
        b = np.ascontiguousarray(bits, dtype=np.uint32)
        kth = np.zeros(1, np.uint32)
        if self.lib.cpu_nth_element_f32(_ptr(b), b.size, int(k), _ptr(work), _ptr(kth)) != 0:
            raise ValueError("cpu_nth_element_f32 rejected its arguments")
        return int(kth[0])


def cpu_baselines() -> CpuBaselines:
    from .build import build_baselines
    return CpuBaselines(build_baselines())


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(_build())
    return _default


def key_cmp(dtype, a, b):
    return default().key_cmp(dtype, a, b)


def sort_order(keys, dtype):
    return default().sort_order(keys, dtype)


def select(keys, dtype, k):
    return default().select(keys, dtype, k)


def select_largest(keys, dtype, k):
    return default().select_largest(keys, dtype, k)


def select_runs(keys, run_off, k):
    return default().select_runs(keys, run_off, k)


def runs_delete_min(keys, run_off, cursor, k):
    return default().runs_delete_min(keys, run_off, cursor, k)


def select_batched(keys, row_off, row_k, dtype):
    return default().select_batched(keys, row_off, row_k, dtype)


def bernoulli_sample(n, seed, threshold):
    return default().bernoulli_sample(n, seed, threshold)


def sample_threshold(rho):
    return default().sample_threshold(rho)


def frequent(objects, mask, k, kstar=0, exact=False):
    return default().frequent(objects, mask, k, kstar, exact)


def frequent_plan(n, k, eps, delta, pes=1, exact=False):
    return default().frequent_plan(n, k, eps, delta, pes, exact)

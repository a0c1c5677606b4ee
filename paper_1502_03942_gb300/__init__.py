"""Python binding of libtopk (include/topk.h): exact k-smallest selection on a
GB300 GPU.

Argument marshalling only.  Every step of the selection runs in the library's
CUDA kernels; PyTorch provides device memory and streams.  There is no CPU
fallback: if the compiled library is missing, every call raises.

The C names are kept: ``topk_select``, ``topk_select_sorted_runs``,
``topk_select_batched``, ``topk_status_sync`` and the ``topk_serve_*`` family,
each taking a :class:`Context` (or server) first and torch tensors for the
device buffers.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtopk.so")

TOPK_U32, TOPK_I32, TOPK_F32, TOPK_BF16, TOPK_U64 = 0, 1, 2, 3, 4
TOPK_OK, TOPK_EINVAL, TOPK_ENOMEM, TOPK_ECUDA, TOPK_ETIMEOUT = 0, 1, 2, 3, 4
TOPK_EBUDGET, TOPK_EBUSY, TOPK_EINTERNAL = 5, 6, 7
TOPK_FLAG_CHECK_SORTED = 0x1
TOPK_FLAG_RAW_DELTA = 0x2
TOPK_FLAG_TINY_CAND = 0x4
TOPK_FLAG_NO_BULK_COPY = 0x8
TOPK_FLAG_LARGEST = 0x10

DTYPE_NAMES = {TOPK_U32: "u32", TOPK_I32: "i32", TOPK_F32: "f32", TOPK_BF16: "bf16",
               TOPK_U64: "u64"}


class TopkError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


class topk_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("partitions", ctypes.c_uint32),
                ("sample_size", ctypes.c_uint32), ("buckets", ctypes.c_uint32),
                ("finish_threshold", ctypes.c_uint32), ("delta_factor", ctypes.c_float),
                ("flags", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("split_rows", ctypes.c_uint32)]


TOPK_FREQ_PAC = 0
TOPK_FREQ_EC = 1


class topk_freq_params(ctypes.Structure):
    _fields_ = [("algorithm", ctypes.c_uint32), ("k", ctypes.c_uint32), ("epsilon", ctypes.c_double),
                ("delta", ctypes.c_double), ("rho", ctypes.c_double), ("kstar", ctypes.c_uint32),
                ("pes", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("max_distinct", ctypes.c_uint64)]


class topk_stats(ctypes.Structure):
    _fields_ = [("levels_grid", ctypes.c_uint32), ("levels_block", ctypes.c_uint32),
                ("pivot_failures", ctypes.c_uint32), ("overflows", ctypes.c_uint32),
                ("first_candidates", ctypes.c_uint64), ("sample_kept", ctypes.c_uint64)]


class topk_request(ctypes.Structure):
    _fields_ = [("d_keys", ctypes.c_void_p), ("n", ctypes.c_uint64), ("k", ctypes.c_uint64),
                ("dtype", ctypes.c_int), ("d_out_keys", ctypes.c_void_p), ("d_out_idx", ctypes.c_void_p),
                ("d_kth_key", ctypes.c_void_p), ("d_kth_idx", ctypes.c_void_p),
                ("arrival_ns", ctypes.c_uint64)]


class topk_serve_report(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("keys", ctypes.c_uint64),
                ("p50_ns", ctypes.c_uint64), ("p99_ns", ctypes.c_uint64), ("max_ns", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("batched_requests", ctypes.c_uint64),
                ("peak_inflight_bytes", ctypes.c_uint64), ("elapsed_s", ctypes.c_double),
                ("reserved_bytes", ctypes.c_uint64), ("budget_waits", ctypes.c_uint64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libtopk.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtopk.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    st = ctypes.c_int
    lib.topk_ctx_create.argtypes = [ctypes.POINTER(vp), i32]
    lib.topk_ctx_create.restype = st
    lib.topk_ctx_destroy.argtypes = [vp]
    lib.topk_ctx_destroy.restype = None
    lib.topk_ctx_reserve.argtypes = [vp, u64, i32]
    lib.topk_ctx_reserve.restype = st
    lib.topk_select.argtypes = [vp, vp, u64, u64, i32, vp, vp, vp, vp, vp, vp]
    lib.topk_select.restype = st
    if hasattr(lib, "topk_select_sorted_runs"):
        lib.topk_select_sorted_runs.argtypes = [vp, vp, vp, u32, u64, i32, vp, vp, vp, vp, vp, vp]
        lib.topk_select_sorted_runs.restype = st
    if hasattr(lib, "topk_select_sorted_runs_flexible"):
        lib.topk_select_sorted_runs_flexible.argtypes = [vp, vp, vp, u32, u64, u64, i32, vp, vp, vp, vp, vp, vp, vp]
        lib.topk_select_sorted_runs_flexible.restype = st
    if hasattr(lib, "topk_select_kth"):
        lib.topk_select_kth.argtypes = [vp, vp, u64, u64, i32, vp, vp, vp, vp]
        lib.topk_select_kth.restype = st
    if hasattr(lib, "topk_frequent"):
        lib.topk_frequent_plan.argtypes = [u64, ctypes.POINTER(topk_freq_params), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(u32)]
        lib.topk_frequent_plan.restype = st
        lib.topk_frequent.argtypes = [vp, vp, u64, i32, ctypes.POINTER(topk_freq_params), vp, vp, vp, vp]
        lib.topk_frequent.restype = st
    if hasattr(lib, "topk_runs_delete_min"):
        lib.topk_runs_delete_min.argtypes = [vp, vp, vp, u32, vp, u64, i32, vp, vp, vp, vp, vp]
        lib.topk_runs_delete_min.restype = st
        lib.topk_runs_delete_min_flexible.argtypes = [vp, vp, vp, u32, vp, u64, u64, i32, vp, vp, vp, vp, vp, vp]
        lib.topk_runs_delete_min_flexible.restype = st
    if hasattr(lib, "topk_select_batched"):
        lib.topk_select_batched.argtypes = [vp, vp, vp, vp, u32, i32, vp, vp, vp, vp, vp, vp, vp]
        lib.topk_select_batched.restype = st
    if hasattr(lib, "topk_debug_wait_timeout"):
        lib.topk_debug_wait_timeout.argtypes = [vp, u32, vp]
        lib.topk_debug_wait_timeout.restype = st
    if hasattr(lib, "topk_tune_batched"):
        lib.topk_tune_batched.argtypes = [vp, vp, vp, vp, u32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.topk_tune_batched.restype = st
        lib.topk_tuning_save.argtypes = [vp, ctypes.c_char_p]
        lib.topk_tuning_save.restype = st
        lib.topk_tuning_load.argtypes = [vp, ctypes.c_char_p]
        lib.topk_tuning_load.restype = st
    if hasattr(lib, "topk_select_noalloc"):
        lib.topk_select_noalloc.argtypes = [vp, u64, u64, i32, vp, vp, vp, vp, vp, vp]
        lib.topk_select_noalloc.restype = st
    if hasattr(lib, "topk_serve_create"):
        lib.topk_serve_create.argtypes = [ctypes.POINTER(vp), i32, u64, u32]
        lib.topk_serve_create.restype = st
        lib.topk_serve_submit.argtypes = [vp, ctypes.POINTER(topk_request), ctypes.POINTER(u64)]
        if hasattr(lib, "topk_serve_replay"):
            lib.topk_serve_replay.argtypes = [vp, vp, vp, u64, vp, vp]
            lib.topk_serve_replay.restype = st
        lib.topk_serve_submit.restype = st
        lib.topk_serve_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int)]
        lib.topk_serve_poll.restype = st
        lib.topk_serve_wait.argtypes = [vp, u64, u64]
        lib.topk_serve_wait.restype = st
        lib.topk_serve_stats.argtypes = [vp, ctypes.POINTER(topk_serve_report)]
        lib.topk_serve_stats.restype = st
        lib.topk_serve_now_ns.argtypes = [vp]
        lib.topk_serve_now_ns.restype = u64
        lib.topk_serve_destroy.argtypes = [vp]
        lib.topk_serve_destroy.restype = None
    lib.topk_status_sync.argtypes = [vp, vp]
    lib.topk_status_sync.restype = st
    lib.topk_last_stats.argtypes = [vp, ctypes.POINTER(topk_stats)]
    lib.topk_last_stats.restype = st
    lib.topk_status_string.argtypes = [st]
    lib.topk_status_string.restype = ctypes.c_char_p
    lib.topk_ctx_profile.argtypes = [vp, i32]
    lib.topk_ctx_profile.restype = st
    lib.topk_ctx_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64),
                                          ctypes.POINTER(u64), i32]
    lib.topk_ctx_profile_read.restype = st
    lib.topk_debug_philox.argtypes = [u32, u32, u32, u32, u32, u32, vp, u32]
    lib.topk_debug_philox.restype = st
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load_library().topk_status_string(status).decode()
    except RuntimeError:
        return f"status {status}"


def _check(status: int, what: str):
    if status != TOPK_OK:
        raise TopkError(status, what)


def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    m = {torch.uint32: TOPK_U32, torch.int32: TOPK_I32, torch.float32: TOPK_F32,
         torch.bfloat16: TOPK_BF16, torch.uint64: TOPK_U64}
    if t.dtype not in m:
        raise TypeError(f"unsupported key dtype {t.dtype}")
    return m[t.dtype]


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


TOPK_SPLIT_NONE = 0xFFFFFFFF


def make_params(seed=0, partitions=0, sample_size=0, finish_threshold=0, delta_factor=0.0,
                flags=0, block_threads=0, split_rows=0) -> topk_params:
    return topk_params(seed, partitions, sample_size, 0, finish_threshold, delta_factor, flags, block_threads,
                       split_rows)


class Context:
    """Owns a topk_ctx (device scratch + latched device status)."""

    def __init__(self, device: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.topk_ctx_create(ctypes.byref(h), int(device)), "topk_ctx_create")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load_library().topk_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, n: int, dtype: int):
        _check(load_library().topk_ctx_reserve(self.handle, int(n), int(dtype)), "topk_ctx_reserve")

    def sync(self, stream=None) -> int:
        """topk_status_sync: waits for the stream, returns the latched status."""
        return load_library().topk_status_sync(self.handle, _stream_ptr(stream))

    def profile(self, enable: bool = True):
        """Count kernel launches and time the first-level pass with CUDA events."""
        _check(load_library().topk_ctx_profile(self.handle, 1 if enable else 0), "topk_ctx_profile")

    def profile_read(self, reset: bool = True) -> dict:
        ms, passes, launches = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load_library().topk_ctx_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(passes),
                                                    ctypes.byref(launches), 1 if reset else 0),
               "topk_ctx_profile_read")
        return {"pass_ms": ms.value, "passes": passes.value, "launches": launches.value}

    def last_stats(self) -> dict:
        s = topk_stats()
        _check(load_library().topk_last_stats(self.handle, ctypes.byref(s)), "topk_last_stats")
        return {f: getattr(s, f) for f, _ in topk_stats._fields_}


def topk_select(ctx: Context, keys, k: int, params: topk_params | None = None, stream=None,
                out=None, check: bool = True):
    """k smallest of the 1-D CUDA tensor ``keys``.

    Returns (out_keys[k], out_idx[k] uint32, kth_key[1], kth_idx[1] uint32) as
    CUDA tensors (outputs allocated here unless ``out`` gives all four).  With
    ``check`` the call waits and raises on a latched device error."""
    torch = _torch()
    if keys.dim() != 1 or not keys.is_cuda:
        raise ValueError("keys must be a 1-D CUDA tensor")
    if not keys.is_contiguous():
        raise ValueError("keys must be contiguous")
    n = keys.numel()
    if out is None:
        kk = max(int(k), 1)
        out = (torch.empty(kk, dtype=keys.dtype, device=keys.device),
               torch.empty(kk, dtype=torch.uint32, device=keys.device),
               torch.empty(1, dtype=keys.dtype, device=keys.device),
               torch.empty(1, dtype=torch.uint32, device=keys.device))
    ok, oi, kk_, ki = out
    st = load_library().topk_select(
        ctx.handle, _ptr(keys), n, int(k), dtype_code(keys), _ptr(ok), _ptr(oi), _ptr(kk_), _ptr(ki),
        ctypes.byref(params) if params is not None else None, _stream_ptr(stream))
    _check(st, "topk_select")
    if check:
        _check(ctx.sync(stream), "topk_select (device)")
    return out


def topk_select_sorted_runs(ctx: Context, keys, run_off, k: int, params: topk_params | None = None,
                            stream=None, out=None, check: bool = True):
    """Rank-k selection over p sorted runs of uint64 keys stored back to back.

    ``run_off``: p + 1 uint64 offsets on the device.  Returns (split[p] uint64,
    kth_key[1] uint64, kth_run[1] uint32, kth_pos[1] uint64)."""
    torch = _torch()
    if keys.dtype != torch.uint64 or run_off.dtype != torch.uint64:
        raise TypeError("keys and run_off must be uint64 tensors")
    p = run_off.numel() - 1
    if out is None:
        out = (torch.empty(max(p, 1), dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint32, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device))
    split, kk, kr, kp = out
    st = load_library().topk_select_sorted_runs(
        ctx.handle, _ptr(keys), _ptr(run_off), p, int(k), TOPK_U64, _ptr(split), _ptr(kk), _ptr(kr),
        _ptr(kp), ctypes.byref(params) if params is not None else None, _stream_ptr(stream))
    _check(st, "topk_select_sorted_runs")
    if check:
        _check(ctx.sync(stream), "topk_select_sorted_runs (device)")
    return out


def topk_select_sorted_runs_flexible(ctx: Context, keys, run_off, kmin: int, kmax: int,
                                     params: topk_params | None = None, stream=None, out=None, check: bool = True):
    """The k smallest over p sorted runs for some k in [kmin, kmax] (amsSelect).

    Returns (split[p] uint64, kth_key[1] uint64, kth_run[1] uint32,
    kth_pos[1] uint64, k[1] uint64)."""
    torch = _torch()
    if keys.dtype != torch.uint64 or run_off.dtype != torch.uint64:
        raise TypeError("keys and run_off must be uint64 tensors")
    p = run_off.numel() - 1
    if out is None:
        out = (torch.empty(max(p, 1), dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint32, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device))
    split, kk, kr, kp, kout = out
    st = load_library().topk_select_sorted_runs_flexible(
        ctx.handle, _ptr(keys), _ptr(run_off), p, int(kmin), int(kmax), TOPK_U64, _ptr(split), _ptr(kk), _ptr(kr),
        _ptr(kp), _ptr(kout), ctypes.byref(params) if params is not None else None, _stream_ptr(stream))
    _check(st, "topk_select_sorted_runs_flexible")
    if check:
        _check(ctx.sync(stream), "topk_select_sorted_runs_flexible (device)")
    return out


def topk_runs_delete_min(ctx: Context, keys, run_off, cursor, k: int, params: topk_params | None = None,
                         stream=None, out=None, check: bool = True):
    """Bulk deleteMin* over a queue of p sorted runs with cursors (Section 5):
    deletes the k smallest objects after the cursors and advances ``cursor``
    (p uint64 CUDA tensor, updated in place) past them.

    Returns (kth_key[1] uint64, kth_run[1] uint32, kth_pos[1] uint64): the
    largest object deleted."""
    torch = _torch()
    if keys.dtype != torch.uint64 or run_off.dtype != torch.uint64 or cursor.dtype != torch.uint64:
        raise TypeError("keys, run_off and cursor must be uint64 tensors")
    p = run_off.numel() - 1
    if cursor.numel() != p:
        raise ValueError("cursor needs one entry per run")
    if out is None:
        out = (torch.empty(1, dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint32, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device))
    kk, kr, kp = out
    st = load_library().topk_runs_delete_min(
        ctx.handle, _ptr(keys), _ptr(run_off), p, _ptr(cursor), int(k), TOPK_U64, _ptr(kk), _ptr(kr), _ptr(kp),
        ctypes.byref(params) if params is not None else None, _stream_ptr(stream))
    _check(st, "topk_runs_delete_min")
    if check:
        _check(ctx.sync(stream), "topk_runs_delete_min (device)")
    return out


def topk_runs_delete_min_flexible(ctx: Context, keys, run_off, cursor, kmin: int, kmax: int,
                                  params: topk_params | None = None, stream=None, out=None, check: bool = True):
    """Flexible bulk deleteMin*: deletes the k smallest remaining objects for
    some k in [kmin, kmax] and advances ``cursor`` in place.

    Returns (kth_key[1], kth_run[1], kth_pos[1], k[1] uint64)."""
    torch = _torch()
    if keys.dtype != torch.uint64 or run_off.dtype != torch.uint64 or cursor.dtype != torch.uint64:
        raise TypeError("keys, run_off and cursor must be uint64 tensors")
    p = run_off.numel() - 1
    if cursor.numel() != p:
        raise ValueError("cursor needs one entry per run")
    if out is None:
        out = (torch.empty(1, dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint32, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device),
               torch.empty(1, dtype=torch.uint64, device=keys.device))
    kk, kr, kp, kout = out
    st = load_library().topk_runs_delete_min_flexible(
        ctx.handle, _ptr(keys), _ptr(run_off), p, _ptr(cursor), int(kmin), int(kmax), TOPK_U64, _ptr(kk),
        _ptr(kr), _ptr(kp), _ptr(kout), ctypes.byref(params) if params is not None else None,
        _stream_ptr(stream))
    _check(st, "topk_runs_delete_min_flexible")
    if check:
        _check(ctx.sync(stream), "topk_runs_delete_min_flexible (device)")
    return out


def topk_select_kth(ctx: Context, keys, k: int, params: topk_params | None = None, stream=None, out=None,
                    check: bool = True):
    """The key of rank k and its position (the k-th smallest, or the k-th
    largest with TOPK_FLAG_LARGEST); the selected set stays in the context.
    Returns (kth_key[1] of the key dtype, kth_idx[1] uint32)."""
    torch = _torch()
    if out is None:
        out = (torch.empty(1, dtype=keys.dtype, device=keys.device),
               torch.empty(1, dtype=torch.uint32, device=keys.device))
    kk, ki = out
    st = load_library().topk_select_kth(ctx.handle, _ptr(keys), keys.numel(), int(k), dtype_code(keys), _ptr(kk),
                                        _ptr(ki), ctypes.byref(params) if params is not None else None,
                                        _stream_ptr(stream))
    _check(st, "topk_select_kth")
    if check:
        _check(ctx.sync(stream), "topk_select_kth (device)")
    return out


def make_freq_params(k: int, algorithm: int = TOPK_FREQ_EC, epsilon: float = 3e-4, delta: float = 1e-4,
                     rho: float = 0.0, kstar: int = 0, pes: int = 0, seed: int = 0x5EED,
                     max_distinct: int = 0) -> topk_freq_params:
    return topk_freq_params(algorithm=algorithm, k=k, epsilon=epsilon, delta=delta, rho=rho, kstar=kstar,
                            pes=pes, seed=seed, max_distinct=max_distinct)


def topk_frequent_plan(n: int, fp: topk_freq_params):
    """(rho, kstar) that topk_frequent uses for n objects (host only)."""
    rho = ctypes.c_double()
    ks = ctypes.c_uint32()
    _check(load_library().topk_frequent_plan(int(n), ctypes.byref(fp), ctypes.byref(rho), ctypes.byref(ks)),
           "topk_frequent_plan")
    return rho.value, ks.value


def topk_frequent(ctx: Context, objects, fp: topk_freq_params, stream=None, out=None, check: bool = True):
    """Top-k most frequent of the uint32 objects (Algorithm PAC or EC,
    Section 7).  Returns (objects[k] uint32, counts[k] uint64,
    sample_size[1] uint64); counts are sample counts (PAC) or exact counts
    (EC); any order."""
    torch = _torch()
    if objects.dtype not in (torch.uint32, torch.int32):
        raise TypeError("objects must be a 32-bit tensor")
    k = int(fp.k)
    if out is None:
        out = (torch.empty(k, dtype=torch.uint32, device=objects.device),
               torch.empty(k, dtype=torch.uint64, device=objects.device),
               torch.empty(1, dtype=torch.uint64, device=objects.device))
    oo, oc, ss = out
    st = load_library().topk_frequent(ctx.handle, _ptr(objects), objects.numel(), TOPK_U32, ctypes.byref(fp),
                                      _ptr(oo), _ptr(oc), _ptr(ss), _stream_ptr(stream))
    _check(st, "topk_frequent")
    if check:
        _check(ctx.sync(stream), "topk_frequent (device)")
    return out


def topk_select_batched(ctx: Context, keys, row_off, row_k, params: topk_params | None = None,
                        stream=None, out=None, out_off=None, check: bool = True):
    """Independent selections over the rows keys[row_off[i]:row_off[i+1]],
    each with its own k = row_k[i], in one persistent launch.

    ``row_off``: rows + 1 uint64 CUDA offsets; ``row_k``: rows uint32.  The
    output offsets are the prefix sums of row_k (computed here with torch
    unless ``out_off`` is given).  Returns (out_keys, out_idx row-local
    uint32, kth_keys[rows], kth_idx[rows] uint32, out_off)."""
    torch = _torch()
    rows = row_k.numel()
    if out_off is None:
        out_off = torch.zeros(rows + 1, dtype=torch.int64, device=keys.device)
        out_off[1:] = torch.cumsum(row_k.view(torch.int32).to(torch.int64), 0)
        out_off = out_off.view(torch.uint64)
    if out is None:
        total = int(out_off.view(torch.int64)[-1].item())
        out = (torch.empty(max(total, 1), dtype=keys.dtype, device=keys.device),
               torch.empty(max(total, 1), dtype=torch.uint32, device=keys.device),
               torch.empty(rows, dtype=keys.dtype, device=keys.device),
               torch.empty(rows, dtype=torch.uint32, device=keys.device))
    ok, oi, kk, ki = out
    st = load_library().topk_select_batched(
        ctx.handle, _ptr(keys), _ptr(row_off), _ptr(row_k), rows, dtype_code(keys), _ptr(ok), _ptr(oi),
        _ptr(out_off), _ptr(kk), _ptr(ki), ctypes.byref(params) if params is not None else None,
        _stream_ptr(stream))
    _check(st, "topk_select_batched")
    if check:
        _check(ctx.sync(stream), "topk_select_batched (device)")
    return ok, oi, kk, ki, out_off


def topk_tune_batched(ctx: Context, keys, row_off, row_k, out, out_off, base: topk_params | None = None,
                      stream=None) -> topk_params:
    """Times every candidate setting of topk_select_batched on this batch and
    makes the fastest the context's choice for its dtype and row count;
    returns it.  ``out`` / ``out_off`` as topk_select_batched (overwritten;
    they end up holding the chosen setting's result)."""
    ok, oi, kk, ki = out
    best = topk_params()
    st = load_library().topk_tune_batched(
        ctx.handle, _ptr(keys), _ptr(row_off), _ptr(row_k), row_k.numel(), dtype_code(keys), _ptr(ok), _ptr(oi),
        _ptr(out_off), _ptr(kk), _ptr(ki), ctypes.byref(base) if base is not None else None, ctypes.byref(best),
        _stream_ptr(stream))
    _check(st, "topk_tune_batched")
    return best


def topk_debug_wait_timeout(ctx: Context, limit_us: int, stream=None):
    """Enqueues a bounded wait that expires; topk_status_sync then reports
    TOPK_ETIMEOUT (see include/topk.h)."""
    _check(load_library().topk_debug_wait_timeout(ctx.handle, int(limit_us), _stream_ptr(stream)),
           "topk_debug_wait_timeout")


def topk_tuning_save(ctx: Context, path: str):
    _check(load_library().topk_tuning_save(ctx.handle, os.fsencode(path)), "topk_tuning_save")


def topk_tuning_load(ctx: Context, path: str):
    _check(load_library().topk_tuning_load(ctx.handle, os.fsencode(path)), "topk_tuning_load")


class Server:
    """topk_serve_*: requests submitted without blocking, admitted under an HBM
    budget, small ones batched as they arrive, run concurrently on slots."""

    def __init__(self, device: int = 0, hbm_budget: int = 64 << 30, max_slots: int = 8):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.topk_serve_create(ctypes.byref(h), int(device), int(hbm_budget), int(max_slots)),
               "topk_serve_create")
        self.handle = h
        self._keep = {}

    def now_ns(self) -> int:
        return load_library().topk_serve_now_ns(self.handle)

    def submit(self, keys, k: int, out, arrival_ns: int = 0) -> int:
        """Queues topk_select(keys, k) into ``out`` (the four output tensors of
        topk_select).  Returns the ticket; raises TopkError on rejection."""
        ok, oi, kk, ki = out
        req = topk_request(keys.data_ptr(), keys.numel(), int(k), dtype_code(keys), ok.data_ptr(),
                           oi.data_ptr(), kk.data_ptr(), ki.data_ptr(), int(arrival_ns))
        t = ctypes.c_uint64()
        _check(load_library().topk_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)),
               "topk_serve_submit")
        self._keep[t.value] = (keys, out)  # buffers must outlive the request
        return t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(load_library().topk_serve_poll(self.handle, int(ticket), ctypes.byref(d)), "topk_serve_poll")
        return bool(d.value)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        """Final status of the request (TOPK_ETIMEOUT if still running)."""
        st = load_library().topk_serve_wait(self.handle, int(ticket), int(timeout_s * 1e9))
        if st != TOPK_ETIMEOUT:
            self._keep.pop(int(ticket), None)
        return st

    def replay(self, reqs, done_before, want_lags: bool = True):
        """topk_serve_replay over a numpy array of topk_request records
        (dtype ``np.dtype(topk_request)``) and an int64 array ``done_before``.
        The caller keeps every input and output buffer alive until the
        requests finish.  Returns (tickets, lags_ns) as numpy uint64 arrays."""
        import numpy as np
        count = len(reqs)
        reqs = np.ascontiguousarray(reqs)
        done_before = np.ascontiguousarray(done_before, dtype=np.int64)
        tickets = np.zeros(count, np.uint64)
        lags = np.zeros(count, np.uint64) if want_lags else None
        _check(load_library().topk_serve_replay(
            self.handle, reqs.ctypes.data_as(ctypes.c_void_p), done_before.ctypes.data_as(ctypes.c_void_p),
            count, tickets.ctypes.data_as(ctypes.c_void_p),
            lags.ctypes.data_as(ctypes.c_void_p) if lags is not None else None), "topk_serve_replay")
        return tickets, lags

    def stats(self) -> dict:
        r = topk_serve_report()
        _check(load_library().topk_serve_stats(self.handle, ctypes.byref(r)), "topk_serve_stats")
        return {f: getattr(r, f) for f, _ in topk_serve_report._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load_library().topk_serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_MAX_N = 1 << 22


def topk_select_noalloc(keys, k: int, stream=None, out=None, status=None):
    """topk_select without any allocation inside the library (scratch in a
    fixed device array; n <= 2^22).  For callers that cannot allocate at the
    point of the call; ``out`` and ``status`` (one uint32 CUDA word) must then
    be provided by the caller, otherwise they are allocated here.  Runs on
    ``keys``' device (on ``stream``, else that device's current stream).
    Returns the four outputs; the call does not wait."""
    torch = _torch()
    if keys.dim() != 1 or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous 1-D CUDA tensor")
    with torch.cuda.device(keys.device):
        if out is None:
            kk = max(int(k), 1)
            out = (torch.empty(kk, dtype=keys.dtype, device=keys.device),
                   torch.empty(kk, dtype=torch.uint32, device=keys.device),
                   torch.empty(1, dtype=keys.dtype, device=keys.device),
                   torch.empty(1, dtype=torch.uint32, device=keys.device))
        ok, oi, kk_, ki = out
        st = load_library().topk_select_noalloc(
            _ptr(keys), keys.numel(), int(k), dtype_code(keys), _ptr(ok), _ptr(oi), _ptr(kk_), _ptr(ki),
            _ptr(status) if status is not None else None,
            _stream_ptr(stream if stream is not None else torch.cuda.current_stream(keys.device)))
    _check(st, "topk_select_noalloc")
    return out


def topk_debug_philox(c, key, count: int):
    """Philox4x32-10 outputs for counters c0+i (i < count), as a uint32 tensor."""
    torch = _torch()
    out = torch.empty(4 * count, dtype=torch.uint32, device="cuda")
    _check(load_library().topk_debug_philox(c[0], c[1], c[2], c[3], key[0], key[1], _ptr(out), count),
           "topk_debug_philox")
    return out

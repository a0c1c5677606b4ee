"""The C ABI library builds, loads and exports every symbol the headers declare
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(topk_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1502_03942_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("topk_select", "topk_select_sorted_runs", "topk_select_batched",
                     "topk_status_sync", "topk_ctx_create", "topk_ctx_destroy"):
        assert required in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_argument_errors_enqueue_nothing(lib):
    """Argument checks run on the host before any device work."""
    lib.topk_select.restype = ctypes.c_int
    lib.topk_select.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_uint64] * 2 + [ctypes.c_int] + \
        [ctypes.c_void_p] * 6
    # null context
    assert lib.topk_select(None, 16, 10, 1, 0, 16, 16, 16, 16, None, None) == 1
    lib.topk_status_string.restype = ctypes.c_char_p
    assert lib.topk_status_string(1) == b"invalid argument"


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1502_03942_gb300 as tk
    saved = tk._lib
    tk._lib = None
    try:
        with pytest.raises(RuntimeError):
            tk.load_library(str(tmp_path / "missing.so"))
    finally:
        tk._lib = saved

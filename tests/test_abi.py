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


def test_struct_layouts_match_binding(tmp_path):
    """The binding's ctypes structs have the header's sizes and offsets
    (a plain C program compiled against include/topk.h prints them)."""
    import subprocess
    import paper_1502_03942_gb300 as tk
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "topk.h"\n'
                   "int main(void) {\n"
                   '  printf("%zu %zu %zu\\n", sizeof(topk_params), offsetof(topk_params, flags),'
                   " offsetof(topk_params, block_threads));\n"
                   '  printf("%zu %zu\\n", sizeof(topk_stats), offsetof(topk_stats, sample_kept));\n'
                   '  printf("%zu %zu\\n", sizeof(topk_request), offsetof(topk_request, arrival_ns));\n'
                   '  printf("%zu %zu\\n", sizeof(topk_serve_report), offsetof(topk_serve_report, budget_waits));\n'
                   '  printf("%zu %zu %zu\\n", sizeof(topk_freq_params), offsetof(topk_freq_params, seed),'
                   " offsetof(topk_freq_params, max_distinct));\n"
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [list(map(int, line.split())) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                                   check=True).stdout.splitlines()]
    assert got[0] == [ctypes.sizeof(tk.topk_params), tk.topk_params.flags.offset, tk.topk_params.block_threads.offset]
    assert got[1] == [ctypes.sizeof(tk.topk_stats), tk.topk_stats.sample_kept.offset]
    assert got[2] == [ctypes.sizeof(tk.topk_request), tk.topk_request.arrival_ns.offset]
    assert got[3] == [ctypes.sizeof(tk.topk_serve_report), tk.topk_serve_report.budget_waits.offset]
    assert got[4] == [ctypes.sizeof(tk.topk_freq_params), tk.topk_freq_params.seed.offset,
                      tk.topk_freq_params.max_distinct.offset]


def test_tuning_calls_reject_bad_arguments(lib):
    lib.topk_tuning_save.restype = ctypes.c_int
    lib.topk_tuning_load.restype = ctypes.c_int
    lib.topk_tuning_save.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    lib.topk_tuning_load.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    assert lib.topk_tuning_save(None, b"/tmp/x") == 1
    assert lib.topk_tuning_load(None, b"/tmp/x") == 1

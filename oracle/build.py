"""Compiles the C oracle into a shared library next to its source.

Test infrastructure: builds the checker only.  Plain gcc, no CUDA, no flags that
depend on the host CPU, so the same source builds on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB_PATH = os.path.join(HERE, "liboracle.so")
CFLAGS = ["-O2", "-std=c99", "-Wall", "-Wextra", "-fPIC", "-shared"]


def compile_source(src: str, out: str) -> str:
    """gcc one oracle source file into a shared library at ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-I", HERE, src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    fresh = os.path.exists(LIB_PATH) and all(
        os.path.getmtime(LIB_PATH) >= os.path.getmtime(os.path.join(HERE, f))
        for f in ("oracle.c", "oracle.h"))
    if force or not fresh:
        compile_source(SRC, LIB_PATH)
    build_baselines(force)
    return LIB_PATH


BASELINES_SRC = os.path.join(HERE, "cpu_baselines.cpp")
BASELINES_LIB = os.path.join(HERE, "libcpu_baselines.so")


def build_baselines(force: bool = False) -> str:
    """The benchmark's timed CPU baselines (threaded sort-and-take, one-core
    nth_element): g++, no host-specific flags."""
    fresh = os.path.exists(BASELINES_LIB) and \
        os.path.getmtime(BASELINES_LIB) >= os.path.getmtime(BASELINES_SRC)
    if force or not fresh:
        tmp = BASELINES_LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-fPIC", "-shared", "-pthread",
                        BASELINES_SRC, "-o", tmp], check=True)
        os.replace(tmp, BASELINES_LIB)
    return BASELINES_LIB


if __name__ == "__main__":
    print(build(force=True))

"""Seeded synthetic inputs for the selection workloads.

This module only draws input data; it holds none of the selection arithmetic.
The tests, the smoke check and the benchmark take their inputs from here, and
the same bytes go to the CUDA path and to the CPU oracle.

Host generators use numpy's Philox bit generator.  Device generators (used only
by the benchmark at full size, where host generation would take minutes) follow
the same recipes with torch's CUDA generator; their bytes differ from the host
ones, and every check on them runs on the bytes actually generated.

Recipes (the paper's own experiments use synthetic Zipf data, Section 10.1):
  uniform_u32 : u32 uniform on [0, 2^32).
  uniform_f32 : U(0,1) with a uniform 24-bit mantissa: (u32 >> 8) * 2^-24.
  normal_f32  : N(0, sigma^2) by the Box-Muller transform in float64, then
                rounded to float32.
  zipf        : ranks r in 1..support with P(r) proportional to r^-s, drawn by
                inverting the cumulative distribution in float64; the key is
                the rank itself (f32 value r; u32 value r; bf16 bit pattern
                0x3F80 + r, which is increasing in r and distinct for
                r < 0x4000).
  sorted_runs : p runs, run length floor(2^U(lo, hi)), u64 uniform keys, each
                run sorted ascending.
  batched     : rows of length floor(2^U(lo, hi)), N(0, 3^2) f32 keys,
                k uniform on 1..kmax (clamped to the row length).
  objects     : inputs of the top-k most frequent objects (Section 10.2):
                Zipf ranks with s = 1 over 2^20 values (the most frequent
                object j times as frequent as the one of rank j), or the
                negative binomial distribution with r = 1000, p = 0.05; the
                object is the value times 0x9E3779B1 mod 2^32 (a bijection,
                so object order is unrelated to frequency).
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def uniform_u32(n: int, seed: int) -> np.ndarray:
    return rng(seed).integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)


def uniform_u64(n: int, seed: int) -> np.ndarray:
    return rng(seed).integers(0, np.iinfo(np.uint64).max, size=n, dtype=np.uint64,
                              endpoint=True)


def uniform_f32(n: int, seed: int) -> np.ndarray:
    u = uniform_u32(n, seed) >> np.uint32(8)
    return (u.astype(np.float64) * 2.0 ** -24).astype(np.float32)


def normal_f32(n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    g = rng(seed)
    u1 = 1.0 - g.random(n)            # (0, 1]: log is finite
    u2 = g.random(n)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return (sigma * z).astype(np.float32)


def zipf_cdf(s: float = 1.2, support: int = 10_000) -> np.ndarray:
    w = np.arange(1, support + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_ranks(n: int, seed: int, s: float = 1.2, support: int = 10_000) -> np.ndarray:
    cdf = zipf_cdf(s, support)
    u = rng(seed).random(n)
    r = np.searchsorted(cdf, u, side="right") + 1
    return np.minimum(r, support).astype(np.uint32)


def zipf_f32(n: int, seed: int, s: float = 1.2, support: int = 10_000) -> np.ndarray:
    return zipf_ranks(n, seed, s, support).astype(np.float32)


def zipf_u32(n: int, seed: int, s: float = 1.2, support: int = 10_000) -> np.ndarray:
    return zipf_ranks(n, seed, s, support)


def zipf_bf16_bits(n: int, seed: int, s: float = 1.2, support: int = 10_000) -> np.ndarray:
    return (np.uint32(0x3F80) + zipf_ranks(n, seed, s, support)).astype(np.uint16)


def f32_dataset(name: str, n: int, seed: int) -> np.ndarray:
    if name == "uniform":
        return uniform_f32(n, seed)
    if name == "normal":
        return normal_f32(n, seed)
    if name == "zipf":
        return zipf_f32(n, seed)
    raise ValueError(name)


def sorted_runs(p: int, lo: float, hi: float, seed: int):
    """(keys u64 concatenated, run_off[p+1])."""
    g = rng(seed)
    lens = np.floor(2.0 ** g.uniform(lo, hi, size=p)).astype(np.uint64)
    off = np.zeros(p + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    keys = g.integers(0, np.iinfo(np.uint64).max, size=int(off[-1]), dtype=np.uint64,
                      endpoint=True)
    for r in range(p):
        a, b = int(off[r]), int(off[r + 1])
        keys[a:b].sort()
    return keys, off


def batched_rows(rows: int, lo: float, hi: float, kmax: int, seed: int,
                 sigma: float = 3.0):
    """(keys f32 concatenated, row_off[rows+1], row_k[rows])."""
    g = rng(seed)
    lens = np.floor(2.0 ** g.uniform(lo, hi, size=rows)).astype(np.uint64)
    off = np.zeros(rows + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    ks = g.integers(1, kmax, size=rows, endpoint=True).astype(np.uint64)
    ks = np.minimum(ks, lens).astype(np.uint32)
    keys = normal_f32(int(off[-1]), seed + 1, sigma)
    return keys, off, ks


OBJECT_SCRAMBLE = 0x9E3779B1


def zipf_objects(n: int, seed: int, s: float = 1.0, support: int = 1 << 20) -> np.ndarray:
    r = zipf_ranks(n, seed, s, support).astype(np.uint64)
    return ((r * OBJECT_SCRAMBLE) & 0xFFFFFFFF).astype(np.uint32)


def negbin_objects(n: int, seed: int, r: int = 1000, p: float = 0.05) -> np.ndarray:
    v = rng(seed).negative_binomial(r, p, size=n).astype(np.uint64)
    return ((v * OBJECT_SCRAMBLE) & 0xFFFFFFFF).astype(np.uint32)


# ---------------------------------------------------------------- device side

def device_zipf_objects(n: int, seed: int, s: float = 1.0, support: int = 1 << 20, device="cuda"):
    """zipf_objects drawn on the device with torch (benchmark inputs)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    cdf = torch.from_numpy(zipf_cdf(s, support)).to(device)
    out = torch.empty(n, dtype=torch.int32, device=device)
    step = 1 << 26
    for a in range(0, n, step):
        m = min(step, n - a)
        u = torch.rand(m, generator=g, device=device, dtype=torch.float64)
        r = torch.clamp(torch.searchsorted(cdf, u, right=True) + 1, max=support).to(torch.int64)
        o = (r * OBJECT_SCRAMBLE) & 0xFFFFFFFF
        out[a:a + m] = torch.where(o >= (1 << 31), o - (1 << 32), o).to(torch.int32)
    return out.view(torch.uint32)

def device_f32_dataset(name: str, n: int, seed: int, device="cuda"):
    """Same recipes drawn on the device with torch (benchmark inputs)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    if name == "uniform":
        u = torch.randint(0, 1 << 24, (n,), generator=g, device=device, dtype=torch.int32)
        return u.to(torch.float32) * (2.0 ** -24)
    if name == "normal":
        out = torch.empty(n, dtype=torch.float32, device=device)
        step = 1 << 26
        for a in range(0, n, step):
            m = min(step, n - a)
            u1 = 1.0 - torch.rand(m, generator=g, device=device, dtype=torch.float64)
            u2 = torch.rand(m, generator=g, device=device, dtype=torch.float64)
            z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
            out[a:a + m] = z.to(torch.float32)
        return out
    if name == "zipf":
        cdf = torch.from_numpy(zipf_cdf()).to(device)
        out = torch.empty(n, dtype=torch.float32, device=device)
        step = 1 << 26
        for a in range(0, n, step):
            m = min(step, n - a)
            u = torch.rand(m, generator=g, device=device, dtype=torch.float64)
            r = torch.searchsorted(cdf, u, right=True) + 1
            out[a:a + m] = torch.clamp(r, max=cdf.numel()).to(torch.float32)
        return out
    raise ValueError(name)

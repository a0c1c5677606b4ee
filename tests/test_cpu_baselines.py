"""The benchmark's CPU baselines and host-side timing helpers (CPU only).

The threaded sort-and-take and the one-core nth_element of oracle/cpu_baselines
must return exactly the oracle's answer (they are timed as alternatives to the
GPU path, so a wrong answer would make their times meaningless)."""
import numpy as np
import pytest

import oracle
from paper_1502_03942_gb300 import workloads as wl


@pytest.mark.parametrize("ds", ["uniform", "normal", "zipf"])
def test_cpu_baselines_match_oracle(ds):
    orc = oracle.default()
    cb = oracle.cpu_baselines()
    x = wl.f32_dataset(ds, 300_007, seed=2).view(np.uint32)
    work = np.empty(x.size, np.uint64)
    sel = np.empty(x.size, np.uint32)
    for threads in (1, 3, 8):
        cb.sort_chunks(x, threads, work)
        for k in (1, 1024, x.size // 2, x.size):
            kth = cb.take_k(work, threads, k, sel)
            want_sel, want_kth = orc.select(x, "f32", k)
            assert kth == want_kth
            assert np.array_equal(np.sort(sel[:k]), np.sort(want_sel))
    w2 = np.empty(x.size, np.uint64)
    for k in (1, 1024, x.size // 2, x.size):
        assert cb.nth_element(x, k, w2) == orc.select(x, "f32", k)[1]


def test_time_oracle_uses_every_core():
    import bench
    info = bench.host_info()
    assert info["cores"] >= 1 and info["nproc"] >= 1
    keys = {ds: wl.f32_dataset(ds, 1 << 18, seed=2).view(np.uint32) for ds in bench.DATASETS}
    r = bench.time_oracle(keys, budget_s=0.5, slice_n=1 << 16)
    assert r["cores"] == info["cores"] and r["value"] > 0 and r["kind"] == "oracle"

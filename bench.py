"""Benchmark: single large selection on one GB300 (and N independent replicas).

Workload (one "step"): n = 2^28 float32 keys in HBM, three datasets
(U(0,1), N(0,1), Zipf s = 1.2 over 10^4 values), k in {1, 1024, 2^20, n/2}:
twelve calls of topk_select, each selecting the k smallest (index tie-break)
and the rank-k key.  Every input is 1 GiB, larger than the 129 MB L2, so no
flush is needed between calls.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead
(test infrastructure, single thread) on a bounded sample of the same workload.
Under torchrun every rank runs its own replica on its own GPU (the selection
does not shard across GPUs here: "replicas only"), timings are max-reduced.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1 << 28
KS = (1, 1024, 1 << 20, N // 2)
DATASETS = ("uniform", "normal", "zipf")
METRIC = "keys/s and HBM GB/s (% of peak) per selection; batched & served vs per-call"
WORKLOAD = "single large selection: n=2^28 f32 x {uniform, normal, zipf} x k in {1, 1024, 2^20, n/2}, p=148"


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# the sources the first-level pass is compiled from (its traffic record is
# valid while these are unchanged)
FIRST_PASS_SOURCES = ("common.cuh", "select.cu", "select_block.cuh", "select_core.cuh", "select_impl.cuh")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1502_03942_gb300", "csrc")
    for f in FIRST_PASS_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic():
    """ncu DRAM bytes per first-level pass launch, if taken on the current source."""
    path = os.path.join(ROOT, "profiles", "first_pass_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_hash") != source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled while the timed
    region runs: NVML read directly every 5 ms (read-only queries), else
    nvidia-smi at its 200 ms minimum period."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    SMI_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                  "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.device_index = device_index
        self.rows = []          # (sm_mhz, max_mhz, reasons set)
        self.source = None
        self._stop = threading.Event()
        self.proc = None
        self.thread = None

    def _nvml_handle(self):
        import ctypes
        import torch
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit")
        pr = torch.cuda.get_device_properties(self.device_index)
        bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0:
            raise RuntimeError("nvml handle")
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons

    def _poll_nvml(self, lib, h, reasons):
        import ctypes
        mhz, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    reasons(h, ctypes.byref(rs)) == 0):
                self.rows.append((float(mhz.value), float(mx.value),
                                  {n for b, n in self.REASONS.items() if rs.value & b}))
            self._stop.wait(0.005)

    def _read_smi(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.proc.stdout:
            p = [x.strip() for x in line.split(",")]
            if len(p) == 7 and p[0].replace(".", "").isdigit() and p[1].replace(".", "").isdigit():
                self.rows.append((float(p[0]), float(p[1]),
                                  {names[i] for i in range(4) if p[3 + i].lower() == "active"}))

    def __enter__(self):
        try:
            lib, h, reasons = self._nvml_handle()
            self.thread = threading.Thread(target=self._poll_nvml, args=(lib, h, reasons), daemon=True)
            self.source = "nvml 5 ms"
        except Exception:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.device_index), f"--query-gpu={self.SMI_FIELDS}",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.thread = threading.Thread(target=self._read_smi, daemon=True)
                self.source = "nvidia-smi 200 ms"
            except Exception:
                self.thread = None
        if self.thread is not None:
            self.thread.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                "sm_max_mhz": max(r[1] for r in self.rows),
                "reasons": sorted(set().union(*(r[2] for r in self.rows))),
                "samples": len(self.rows), "source": self.source}


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of every rank's x (a float): the whole job ends when the
    slowest rank does.  Without a process group, x itself."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes(k):
    """One read of the input plus the output pairs (key + u32 index)."""
    return N * 4 + k * 8


# ------------------------------------------------------------------ oracle

def host_info():
    """Host CPU: usable cores and model name (for the CPU baselines)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cores": cores, "cpu_model": model or "unknown",
            "arch": platform.machine()}


class numa_local:
    """Within the block, the process runs on the CPUs of the GPU's own NUMA
    node (from sysfs), so that pinned host buffers allocated there are local
    to the GPU; the previous CPU set is restored afterwards.  Does nothing
    where sysfs gives no node."""

    def __init__(self, device_index):
        self.device_index = device_index
        self.saved = None

    def _cpus(self):
        import torch
        pr = torch.cuda.get_device_properties(self.device_index)
        bus = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        node = int(open(f"/sys/bus/pci/devices/{bus}/numa_node").read().strip())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return cpus or None

    def __enter__(self):
        try:
            cpus = self._cpus()
            if cpus:
                self.saved = os.sched_getaffinity(0)
                os.sched_setaffinity(0, cpus)
        except Exception:
            self.saved = None
        return self

    def __exit__(self, *exc):
        if self.saved is not None:
            os.sched_setaffinity(0, self.saved)


def time_oracle(host_keys, budget_s=20.0, slice_n=1 << 22, threads=None):
    """The CPU oracle as it stands (one full qsort of all pairs per selection)
    on every host core: each thread runs oracle selections on its own
    slice_n-key slice of one dataset's input (same bytes as the GPU arm),
    every k of the workload scaled to the slice, until the budget is spent.
    ctypes releases the GIL, so the threads' sorts run in parallel."""
    import concurrent.futures as cf
    import numpy as np
    import oracle
    orc = oracle.default()
    info = host_info()
    threads = threads or info["cores"]
    items = []
    for rep in range(64):
        for ds in DATASETS:
            x = host_keys[ds]
            for k in KS:
                kk = max(1, min(slice_n, k * slice_n // N if k > 1024 else k))
                for t in range(threads):
                    j = (rep * threads + t) % (x.size // slice_n)
                    items.append((ds, j, kk))
    t0 = time.perf_counter()
    done = [0]

    def work(item):
        ds, j, kk = item
        if time.perf_counter() - t0 > budget_s:
            return 0
        orc.select(host_keys[ds][j * slice_n:(j + 1) * slice_n], "f32", kk)
        return slice_n

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        keys = sum(ex.map(work, items))
    wall = time.perf_counter() - t0
    calls = keys // slice_n
    return {"value": keys / wall, "unit": "keys/s", "cores": threads, "kind": "oracle",
            "cpu_model": info["cpu_model"], "nproc": info["nproc"], "arch": info["arch"],
            "sample": f"{calls} oracle selections (full qsort of all pairs each), {threads} at a time, on "
                      f"{slice_n}-key slices of the workload's own inputs (k scaled by slice/n above "
                      f"1024), {wall:.1f} s wall"}


def time_cpu_selection(host_keys):
    """SURVEY-style CPU baselines on the full 2^28-key inputs: sort-and-take
    on every host core (per-thread std::sort of one chunk, then a merge of
    the chunks up to rank k), and std::nth_element on one core (normal
    dataset).  Per selection: its own sort plus its merge."""
    import numpy as np
    import oracle
    cb = oracle.cpu_baselines()
    info = host_info()
    th = info["cores"]
    work = np.empty(N, np.uint64)
    sel = np.empty(N // 2, np.uint32)
    per, total = {}, 0.0
    for ds in DATASETS:
        t0 = time.perf_counter()
        cb.sort_chunks(host_keys[ds], th, work)
        t_sort = time.perf_counter() - t0
        for k in KS:
            t0 = time.perf_counter()
            cb.take_k(work, th, k, sel)
            t = t_sort + time.perf_counter() - t0
            per[f"{ds}/k={k}"] = {"ms": 1e3 * t}
            total += t
    del work
    nth, t_nth = {}, 0.0
    w1 = np.empty(N, np.uint64)
    for k in KS:
        t0 = time.perf_counter()
        cb.nth_element(host_keys["normal"], k, w1)
        t = time.perf_counter() - t0
        nth[f"normal/k={k}"] = {"ms": 1e3 * t}
        t_nth += t
    return {"sort_take": {"value": len(DATASETS) * len(KS) * N / total, "unit": "keys/s", "cores": th,
                          "kind": "sort-and-take: per-thread std::sort of n/cores pairs + heap merge to rank k",
                          "sample": "the full 2^28-key inputs of all 12 selections, one sort each",
                          "per_case": per},
            "nth_element": {"value": len(KS) * N / t_nth, "unit": "keys/s", "cores": 1,
                            "kind": "std::nth_element on (key image, position) pairs, one core",
                            "sample": "the full 2^28-key normal input, k in {1, 1024, 2^20, n/2}",
                            "per_case": nth},
            "cpu_model": info["cpu_model"], "nproc": info["nproc"], "arch": info["arch"]}


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    import numpy as np
    from paper_1502_03942_gb300 import workloads as wl
    info = host_info()
    slice_n = 1 << 22
    host_keys = {ds: wl.f32_dataset(ds, slice_n * info["cores"], seed=2).view(np.uint32) for ds in DATASETS}
    base = {"metric": METRIC, "unit": "keys/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "keys": "f32",
                       "arm": f"CPU oracle on {info['cores']} host cores ({info['cpu_model']})"}}
    budget = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        time_oracle(host_keys, budget_s=budget / 4, slice_n=1 << 20)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(time_oracle(host_keys, budget_s=budget, slice_n=slice_n))
    wall = time.perf_counter() - t0
    v = statistics.median(r["value"] for r in vals)
    line = dict(base)
    cb = dict(vals[-1])
    cb["value"] = v
    line.update({"value": v, "ms_per_step": 1e3 * wall / max(1, args.steps), "cpu_baseline": cb,
                 "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0}})
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------- batched and served extras

def measure_plain(tk, wl, torch, ctx):
    """n = 2^20 u32 uniform keys (seed 1), k = 1000, p = 64: the input is 4 MiB
    and stays in L2, so the call is timed both warm (back to back) and with
    L2 flushed before every call (a 256 MiB buffer written in between, outside
    the call's own events)."""
    import numpy as np
    n, k = 1 << 20, 1000
    x = torch.from_numpy(wl.uniform_u32(n, 1).view(np.int32)).cuda().view(torch.uint32)
    p = tk.make_params(partitions=64)
    out = tk.topk_select(ctx, x, k, params=p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    reps = 50
    warm, cold = [], []
    for _ in range(5):
        tk.topk_select(ctx, x, k, params=p, out=out, check=False)
    for r in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tk.topk_select(ctx, x, k, params=p, out=out, check=False)
        e1.record()
        torch.cuda.synchronize()
        warm.append(e0.elapsed_time(e1))
        flush.fill_(r & 0xFF)
        e0.record()
        tk.topk_select(ctx, x, k, params=p, out=out, check=False)
        e1.record()
        torch.cuda.synchronize()
        cold.append(e0.elapsed_time(e1))
    st = ctx.sync()
    wm, cm = statistics.median(warm), statistics.median(cold)
    return {"workload": "plain selection: n=2^20 u32 uniform (seed 1), k=1000, p=64", "status": st,
            "warm_ms": wm, "l2_flushed_ms": cm, "warm_keys_per_s": n / (wm / 1e3),
            "l2_flushed_keys_per_s": n / (cm / 1e3)}


def measure_batched(tk, wl, torch, ctx):
    """4096 rows of N(0,3) f32, lengths 2^U(10,18), k in 1..1024: one
    graph-captured persistent launch against one topk_select per row."""
    import numpy as np
    keys, off, ks = wl.batched_rows(4096, 10, 18, 1024, seed=4)
    d_keys = torch.from_numpy(keys).cuda()
    d_off = torch.from_numpy(off.view(np.int64)).cuda().view(torch.uint64)
    d_k = torch.from_numpy(ks.view(np.int32)).cuda().view(torch.uint32)
    oo = np.zeros(4097, np.uint64)
    oo[1:] = np.cumsum(ks.astype(np.uint64))
    d_oo = torch.from_numpy(oo.view(np.int64)).cuda().view(torch.uint64)
    total = int(oo[-1])
    out = (torch.empty(total, dtype=torch.float32, device="cuda"),
           torch.empty(total, dtype=torch.uint32, device="cuda"),
           torch.empty(4096, dtype=torch.float32, device="cuda"),
           torch.empty(4096, dtype=torch.uint32, device="cuda"))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def graph_ms(params):
        for _ in range(3):
            tk.topk_select_batched(ctx, d_keys, d_off, d_k, params=params, out=out, out_off=d_oo, check=False)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            tk.topk_select_batched(ctx, d_keys, d_off, d_k, params=params, out=out, out_off=d_oo, check=False)
        g.replay()
        torch.cuda.synchronize()
        reps = 10
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_default = graph_ms(tk.make_params(block_threads=1024, sample_size=2048))
    best = tk.topk_tune_batched(ctx, d_keys, d_off, d_k, out, d_oo)
    t_batched = graph_ms(None)  # the context's tuned choice
    # one launch sequence per row, same data and outputs
    rows = [(int(off[i]), int(off[i + 1]), int(ks[i]), int(oo[i])) for i in range(4096)]
    views = [(d_keys[a:b], k, (out[0][o:o + k], out[1][o:o + k], out[2][i:i + 1], out[3][i:i + 1]))
             for i, (a, b, k, o) in enumerate(rows)]
    for v, k, o in views[:64]:
        tk.topk_select(ctx, v, k, out=o, check=False)
    torch.cuda.synchronize()
    e0.record()
    for v, k, o in views:
        tk.topk_select(ctx, v, k, out=o, check=False)
    e1.record()
    torch.cuda.synchronize()
    t_calls = e0.elapsed_time(e1)
    st = ctx.sync()
    n_keys = int(off[-1])
    return {"workload": "4096 rows f32 N(0,3), n=2^U(10,18), k=U[1,1024], one graph-captured launch",
            "status": st, "batched_ms": t_batched, "per_call_ms": t_calls,
            "tuned": {"block_threads": best.block_threads, "sample_size": best.sample_size,
                      "finish_threshold": best.finish_threshold},
            "untuned_ms": t_default,
            "speedup_vs_per_call": t_calls / t_batched, "keys_per_s": n_keys / (t_batched / 1e3),
            "algorithmic_GBps": (n_keys * 4 + total * 8) / (t_batched / 1e3) / 1e9}


def measure_sorted_runs(tk, wl, torch, ctx):
    """1024 sorted u64 runs of 2^U(10,20) keys: one multisequence selection
    per k in {1, 2^16, total/2}."""
    import numpy as np
    keys, off = wl.sorted_runs(1024, 10, 20, seed=3)
    d_keys = torch.from_numpy(keys.view(np.int64)).cuda().view(torch.uint64)
    d_off = torch.from_numpy(off.view(np.int64)).cuda().view(torch.uint64)
    total = int(off[-1])
    res = {"workload": "1024 sorted u64 runs, lengths 2^U(10,20), k in {1, 2^16, total/2}; "
                       "flexible k in [k, 1.1 k] for k in {2^16, total/2}", "total": total}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, k in (("k1", 1), ("k65536", 1 << 16), ("half", total // 2)):
        out = tk.topk_select_sorted_runs(ctx, d_keys, d_off, k)
        for _ in range(2):
            tk.topk_select_sorted_runs(ctx, d_keys, d_off, k, out=out, check=False)
        torch.cuda.synchronize()
        reps = 10
        e0.record()
        for _ in range(reps):
            tk.topk_select_sorted_runs(ctx, d_keys, d_off, k, out=out, check=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tk.topk_select_sorted_runs(ctx, d_keys, d_off, k, out=out, check=True)
        stt = ctx.last_stats()
        res[name] = {"ms": ms, "keys_per_s": total / (ms / 1e3), "rounds_grid": stt["levels_grid"],
                     "rounds_block": stt["levels_block"]}
    # flexible k (amsSelect): any k within 10% above the same targets
    for name, kmin in (("flex_k65536", 1 << 16), ("flex_half", total // 2)):
        kmax = kmin + kmin // 10
        out = tk.topk_select_sorted_runs_flexible(ctx, d_keys, d_off, kmin, kmax)
        for _ in range(2):
            tk.topk_select_sorted_runs_flexible(ctx, d_keys, d_off, kmin, kmax, out=out, check=False)
        torch.cuda.synchronize()
        reps = 10
        e0.record()
        for _ in range(reps):
            tk.topk_select_sorted_runs_flexible(ctx, d_keys, d_off, kmin, kmax, out=out, check=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tk.topk_select_sorted_runs_flexible(ctx, d_keys, d_off, kmin, kmax, out=out, check=True)
        stt = ctx.last_stats()
        res[name] = {"ms": ms, "keys_per_s": total / (ms / 1e3), "kmin": kmin, "kmax": kmax,
                     "k": int(out[4].cpu().view(torch.int64)[0]), "rounds_grid": stt["levels_grid"],
                     "rounds_block": stt["levels_block"]}
    # bulk deleteMin* (Section 5): consecutive pops from cursors at 0
    d_cur = torch.zeros(1024, dtype=torch.uint64, device="cuda")
    for name, kmin, kmax in (("delete_min_k65536", 1 << 16, None), ("delete_min_flex_k65536", 1 << 16,
                                                                    (1 << 16) + (1 << 16) // 10)):
        def pop():
            if kmax is None:
                return tk.topk_runs_delete_min(ctx, d_keys, d_off, d_cur, kmin, check=False)
            return tk.topk_runs_delete_min_flexible(ctx, d_keys, d_off, d_cur, kmin, kmax, check=False)
        d_cur.zero_()
        for _ in range(2):
            pop()
        d_cur.zero_()
        torch.cuda.synchronize()
        reps = 10
        e0.record()
        for _ in range(reps):
            pop()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        deleted = int(d_cur.view(torch.int64).sum().item())
        res[name] = {"ms_per_pop": ms, "pops": reps, "deleted": deleted,
                     "deleted_per_s": deleted / (reps * ms / 1e3)}
    res["workload"] += "; deleteMin* pops of 2^16 (and flexible [2^16, 1.1*2^16]) from empty cursors"
    res["status"] = ctx.sync()
    return res


def measure_frequent(tk, wl, torch, ctx, peak_gbs):
    """Top-k most frequent objects (Section 7, experiments of Section 10.2):
    n = 2^28 Zipf objects (s = 1, 2^20 values), k = 32, eps = 3e-4,
    delta = 1e-4; Algorithm EC at its planned rate, Algorithm PAC at its
    planned rate (1 on one GPU: every object counted) and at EC's rate."""
    n = 1 << 28
    d_obj = wl.device_zipf_objects(n, seed=2024)
    res = {"workload": "n=2^28 u32 objects, Zipf s=1 over 2^20 values, k=32, eps=3e-4, delta=1e-4"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ec = tk.make_freq_params(32, algorithm=tk.TOPK_FREQ_EC, epsilon=3e-4, delta=1e-4, seed=3)
    ec_rho, ec_kstar = tk.topk_frequent_plan(n, ec)
    cases = (("ec", ec, 2),
             ("pac", tk.make_freq_params(32, algorithm=tk.TOPK_FREQ_PAC, epsilon=3e-4, delta=1e-4, seed=3), 1),
             ("pac_at_ec_rate", tk.make_freq_params(32, algorithm=tk.TOPK_FREQ_PAC, rho=ec_rho, seed=3), 1))
    for name, fp, passes in cases:
        rho, kstar = tk.topk_frequent_plan(n, fp)
        out = tk.topk_frequent(ctx, d_obj, fp)
        for _ in range(2):
            tk.topk_frequent(ctx, d_obj, fp, out=out, check=False)
        torch.cuda.synchronize()
        reps = 5
        e0.record()
        for _ in range(reps):
            tk.topk_frequent(ctx, d_obj, fp, out=out, check=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = passes * 4 * n / (ms / 1e3) / 1e9
        res[name] = {"ms": ms, "objects_per_s": n / (ms / 1e3), "rho": rho, "kstar": kstar,
                     "sample_size": int(out[2].view(torch.int64).item()),
                     "input_passes": passes, "input_gbs": gbs, "frac_of_hbm": gbs / peak_gbs}
    res["status"] = ctx.sync()
    return res


def measure_served(tk, wl, torch, seconds=10.0, rate=20000.0, seed=5, budget=64 << 30, per_call=True):
    """Poisson arrivals at `rate`/s for `seconds`: n = 2^U(10,26), u32 or bf16,
    uniform or Zipf (s=1.2, 10^4 values), k = 2^U(0, log2(n/4)); 64 GB budget.
    Inputs come from a pool of distinct device arrays; outputs from a ring
    arena that is reused only after the request that held it completed.  The
    trace is submitted by the library's native replay at the scheduled times
    (submit_lag_p99_ms: how late the submissions were)."""
    import numpy as np
    g = np.random.Generator(np.random.Philox(seed))
    pool = []
    for i in range(48):
        n = int(2.0 ** g.uniform(10, 26))
        bf16 = bool(g.integers(0, 2))
        zipf = bool(g.integers(0, 2))
        if bf16:
            bits = wl.zipf_bf16_bits(n, 100 + i) if zipf else \
                np.random.Generator(np.random.Philox(100 + i)).integers(0, 1 << 16, size=n).astype(np.uint16)
            t = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
        else:
            bits = wl.zipf_u32(n, 100 + i) if zipf else wl.uniform_u32(n, 100 + i)
            t = torch.from_numpy(bits.view(np.int32)).cuda().view(torch.uint32)
        pool.append(t)
    count = int(rate * seconds)
    gaps = g.exponential(1.0 / rate, size=count)
    which = g.integers(0, len(pool), size=count)
    ks = []
    for i in range(count):
        n = pool[which[i]].numel()
        ks.append(max(1, min(n, int(2.0 ** g.uniform(0, np.log2(max(2.0, n / 4)))))))
    arena_bytes = 6 << 30
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def carve(v, keys, k):
        """Outputs at virtual arena offset v (monotone; physical = v mod size,
        never straddling the end).  Returns (outputs, v_start, v_end)."""
        w = keys.element_size()
        kbytes = (k * w + 15) & ~15
        need = kbytes + ((4 * k + 15) & ~15) + 64
        if v % arena_bytes + need > arena_bytes:
            v += arena_bytes - v % arena_bytes
        base = v % arena_bytes
        kk = arena[base:base + k * w].view(keys.dtype)
        ii = arena[base + kbytes: base + kbytes + 4 * k].view(torch.uint32)
        e = (base + kbytes + 4 * k + 15) & ~15
        kt = arena[e:e + w].view(keys.dtype)
        it = arena[e + 16:e + 20].view(torch.uint32)
        return (kk, ii, kt, it), v, v + need

    # the trace: each request's outputs at a virtual arena offset (monotone;
    # physical = offset mod size, never straddling the end); a request whose
    # region reuses memory waits (natively, in the replay) for every request
    # allocated more than one arena length before its end
    w_of = np.array([pool[which[i]].element_size() for i in range(count)], np.int64)
    k_arr = np.array(ks, np.int64)
    kb = (k_arr * w_of + 15) & ~15
    need = kb + ((4 * k_arr + 15) & ~15) + 64
    v0 = np.zeros(count, np.int64)
    v = 0
    for i in range(count):
        if v % arena_bytes + need[i] > arena_bytes:
            v += arena_bytes - v % arena_bytes
        v0[i] = v
        v += need[i]
    v1 = v0 + need
    done_before = np.searchsorted(v0, v1 - arena_bytes, side="left") - 1
    phys = v0 % arena_bytes
    base = arena.data_ptr()
    reqs = np.zeros(count, dtype=np.dtype(tk.topk_request))
    reqs["d_keys"] = [pool[which[i]].data_ptr() for i in range(count)]
    reqs["n"] = [pool[which[i]].numel() for i in range(count)]
    reqs["k"] = k_arr
    reqs["dtype"] = [tk.dtype_code(pool[which[i]]) for i in range(count)]
    reqs["d_out_keys"] = base + phys
    reqs["d_out_idx"] = base + phys + kb
    kth = (base + phys + kb + 4 * k_arr + 15) & ~15
    reqs["d_kth_key"] = kth
    reqs["d_kth_idx"] = kth + 16
    srv = tk.Server(0, hbm_budget=budget, max_slots=16)
    t0 = srv.now_ns() + 20_000_000
    reqs["arrival_ns"] = t0 + np.cumsum((gaps * 1e9).astype(np.int64))
    tickets, lags = srv.replay(reqs, done_before)
    tickets = [int(t) for t in tickets]
    bad = sum(1 for t in tickets if srv.wait(t) != tk.TOPK_OK)
    st = srv.stats()
    srv.close()
    offered_keys = sum(pool[which[i]].numel() for i in range(count))
    served_s = st["elapsed_s"]
    res = {"workload": f"Poisson {rate:.0f} req/s for {seconds} s, n=2^U(10,26) u32|bf16 uniform|Zipf, "
                       f"k=2^U(0,log2(n/4)), {budget / 2**20:.0f} MiB budget, 16 slots",
           "requests": count, "failed": bad + st["failed"], "p50_ms": st["p50_ns"] / 1e6,
           "p99_ms": st["p99_ns"] / 1e6, "keys_per_s": st["keys"] / served_s if served_s else None,
           "offered_keys_per_s": offered_keys / seconds, "batched_requests": st["batched_requests"],
           "batches": st["batches"], "peak_inflight_GB": st["peak_inflight_bytes"] / 1e9,
           "budget_GB": budget / 1e9, "slots_reserved_GB": st["reserved_bytes"] / 1e9,
           "budget_waits": st["budget_waits"],
           "served_s": served_s, "submit_lag_p99_ms": float(np.percentile(lags, 99)) / 1e6}
    if not per_call:
        return res
    # the same requests, one launch sequence per request, back to back
    ctx = tk.Context(0)
    outs = {}
    for i in range(min(count, 64)):
        keys, k = pool[which[i]], ks[i]
        tk.topk_select(ctx, keys, k, out=carve(0, keys, k)[0], check=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(count):
        keys, k = pool[which[i]], ks[i]
        tk.topk_select(ctx, keys, k, out=carve(0, keys, k)[0], check=False)
    e1.record()
    torch.cuda.synchronize()
    per_call_s = e0.elapsed_time(e1) / 1e3
    ctx.close()
    res.update({"per_call_keys_per_s": offered_keys / per_call_s, "per_call_s": per_call_s})
    return res


# --------------------------------------------------------------- GPU arm

def run_ours(args):
    import torch
    import paper_1502_03942_gb300 as tk
    from paper_1502_03942_gb300 import workloads as wl

    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    ctx = tk.Context(local)
    params = tk.make_params(partitions=148)
    data = {ds: wl.device_f32_dataset(ds, N, seed=2 + rank) for ds in DATASETS}
    outs = {k: (torch.empty(k, dtype=torch.float32, device="cuda"),
                torch.empty(k, dtype=torch.uint32, device="cuda"),
                torch.empty(1, dtype=torch.float32, device="cuda"),
                torch.empty(1, dtype=torch.uint32, device="cuda")) for k in KS}
    stream = torch.cuda.current_stream()

    def step():
        for ds in DATASETS:
            for k in KS:
                tk.topk_select(ctx, data[ds], k, params=params, out=outs[k], check=False, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    st = ctx.sync(stream)
    if st != 0:
        raise tk.TopkError(st, "warm-up")
    ctx.profile(True)
    ctx.profile_read(reset=True)

    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    st = ctx.sync(stream)
    if st != 0:
        raise tk.TopkError(st, "timed region")
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    ms = max_over_ranks(ms, dist, "cuda")

    # per selection: each (dataset, k) call alone between CUDA events on the
    # stream, the twelve calls interleaved, median over repetitions
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    reps = max(3, min(args.steps, 8))
    evs = []
    for _ in range(reps):
        for ds in DATASETS:
            for k in KS:
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                tk.topk_select(ctx, data[ds], k, params=params, out=outs[k], check=False, stream=stream)
                a1.record(stream)
                evs.append((ds, k, a0, a1))
    torch.cuda.synchronize()
    case_ms = {}
    for ds, k, a0, a1 in evs:
        case_ms.setdefault((ds, k), []).append(a0.elapsed_time(a1))
    per_case = {}
    for (ds, k), v in case_ms.items():
        m = statistics.median(v)
        gbs = algorithmic_bytes(k) / (m / 1e3) / 1e9
        tk.topk_select(ctx, data[ds], k, params=params, out=outs[k], check=True, stream=stream)
        stt = ctx.last_stats()
        # the first-level pass of this case alone (the library's own CUDA
        # events around it), so the rest of the call can be told apart
        ctx.profile(True)
        ctx.profile_read(reset=True)
        for _ in range(reps):
            tk.topk_select(ctx, data[ds], k, params=params, out=outs[k], check=False, stream=stream)
        torch.cuda.synchronize()
        pp = ctx.profile_read(reset=True)
        ctx.profile(False)
        fp = pp["pass_ms"] / max(1, pp["passes"])
        per_case[f"{ds}/k={k}"] = {"ms": m, "keys_per_s": N / (m / 1e3), "algorithmic_GBps": gbs,
                                   "frac_of_hbm": gbs / peak, "grid_levels": stt["levels_grid"],
                                   "first_candidates": stt["first_candidates"],
                                   "first_pass_ms": fp, "rest_ms": m - fp}

    # end to end: pinned host input -> device, select, outputs -> host.  The
    # next dataset's input is copied on its own stream while the current one
    # is selected (two device input buffers), and each dataset's outputs go
    # back on a third stream while the next dataset is selected; pinned
    # buffers are allocated from CPUs on the GPU's own NUMA node.
    e2e = None
    if True:  # every rank: the timing is max-reduced across ranks
        with numa_local(local):
            host = {ds: torch.empty(N, dtype=torch.float32, pin_memory=True) for ds in DATASETS}
            hout = {(ds, k): tuple(torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs[k])
                    for ds in DATASETS for k in KS}
        for ds in DATASETS:
            host[ds].copy_(data[ds])
        dev = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in range(2)]
        douts = {(ds, k): tuple(torch.empty_like(t) for t in outs[k]) for ds in DATASETS for k in KS}
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        h2d = 3 * N * 4
        d2h = sum(k * 8 + 8 for k in KS) * len(DATASETS)
        steps_e2e = max(1, min(args.steps, 3))

        freed = [None, None]            # selections done with input buffer b
        copied = {ds: None for ds in DATASETS}  # dataset's outputs back on the host

        def e2e_step():
            for i, ds in enumerate(DATASETS):
                b = i % 2
                buf = dev[b]
                with torch.cuda.stream(s_in):
                    if freed[b] is not None:
                        s_in.wait_event(freed[b])
                    buf.copy_(host[ds], non_blocking=True)
                    arrived = torch.cuda.Event()
                    arrived.record(s_in)
                stream.wait_event(arrived)
                if copied[ds] is not None:
                    stream.wait_event(copied[ds])
                for k in KS:
                    tk.topk_select(ctx, buf, k, params=params, out=douts[(ds, k)], check=False, stream=stream)
                freed[b] = torch.cuda.Event()
                freed[b].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(freed[b])
                    for k in KS:
                        for h, d in zip(hout[(ds, k)], douts[(ds, k)]):
                            h.copy_(d, non_blocking=True)
                    copied[ds] = torch.cuda.Event()
                    copied[ds].record(s_out)

        e2e_step()
        torch.cuda.synchronize()
        # the host link alone: one pinned 1 GiB copy to the device
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        dev[0].copy_(host[DATASETS[0]], non_blocking=True)
        l1.record(stream)
        torch.cuda.synchronize()
        link_gbs = N * 4 / (l0.elapsed_time(l1) / 1e3) / 1e9
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            e2e_step()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, dist, "cuda")
        e2e = {"value": world * steps_e2e * len(DATASETS) * len(KS) * N / t_e2e, "unit": "keys/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "h2d_GBps_achieved": steps_e2e * h2d / t_e2e / 1e9, "h2d_link_GBps": link_gbs,
               "overlap": "H2D of the next dataset and D2H of the last one's outputs run beside the selections"}
        del host, hout, dev, douts

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    per_step = len(DATASETS) * len(KS)
    keys_per_s = world * args.steps * per_step * N / (ms / 1e3)
    alg_bytes = sum(algorithmic_bytes(k) for k in KS) * len(DATASETS)
    # dominant kernel: the first-level pass that streams all n keys
    pass_ms_avg = prof["pass_ms"] / max(1, prof["passes"])
    pass_alg = sum(N * 4 + (k * 8 if k == N // 2 else 0) for k in KS) / len(KS)
    achieved = pass_alg / (pass_ms_avg / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": keys_per_s, "unit": "keys/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "keys": "f32 (order-preserving u32 image, u32 index tie-break)",
                   "global_batch": per_step, "seq_len": N, "parallelism": f"replicas{world}",
                   "l2": "inputs 1 GiB > L2, no flush",
                   "algorithmic_GBps": alg_bytes * args.steps / (ms / 1e3) / 1e9,
                   "algorithmic_frac_of_hbm": alg_bytes * args.steps / (ms / 1e3) / 1e9 / peak},
        "roofline": {"bound": "hbm", "kernel": "first-level pass (streams all n keys)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": committed_traffic(),
                     "launch_ms_avg": pass_ms_avg, "algorithmic_bytes_per_launch": pass_alg},
        "per_case": per_case,
        "per_case_min_frac": min(v["frac_of_hbm"] for v in per_case.values()),
        "gpu_launches": int(prof["launches"]),
        "clocks": clocks.summary(),
        "e2e": e2e,
    }
    if not args.no_extras:
        for key, fn in (("plain", lambda: measure_plain(tk, wl, torch, ctx)),
                        ("batched", lambda: measure_batched(tk, wl, torch, ctx)),
                        ("sorted_runs", lambda: measure_sorted_runs(tk, wl, torch, ctx)),
                        ("frequent", lambda: measure_frequent(tk, wl, torch, ctx, peak)),
                        ("served", lambda: measure_served(tk, wl, torch)),
                        ("served_pressure", lambda: measure_served(tk, wl, torch, seconds=4.0, budget=1 << 29,
                                                                   per_call=False))):
            try:
                line[key] = fn()
            except Exception as e:  # reported in the line, never hides the main metric
                line[key] = {"error": repr(e)}
    if world == 1 and not args.no_cpu_baseline:
        host_keys = {ds: data[ds].view(torch.int32).cpu().numpy().view("uint32") for ds in DATASETS}
        line["cpu_baseline"] = time_oracle(host_keys)
        line["cpu_selection"] = time_cpu_selection(host_keys)
        del host_keys
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_probe(spec):
    """One selection for profilers: DATASET:N:K[:FLAGS] (after one warm-up)."""
    import torch
    import paper_1502_03942_gb300 as tk
    from paper_1502_03942_gb300 import workloads as wl
    parts = spec.split(":")
    ds, n, k = parts[0], int(parts[1]), int(parts[2])
    flags = int(parts[3], 0) if len(parts) > 3 else 0
    ctx = tk.Context(0)
    x = wl.device_f32_dataset(ds, n, seed=2)
    p = tk.make_params(partitions=148, flags=flags)
    out = tk.topk_select(ctx, x, k, params=p)
    tk.topk_select(ctx, x, k, params=p, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"probe": spec, "stats": ctx.last_stats()}))
    return 0


def run_probe_frequent(spec):
    """Top-k most frequent objects for profilers: ALG:LOG2N (ALG ec or pac;
    Zipf objects, k = 32, eps = 3e-4, delta = 1e-4), two calls."""
    import torch
    import paper_1502_03942_gb300 as tk
    from paper_1502_03942_gb300 import workloads as wl
    alg, log2n = spec.split(":")
    ctx = tk.Context(0)
    x = wl.device_zipf_objects(1 << int(log2n), seed=2024)
    fp = tk.make_freq_params(32, algorithm=tk.TOPK_FREQ_EC if alg == "ec" else tk.TOPK_FREQ_PAC,
                             epsilon=3e-4, delta=1e-4, seed=3)
    out = tk.topk_frequent(ctx, x, fp)
    tk.topk_frequent(ctx, x, fp, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"probe_frequent": spec, "sample_size": int(out[2].view(torch.int64).item())}))
    return 0


def run_probe_runs(spec):
    """Multisequence selection for profilers: K (1024 sorted u64 runs of
    2^U(10,20) keys; "half" for total/2), two calls."""
    import numpy as np
    import torch
    import paper_1502_03942_gb300 as tk
    from paper_1502_03942_gb300 import workloads as wl
    keys, off = wl.sorted_runs(1024, 10, 20, seed=3)
    d_keys = torch.from_numpy(keys.view(np.int64)).cuda().view(torch.uint64)
    d_off = torch.from_numpy(off.view(np.int64)).cuda().view(torch.uint64)
    k = int(off[-1]) // 2 if spec == "half" else int(spec)
    ctx = tk.Context(0)
    out = tk.topk_select_sorted_runs(ctx, d_keys, d_off, k)
    tk.topk_select_sorted_runs(ctx, d_keys, d_off, k, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"probe_runs": spec, "stats": ctx.last_stats()}))
    return 0


def run_probe_batched(spec):
    """The 4096-row batched workload for profilers: THREADS:SPLIT (0 = the
    default split length, -1 = none), two calls."""
    import numpy as np
    import torch
    import paper_1502_03942_gb300 as tk
    from paper_1502_03942_gb300 import workloads as wl
    threads, split = (int(x) for x in spec.split(":"))
    keys, off, ks = wl.batched_rows(4096, 10, 18, 1024, seed=4)
    d_keys = torch.from_numpy(keys).cuda()
    d_off = torch.from_numpy(off.view(np.int64)).cuda().view(torch.uint64)
    d_k = torch.from_numpy(ks.view(np.int32)).cuda().view(torch.uint32)
    ctx = tk.Context(0)
    p = tk.make_params(block_threads=threads, sample_size=1024 if threads == 256 else 2048,
                       split_rows=tk.TOPK_SPLIT_NONE if split < 0 else split)
    res = tk.topk_select_batched(ctx, d_keys, d_off, d_k, params=p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = tk.topk_select_batched(ctx, d_keys, d_off, d_k, params=p, out=res[:4], out_off=res[4])
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"probe_batched": spec, "ms": e0.elapsed_time(e1), "status": ctx.sync()}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain, batched, sorted-runs and served measurements")
    ap.add_argument("--probe", default=None,
                    help="profiling aid: DATASET:N:K[:FLAGS], one warm-up and one timed-by-profiler call")
    ap.add_argument("--probe-runs", default=None,
                    help="profiling aid: K or 'half', two multisequence selections over 1024 sorted runs")
    ap.add_argument("--probe-batched", default=None,
                    help="profiling aid: THREADS:SPLIT, two calls of topk_select_batched on 4096 rows")
    ap.add_argument("--probe-frequent", default=None,
                    help="profiling aid: ALG:LOG2N, two calls of topk_frequent (ec or pac)")
    args = ap.parse_args()
    if args.probe_frequent:
        return run_probe_frequent(args.probe_frequent)
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    if args.probe:
        return run_probe(args.probe)
    if args.probe_batched:
        return run_probe_batched(args.probe_batched)
    if args.probe_runs:
        return run_probe_runs(args.probe_runs)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

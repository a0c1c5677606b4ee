"""topk_select_batched on the GPU against the CPU oracle (bit-exact per row).

Rows of uneven length at arbitrary (unaligned) offsets, each with its own k,
in one persistent launch; every key type; rows longer than the split length
("wide" rows, whose first level runs over the whole GPU) at several split
lengths, with heavy ties and large k; the full batched configuration (4096
rows, lengths 2^U(10,18), N(0,3) keys, k in 1..1024) checked against the
oracle on a sample of rows and by properties on all rows.
"""
import numpy as np
import pytest

import oracle
from paper_1502_03942_gb300 import workloads as wl

from _gpu import bits_of, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03942_gb300 as tk
    return tk


@pytest.fixture(scope="module")
def ctx(tk):
    c = tk.Context(0)
    yield c
    c.close()


def rows_for(name, rows, lo, hi, kmax, seed):
    g = np.random.Generator(np.random.Philox(seed))
    lens = np.floor(2.0 ** g.uniform(lo, hi, size=rows)).astype(np.uint64)
    off = np.zeros(rows + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    total = int(off[-1])
    ks = np.minimum(g.integers(1, kmax + 1, size=rows).astype(np.uint64), lens).astype(np.uint32)
    if name in ("u32", "i32"):
        keys = wl.uniform_u32(total, seed)
    elif name == "f32":
        keys = wl.normal_f32(total, seed, 3.0).view(np.uint32)
    elif name == "bf16":
        keys = g.integers(0, 1 << 16, size=total).astype(np.uint16)
    else:
        keys = (g.integers(0, 50, size=total).astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15))
    return keys, off, ks


def run(tk, ctx, keys, off, ks, name):
    d_keys = to_device(keys, name)
    d_off = to_device(off, "u64")
    d_k = to_device(ks, "u32")
    return tk.topk_select_batched(ctx, d_keys, d_off, d_k)


def check_rows(keys, off, ks, name, res, rows_to_check):
    ok, oi, kk, ki, out_off = res
    got_idx, got_keys = bits_of(oi), bits_of(ok)
    got_kth_idx, got_kth_key = bits_of(ki), bits_of(kk)
    oo = bits_of(out_off).astype(np.int64)
    for i in rows_to_check:
        row = keys[int(off[i]):int(off[i + 1])]
        want_sel, want_kth = oracle.select(row, name, int(ks[i]))
        a, b = oo[i], oo[i + 1]
        assert np.array_equal(np.sort(got_idx[a:b]), np.sort(want_sel)), f"row {i} set differs"
        assert np.array_equal(got_keys[a:b], row[got_idx[a:b]]), f"row {i} keys"
        assert got_kth_idx[i] == want_kth and got_kth_key[i] == row[want_kth], f"row {i} kth"


@pytest.mark.parametrize("name", ["u32", "i32", "f32", "bf16", "u64"])
def test_batched_small(tk, ctx, name):
    keys, off, ks = rows_for(name, 300, 0, 15, 1024, seed=41)
    res = run(tk, ctx, keys, off, ks, name)
    check_rows(keys, off, ks, name, res, range(300))


def test_batched_k_extremes(tk, ctx):
    """k = 1 and k = n in rows longer and shorter than one block's capacity."""
    g = np.random.Generator(np.random.Philox(43))
    lens = np.array([1, 2, 5000, 40000, 70000, 16384, 16385, 3], np.uint64)
    off = np.zeros(lens.size + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    keys = g.integers(0, 100, size=int(off[-1])).astype(np.uint32)
    for ks in (np.ones(lens.size, np.uint32), lens.astype(np.uint32)):
        res = run(tk, ctx, keys, off, ks, "u32")
        check_rows(keys, off, ks, "u32", res, range(lens.size))


def test_batched_rejects_bad_k(tk, ctx):
    keys, off, ks = rows_for("u32", 10, 3, 8, 10, seed=44)
    ks[3] = 0
    with pytest.raises(tk.TopkError) as e:
        run(tk, ctx, keys, off, ks, "u32")
    assert e.value.status == tk.TOPK_EINVAL


def test_batched_config_full_size(tk, ctx):
    """4096 rows, lengths 2^U(10,18), N(0,3) f32, k in 1..1024."""
    keys, off, ks = wl.batched_rows(4096, 10, 18, 1024, seed=4)
    bits = keys.view(np.uint32)
    res = run(tk, ctx, bits, off, ks, "f32")
    g = np.random.Generator(np.random.Philox(45))
    sample = sorted(set(g.integers(0, 4096, size=150).tolist()) | {0, 4095})
    check_rows(bits, off, ks, "f32", res, sample)
    # every row: k outputs, all distinct, each <= the rank-k pair, and exactly
    # k - 1 pairs of the row below the rank-k pair (keys have no NaN / -0)
    ok, oi, kk, ki, out_off = res
    idx = bits_of(oi).astype(np.int64)
    oo = bits_of(out_off).astype(np.int64)
    kth_idx = bits_of(ki).astype(np.int64)
    kth_key = keys[off[:-1].astype(np.int64) + kth_idx]
    row_of_el = np.repeat(np.arange(4096), np.diff(off).astype(np.int64))
    pos_in_row = np.arange(int(off[-1])) - off[:-1].astype(np.int64)[row_of_el]
    kv = kth_key[row_of_el]
    below = (keys < kv) | ((keys == kv) & (pos_in_row < kth_idx[row_of_el]))
    counts = np.bincount(row_of_el, weights=below, minlength=4096).astype(np.int64)
    assert np.array_equal(counts, ks.astype(np.int64) - 1)
    assert np.array_equal(np.diff(oo), ks.astype(np.int64))
    row_of_out = np.repeat(np.arange(4096), ks.astype(np.int64))
    sel_keys = keys[off[:-1].astype(np.int64)[row_of_out] + idx]
    kvo = kth_key[row_of_out]
    assert np.all((sel_keys < kvo) | ((sel_keys == kvo) & (idx <= kth_idx[row_of_out])))
    # distinct positions per row
    combo = row_of_out.astype(np.int64) * (1 << 32) + idx
    assert np.unique(combo).size == combo.size


@pytest.mark.parametrize("threads", [256, 512, 1024])
@pytest.mark.parametrize("name", ["f32", "u64"])
def test_block_variants(tk, ctx, name, threads):
    """Every block size (and its finish capacity) gives the oracle's rows,
    including a finish threshold below the capacity and a small sample."""
    keys, off, ks = rows_for(name, 200, 8, 17, 1024, seed=45)
    d_keys, d_off, d_k = to_device(keys, name), to_device(off, "u64"), to_device(ks, "u32")
    for sample, T in ((0, 0), (512, 1024)):
        p = tk.make_params(block_threads=threads, sample_size=sample, finish_threshold=T)
        res = tk.topk_select_batched(ctx, d_keys, d_off, d_k, params=p)
        check_rows(keys, off, ks, name, res, range(200))


def test_tuner_choice_and_file(tk, tmp_path):
    """The tuner's choice is one of the candidates, the outputs it leaves are
    the oracle's, later calls without settings give the same result, and the
    choice survives a save / load into a fresh context."""
    import torch
    name = "f32"
    keys, off, ks = rows_for(name, 256, 8, 16, 1024, seed=46)
    d_keys, d_off, d_k = to_device(keys, name), to_device(off, "u64"), to_device(ks, "u32")
    c1 = tk.Context(0)
    ok, oi, kk, ki, out_off = tk.topk_select_batched(c1, d_keys, d_off, d_k)
    out = (torch.empty_like(ok), torch.empty_like(oi), torch.empty_like(kk), torch.empty_like(ki))
    best = tk.topk_tune_batched(c1, d_keys, d_off, d_k, out, out_off)
    assert best.block_threads in (256, 512, 1024)
    assert best.sample_size in (1024, 2048, 4096) or best.sample_size <= 4096
    assert best.finish_threshold >= 64
    check_rows(keys, off, ks, name, (*out, out_off), range(256))
    again = tk.topk_select_batched(c1, d_keys, d_off, d_k)
    check_rows(keys, off, ks, name, again, range(0, 256, 7))
    path = tmp_path / "tuning.txt"
    tk.topk_tuning_save(c1, str(path))
    lines = path.read_text().splitlines()
    assert lines[0] == "topk-tuning 2" and len(lines) == 2
    fields = lines[1].split("\t")
    assert fields[3:] == [str(best.block_threads), str(best.sample_size), str(best.finish_threshold),
                          str(best.split_rows)]
    assert best.split_rows in (1 << 13, 1 << 15, 1 << 17, tk.TOPK_SPLIT_NONE)
    c2 = tk.Context(0)
    tk.topk_tuning_load(c2, str(path))
    path2 = tmp_path / "tuning2.txt"
    tk.topk_tuning_save(c2, str(path2))
    assert path2.read_text() == path.read_text()
    bad = tmp_path / "bad.txt"
    bad.write_text("not a tuning file\n")
    with pytest.raises(tk.TopkError) as e:
        tk.topk_tuning_load(c2, str(bad))
    assert e.value.status == tk.TOPK_EINVAL
    c1.close()
    c2.close()


@pytest.mark.parametrize("name", ["u32", "i32", "f32", "bf16", "u64"])
def test_wide_rows(tk, ctx, name):
    """Rows of 2^12 .. 2^17 keys at unaligned offsets with split lengths that
    make most (4096), some (2^15) or none of them wide: every row the
    oracle's, whichever path it took; k up to 4096 and some rows at n/2."""
    keys, off, ks = rows_for(name, 48, 12, 17, 4096, seed=47)
    lens = np.diff(off).astype(np.int64)
    ks[::5] = (lens[::5] // 2).astype(np.uint32)
    d_keys, d_off, d_k = to_device(keys, name), to_device(off, "u64"), to_device(ks, "u32")
    for split in (4096, 1 << 15, tk.TOPK_SPLIT_NONE):
        res = tk.topk_select_batched(ctx, d_keys, d_off, d_k, params=tk.make_params(split_rows=split))
        check_rows(keys, off, ks, name, res, range(48))


@pytest.mark.parametrize("name", ["f32", "u64"])
def test_wide_rows_heavy_ties(tk, ctx, name):
    """Wide rows over a handful of values: the pivots fall inside runs of
    equal keys, so positions decide, in the grid pass and in the finish."""
    g = np.random.Generator(np.random.Philox(48))
    lens = np.floor(2.0 ** g.uniform(14, 17, size=24)).astype(np.uint64)
    off = np.zeros(25, np.uint64)
    off[1:] = np.cumsum(lens)
    vals = g.integers(0, 5, size=int(off[-1]))
    if name == "f32":
        keys = np.array([-1.0, -0.0, 0.0, 2.5, np.inf], np.float32)[vals].view(np.uint32)
    else:
        keys = vals.astype(np.uint64) * np.uint64(0x1234_5678_9ABC)
    ks = np.minimum(g.integers(1, 20000, size=24), lens).astype(np.uint32)
    d_keys, d_off, d_k = to_device(keys, name), to_device(off, "u64"), to_device(ks, "u32")
    res = tk.topk_select_batched(ctx, d_keys, d_off, d_k, params=tk.make_params(split_rows=4096))
    check_rows(keys, off, ks, name, res, range(24))


def test_tuning_file_version_1_is_read(tk, tmp_path):
    """A tuning file written before the split length existed still loads (its
    entries then choose the split length automatically)."""
    import torch
    name = torch.cuda.get_device_name(0)
    path = tmp_path / "v1.txt"
    path.write_text(f"topk-tuning 1\n{name}\t2\t8\t256\t1024\t4096\n")
    c = tk.Context(0)
    tk.topk_tuning_load(c, str(path))
    out = tmp_path / "v2.txt"
    tk.topk_tuning_save(c, str(out))
    assert out.read_text().splitlines()[1].split("\t")[3:] == ["256", "1024", "4096", "0"]
    c.close()

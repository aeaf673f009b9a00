"""Batched hulls (ch_hull_batched): every set's result equals the oracle on
that set alone, with local indices, including empty and one-point sets."""
import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(k, seed, lo=100, hi=200_000):
    sizes, kinds, seeds = W.batched_plan(k, seed, lo, hi)
    sets = [W.make(kd, sz, sd) for kd, sz, sd in zip(kinds, sizes, seeds)]
    return sets


def _run(lib, sets):
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([s.shape[0] for s in sets])
    pts = np.concatenate(sets) if offsets[-1] else np.zeros((0, 2), np.float32)
    res = lib.hull_batched(torch.from_numpy(pts).cuda(), torch.from_numpy(offsets))
    return [r.cpu().numpy() for r in res]


def test_batched_matches_oracle(lib):
    sets = _batch(40, 3)
    for got, s in zip(_run(lib, sets), sets):
        np.testing.assert_array_equal(got, oracle.hull(s))


def test_batched_with_empty_and_tiny_sets(lib):
    rng = np.random.default_rng(2)
    sets = [np.zeros((0, 2), np.float32), W.uniform(1, 1), W.normal(2, 3), np.zeros((0, 2), np.float32),
            rng.integers(0, 5, (1000, 2)).astype(np.float32), W.ring(5000, 4)]
    for got, s in zip(_run(lib, sets), sets):
        np.testing.assert_array_equal(got, oracle.hull(s))


def test_batched_equals_single(lib):
    sets = _batch(12, 9, 1000, 300_000)
    batched = _run(lib, sets)
    for got, s in zip(batched, sets):
        single = lib.hull(torch.from_numpy(s).cuda()).cpu().numpy()
        np.testing.assert_array_equal(got, single)


def _run_raw(lib, sets):
    """ch_hull_batched through the C ABI; returns (out_n list, per-set index arrays)."""
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([s.shape[0] for s in sets])
    pts = np.concatenate(sets) if offsets[-1] else np.zeros((0, 2), np.float32)
    d_pts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    d_off = torch.from_numpy(offsets).cuda()
    out_idx = torch.full((max(int(offsets[-1]), 1),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((len(sets),), -99, dtype=torch.int64, device="cuda")
    st = lib.load().ch_hull_batched(d_pts.data_ptr(), d_off.data_ptr(), len(sets), out_idx.data_ptr(),
                                    out_n.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    ns = out_n.cpu().tolist()
    idx = out_idx.cpu().numpy()
    return ns, [idx[offsets[i]:offsets[i] + max(ns[i], 0)] for i in range(len(sets))]


def test_batched_degenerate_sets(lib):
    suite = W.degenerate_suite()
    sets = list(suite.values())
    ns, got = _run_raw(lib, sets)
    for (name, s), h, g in zip(suite.items(), ns, got):
        want = oracle.hull(s)
        assert h == want.size, name
        np.testing.assert_array_equal(g, want, err_msg=name)


def test_batched_bad_set_does_not_spoil_others(lib):
    good = [W.uniform(3000, 1), W.normal(5000, 2)]
    bad = W.uniform(2000, 3)
    bad[77, 1] = -1.0
    ns, got = _run_raw(lib, [good[0], bad, good[1]])
    assert ns[1] == lib.CH_ERANGE
    np.testing.assert_array_equal(got[0], oracle.hull(good[0]))
    np.testing.assert_array_equal(got[2], oracle.hull(good[1]))


def test_batched_multi_tile_and_large_survivor_sets(lib):
    # sets spanning several 4096-point tiles with ragged ends, and ring sets
    # whose survivors exceed one block (the single-hull fallback)
    sets = [W.normal(4096 * 3 + 1, 5), W.uniform(4095, 6), W.ring(60_000, 7), W.ring(9_000, 8),
            W.normal(1, 9), W.ring(300_000, 10), W.uniform(8193, 11)]
    ns, got = _run_raw(lib, sets)
    for h, g, s in zip(ns, got, sets):
        want = oracle.hull(s)
        assert h == want.size
        np.testing.assert_array_equal(g, want)


def test_batched_repeated_and_odd_offsets(lib):
    # odd set sizes put later sets at 8- but not 16-byte aligned addresses
    sets = [W.uniform(101, 12), W.normal(3333, 13), W.ring(777, 14), W.uniform(1, 15), W.normal(20_001, 16)]
    first = _run_raw(lib, sets)
    second = _run_raw(lib, sets)
    assert first[0] == second[0]
    for a, b, s in zip(first[1], second[1], sets):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, oracle.hull(s))


def test_batched_unaligned_base_tiny_sets_and_ties(lib):
    """The batch starts 8 bytes past a 16-byte boundary (one head point before
    the streamed body), many tiny sets meet inside one warp tile, and extreme
    keys repeat across tiles and sets (lowest index wins)."""
    rng = np.random.default_rng(21)
    sets = [rng.integers(0, 7, (int(rng.integers(1, 60)), 2)).astype(np.float32) for _ in range(300)]
    sets += [np.repeat(W.uniform(50, 3), 40, axis=0), W.normal(30_001, 4),
             rng.integers(0, 1 << 24, (5000, 2)).astype(np.float32), W.ring(20_000, 5)]
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([s.shape[0] for s in sets])
    pts = np.concatenate(sets)
    buf = torch.zeros((pts.shape[0] + 1, 2), dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(pts).cuda()
    d_pts = buf[1:]
    assert d_pts.data_ptr() % 16 == 8
    d_off = torch.from_numpy(offsets).cuda()
    out_idx = torch.full((int(offsets[-1]),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((len(sets),), -99, dtype=torch.int64, device="cuda")
    st = lib.load().ch_hull_batched(d_pts.data_ptr(), d_off.data_ptr(), len(sets), out_idx.data_ptr(),
                                    out_n.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    ns = out_n.cpu().tolist()
    idx = out_idx.cpu().numpy()
    for i, s in enumerate(sets):
        want = oracle.hull(s)
        assert ns[i] == want.size, i
        np.testing.assert_array_equal(idx[offsets[i]:offsets[i] + ns[i]], want, err_msg=str(i))


# --- tile shapes and the autotuner ------------------------------------------

SHAPES = [(128, 16), (256, 8), (256, 16), (256, 32), (512, 8), (512, 16)]


def _shape_sets():
    """Sets that span several tiles of every shape with ragged tails (tile
    sizes 2048 .. 8192), plus empty, one-point and large-survivor sets."""
    sizes = [0, 1, 2047, 2048, 2049, 8191, 8193, 20_000, 70_001]
    kinds = ["uniform", "normal", "ring"]
    sets = [W.make(kinds[i % 3], n, 50 + i) if n else np.zeros((0, 2), np.float32) for i, n in enumerate(sizes)]
    sets.append(W.ring(40_000, 77))   # records beyond one block: the bucketed path
    return sets


@pytest.mark.parametrize("threads,per", SHAPES)
def test_batched_every_tile_shape_matches_oracle(lib, monkeypatch, threads, per):
    monkeypatch.setenv("CH_BLOCK", str(threads))
    monkeypatch.setenv("CH_PPT", str(per))
    sets = _shape_sets()
    assert lib.ch_batched_config(sum(s.shape[0] for s in sets), len(sets)) == (threads, per)
    for got, s in zip(_run(lib, sets), sets):
        np.testing.assert_array_equal(got, oracle.hull(s))


def test_batched_tile_env_and_invalid_shape(lib, monkeypatch):
    monkeypatch.setenv("CH_BLOCK", "256")
    monkeypatch.setenv("CH_TILE", "8192")
    assert lib.ch_batched_config(10_000, 4) == (256, 32)
    monkeypatch.setenv("CH_PPT", "7")   # CH_TILE and CH_PPT disagree
    with pytest.raises(lib.CHError) as e:
        lib.ch_batched_config(10_000, 4)
    assert e.value.status == lib.CH_EINVAL
    sets = [W.uniform(3000, 1), W.normal(5000, 2)]
    with pytest.raises(lib.CHError) as e:
        _run(lib, sets)
    assert e.value.status == lib.CH_EINVAL
    monkeypatch.delenv("CH_PPT")
    monkeypatch.delenv("CH_TILE")
    with pytest.raises(lib.CHError):   # a block size without points per thread
        lib.ch_batched_config(10_000, 4)


_TUNE_CHILD = r"""
import json, sys
import numpy as np
import torch
import paper_2209_12310_gb300 as ch
sys.path.insert(0, sys.argv[2])
from synth import workloads as W
total, k = int(sys.argv[3]), int(sys.argv[4])
if sys.argv[1] == "tune":
    assert ch.ch_batched_config(total, k) == (0, 0)
    sets = [W.make(("uniform", "normal", "ring")[i % 3], total // k, 100 + i) for i in range(k)]
    off = np.zeros(k + 1, np.int64); off[1:] = np.cumsum([s.shape[0] for s in sets])
    ch.hull_batched(torch.from_numpy(np.concatenate(sets)).cuda(), torch.from_numpy(off))
print(json.dumps(ch.ch_batched_config(total, k)))
"""


def test_batched_autotuner_cache_file(lib, tmp_path):
    """First batch of a size class tunes and writes the JSON cache; a new
    process reads its choice from the file (edited here to another shape)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.json"
    env = {k: v for k, v in os.environ.items() if k not in ("CH_BLOCK", "CH_PPT", "CH_TILE")}
    env["CH_TUNE_CACHE"] = str(cache)
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    total, k = 60_000, 6

    def child(mode):
        out = subprocess.run([sys.executable, "-c", _TUNE_CHILD, mode, root, str(total), str(k)], env=env,
                             capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stderr
        return tuple(json.loads(out.stdout.strip().splitlines()[-1]))

    tuned = child("tune")
    assert tuned in SHAPES
    table = json.loads(cache.read_text())
    assert len(table) == 1
    (key, (threads, per, us)), = table.items()
    assert (threads, per) == tuned and us > 0
    other = next(s for s in SHAPES if s != tuned)
    cache.write_text(json.dumps({key: [other[0], other[1], us]}))
    assert child("read") == other


def test_batched_set_left_to_single_hull_path(lib):
    """Sets in convex position overflow their bucket chains; ch_hull_batched
    finishes them with the single-hull path, beside ordinary sets."""
    m = 5000
    x = np.arange(m, dtype=np.int64)
    conv = np.stack([x * 64, x * (x + 1) // 2], 1)
    conv = conv[np.random.default_rng(4).permutation(m)].astype(np.float32)
    assert oracle.hull(conv).size == m
    i = np.arange(11_000, dtype=np.int64)   # a narrow U in convex position: bucket chains overflow
    y = np.concatenate([[0], np.cumsum(i[:-1] - 5500)])
    u_arc = np.stack([i * 1500, y - y.min() + 5], 1)[np.random.default_rng(6).permutation(11_000)].astype(np.float32)
    sets = [W.uniform(30_000, 1), conv, W.ring(50_000, 2), conv[: m // 2].copy(), u_arc]
    for got, s in zip(_run(lib, sets), sets):
        np.testing.assert_array_equal(got, oracle.hull(s))

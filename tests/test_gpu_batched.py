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

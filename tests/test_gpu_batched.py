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

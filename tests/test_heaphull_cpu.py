"""The CPU heaphull comparator (oracle/heaphull_cpu.c) gives the oracle's hull
on 1 and several threads, including degenerate and duplicate-heavy inputs."""
import numpy as np
import pytest

import oracle
from synth import workloads as W


@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("kind,n,seed", [("uniform", 50_000, 1), ("normal", 80_000, 2), ("ring", 30_000, 3)])
def test_heaphull_cpu_matches_oracle(kind, n, seed, threads):
    pts = W.make(kind, n, seed)
    np.testing.assert_array_equal(oracle.heaphull_cpu(pts, threads), oracle.hull(pts))


@pytest.mark.parametrize("threads", [1, 4])
def test_heaphull_cpu_degenerate(threads):
    rng = np.random.default_rng(5)
    cases = [
        np.zeros((0, 2), np.float32),
        np.array([[3, 4]], np.float32),
        np.array([[3, 4], [3, 4], [3, 4]], np.float32),                 # identical
        np.stack([np.arange(50), np.full(50, 7)], 1).astype(np.float32),  # horizontal line
        np.stack([np.arange(50), np.arange(50)], 1).astype(np.float32),   # diagonal line
        rng.integers(0, 4, (2000, 2)).astype(np.float32),                 # dense duplicates
        np.repeat(np.array([[0, 0], [9, 0], [9, 9], [0, 9]], np.float32), 5, axis=0)[rng.permutation(20)],
    ]
    for pts in cases:
        np.testing.assert_array_equal(oracle.heaphull_cpu(pts, threads), oracle.hull(pts))


def test_heaphull_cpu_more_threads_than_points_and_bad_input():
    pts = W.uniform(5, 9)
    np.testing.assert_array_equal(oracle.heaphull_cpu(pts, 64), oracle.hull(pts))
    bad = W.uniform(100, 1)
    bad[57, 1] = 0.5
    with pytest.raises(ValueError):
        oracle.heaphull_cpu(bad, 4)


@pytest.mark.parametrize("threads", [2, 5, 16])
def test_heaphull_cpu_chunk_boundaries(threads):
    """Chunks of the sorted survivors split runs of equal coordinates and
    collinear stretches; the per-chunk chains and the final pass over them
    must still give the oracle's hull."""
    rng = np.random.default_rng(threads)
    cases = [
        W.distorted(120_000, 11),
        rng.integers(0, 64, (100_000, 2)).astype(np.float32),                 # heavy duplicates
        np.repeat(np.stack([np.arange(3000), np.full(3000, 5)], 1), 3, axis=0).astype(np.float32),
        np.concatenate([np.stack([np.full(5000, 7), np.arange(5000)], 1),      # vertical line
                        np.array([[3, 2500], [11, 100]])]).astype(np.float32),
    ]
    cases += [v for v in W.degenerate_suite().values() if v.shape[0] > 0]
    for pts in cases:
        np.testing.assert_array_equal(oracle.heaphull_cpu(pts, threads), oracle.hull(pts))

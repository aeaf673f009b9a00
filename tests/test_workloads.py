"""The seeded input recipe matches the workload configurations it stands in
for: value ranges, distribution parameters, size and kind mixes, and
determinism per seed."""
import math

import numpy as np

from synth import workloads as W

R = 1 << 23


def _ints(pts):
    assert pts.dtype == np.float32 and pts.ndim == 2 and pts.shape[1] == 2
    assert np.all(pts == np.rint(pts)) and pts.min() >= 0 and pts.max() < (1 << 24)
    return pts.astype(np.float64)


def test_uniform_square():
    p = _ints(W.uniform(400_000, 0))
    assert abs(p.mean() / R - 1) < 0.01
    q = np.quantile(p[:, 0], [0.25, 0.5, 0.75]) / (1 << 24)
    np.testing.assert_allclose(q, [0.25, 0.5, 0.75], atol=0.01)


def test_normal_centre_and_sigma():
    p = _ints(W.normal(400_000, 1))
    np.testing.assert_allclose(p.mean(0), [R, R], rtol=2e-3)
    np.testing.assert_allclose(p.std(0), [1 << 21, 1 << 21], rtol=1e-2)


def test_ring_radius_band_and_angles():
    p = _ints(W.ring(200_000, 2)) - R
    r = np.hypot(p[:, 0], p[:, 1])
    assert r.min() > R - 64 - 1.5 and r.max() < R + 1.5
    quad = np.bincount((p[:, 0] > 0).astype(int) * 2 + (p[:, 1] > 0).astype(int), minlength=4)
    assert np.all(np.abs(quad / quad.sum() - 0.25) < 0.01)


def test_distorted_radius_band():
    p = _ints(W.distorted(200_000, 5)) - R
    r = np.hypot(p[:, 0], p[:, 1]) / R
    assert r.min() > 0.98 - 1e-6 and r.max() < 1 + 1e-6
    assert abs(np.median(r) - 0.99) < 0.001   # radius R (1 - 0.02 U)


def test_generators_are_deterministic_per_seed():
    for kind in ("uniform", "normal", "ring", "distorted"):
        a, b = W.make(kind, 10_000, 9), W.make(kind, 10_000, 9)
        np.testing.assert_array_equal(a, b)
        assert not np.array_equal(a, W.make(kind, 10_000, 10))


def test_batched_plan_mix():
    sizes, kinds, seeds = W.batched_plan(4096, 3)
    sizes = np.array(sizes)
    assert sizes.min() >= 100 and sizes.max() <= 1_000_000
    # log-uniform in [100, 1e6]: median near 1e4, a quarter below 10^3
    assert abs(math.log10(np.median(sizes)) - 4) < 0.1
    assert abs((sizes < 1000).mean() - 0.25) < 0.03
    frac = {k: kinds.count(k) / len(kinds) for k in ("uniform", "normal", "ring")}
    assert all(abs(v - 1 / 3) < 0.03 for v in frac.values())
    assert len(set(seeds)) == len(seeds)
    pts, off = W.batched(16, 3)
    assert off[0] == 0 and np.all(np.diff(off) > 0) and off[-1] == pts.shape[0]


def test_serving_plan_stream():
    arrivals, sizes, names = W.serving_plan()
    assert abs(arrivals.size - 200_000) < 5 * math.sqrt(200_000)
    assert arrivals.min() >= 0 and arrivals.max() < 10 and np.all(np.diff(arrivals) >= 0)
    assert sizes.min() >= 1000 and sizes.max() <= 10_000_000
    assert abs(math.log10(np.median(sizes)) - 5) < 0.05
    for name, want in (("normal", 0.5), ("uniform", 0.4), ("ring", 0.1)):
        assert abs((names == name).mean() - want) < 0.01

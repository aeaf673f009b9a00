"""Pins of the CPU oracle against facts fixed independently of it: brute force
on tiny inputs, lattice polygons with closed-form hulls, a library hull on
general-position inputs, and the properties that define the output."""
import numpy as np
import pytest

import oracle
from oracle import brute
from synth import workloads as W
from tests import golden_io
from tests.invariants import check_hull


def _cases_small():
    rng = np.random.default_rng(123)
    out = []
    for trial in range(60):
        n = int(rng.integers(1, 120))
        span = [3, 8, 40, 1000, 1 << 24][trial % 5]
        pts = rng.integers(0, span, (n, 2)).astype(np.float32)
        out.append(pts)
    # collinear-heavy: points on a few lines
    for trial in range(20):
        t = rng.integers(0, 50, 60)
        a, b = rng.integers(-3, 4, 2)
        pts = np.stack([t + 100, a * t // 1 + b * 7 + 500], 1)
        extra = rng.integers(90, 160, (int(rng.integers(0, 4)), 2))
        pts = np.concatenate([pts, extra]).astype(np.float32)
        out.append(pts)
    return out


@pytest.mark.parametrize("k", range(80))
def test_oracle_matches_brute_force(k):
    pts = _cases_small()[k]
    np.testing.assert_array_equal(oracle.hull(pts), brute.hull(pts))


@pytest.mark.parametrize("name", [n for n, v in W.degenerate_suite().items()])
def test_oracle_degenerate_suite(name):
    pts = W.degenerate_suite()[name]
    got = oracle.hull(pts)
    check_hull(pts, got)
    # brute force where it is affordable (distinct points <= ~250)
    if len({(float(a), float(b)) for a, b in pts}) <= 250:
        np.testing.assert_array_equal(got, brute.hull(pts))


def test_oracle_degenerate_closed_forms():
    cases = W.degenerate_suite()
    assert oracle.hull(cases["empty"]).size == 0
    np.testing.assert_array_equal(oracle.hull(cases["one"]), [0])
    np.testing.assert_array_equal(oracle.hull(cases["two"]), [1, 0])   # (3,4) < (9,1)
    np.testing.assert_array_equal(oracle.hull(cases["two_same"]), [0])
    np.testing.assert_array_equal(oracle.hull(cases["identical"]), [0])
    h = cases["horizontal"]
    got = oracle.hull(h)
    assert got.size == 2
    assert h[got[0], 0] == h[:, 0].min() and h[got[1], 0] == h[:, 0].max()
    assert got[0] == np.flatnonzero(h[:, 0] == h[:, 0].min())[0]
    v = cases["vertical"]
    got = oracle.hull(v)
    assert v[got[0], 1] == v[:, 1].min() and v[got[1], 1] == v[:, 1].max()
    sq = cases["square_extremes"]
    got = oracle.hull(sq)
    M = W.COORD_LIMIT - 1
    np.testing.assert_array_equal(sq[got], [[0, 0], [M, 0], [M, M], [0, M]])


@pytest.mark.parametrize("name", golden_io.FIXTURES)
@pytest.mark.parametrize("offset", [1000, W.COORD_LIMIT - 100])
def test_oracle_lattice_polygons(name, offset):
    pts, expected = golden_io.load(name, offset=offset)
    np.testing.assert_array_equal(oracle.hull(pts), expected)


def test_oracle_matches_scipy_on_general_position():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(10, 5000))
        pts = rng.integers(0, 1 << 24, (n, 2)).astype(np.float32)
        got = oracle.hull(pts)
        ref = spatial.ConvexHull(pts.astype(np.float64)).vertices  # CCW in 2-D
        start = int(np.flatnonzero(ref == got[0])[0]) if got[0] in ref else 0
        ref = np.roll(ref, -start)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("kind", ["uniform", "normal", "ring", "distorted"])
def test_oracle_invariants_on_workloads(kind):
    pts = W.make(kind, 200_000, seed=11)
    check_hull(pts, oracle.hull(pts))


def test_oracle_metamorphic_translation_and_mirror():
    rng = np.random.default_rng(9)
    pts = rng.integers(0, 1 << 20, (5000, 2))
    base = oracle.hull(pts.astype(np.float32))
    moved = oracle.hull((pts + [12345, 777]).astype(np.float32))
    np.testing.assert_array_equal(base, moved)
    # mirror x -> C - x reverses orientation; as a set the vertices agree and
    # the cyclic order is reversed
    mir = pts.copy()
    mir[:, 0] = (1 << 20) - mir[:, 0]
    hm = oracle.hull(mir.astype(np.float32))
    assert set(hm.tolist()) == set(base.tolist())
    rev = hm[::-1]
    k = int(np.flatnonzero(rev == base[0])[0])
    np.testing.assert_array_equal(np.roll(rev, -k), base)


def test_oracle_permutation_on_distinct_points():
    rng = np.random.default_rng(10)
    pts = np.unique(rng.integers(0, 1 << 24, (3000, 2)), axis=0)
    perm = rng.permutation(pts.shape[0])
    base = oracle.hull(pts.astype(np.float32))
    got = oracle.hull(pts[perm].astype(np.float32))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    np.testing.assert_array_equal(inv[base], got)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -1.0, 0.5, 16777216.0, 1e30, -np.inf])
def test_oracle_rejects_out_of_domain(bad):
    pts = np.array([[1, 2], [3, 4], [5, 1]], np.float32)
    pts[1, 0] = bad
    with pytest.raises(ValueError):
        oracle.hull(pts)
    assert not oracle.check(pts)


def test_oracle_accepts_domain_edges():
    pts = np.array([[0, 0], [16777215, 0], [16777215, 16777215], [0, 16777215], [-0.0, 5]],
                   np.float32)
    np.testing.assert_array_equal(oracle.hull(pts), [0, 1, 2, 3])


def test_distorted_workload_shape():
    """The 2%-distortion stand-in: integer points in the domain, within 2% of
    the radius inside the circle (plus rounding), angles spread round it."""
    pts = W.distorted(100_000, 5).astype(np.float64)
    assert pts.min() >= 0 and pts.max() < (1 << 24)
    assert np.all(pts == np.rint(pts))
    r = np.hypot(pts[:, 0] - (1 << 23), pts[:, 1] - (1 << 23)) / float(1 << 23)
    assert r.max() <= 1.0 + 1e-6 and r.min() >= 0.98 - 1e-6
    ang = np.arctan2(pts[:, 1] - (1 << 23), pts[:, 0] - (1 << 23))
    assert np.histogram(ang, bins=8)[0].min() > 10_000

"""Pins of the 16-direction filter polygon (oracle/filter16_ref.py): the
octagon definition (already pinned) for the even directions, a polygon with
known extremes, the C hull oracle (a different algorithm) for the strict
interior, and the properties the filter relies on."""
import math

import numpy as np
import pytest

import oracle
from oracle import filter16_ref as G
from oracle import filter_ref as F
from synth import workloads as W
from tests.test_filter_ref import SETS, _strictly_inside_hull_of


@pytest.mark.parametrize("k", range(len(SETS)))
def test_even_directions_are_the_octagon(k):
    """V_0, V_2, ..., V_14 are Alg. 2's W, SW, S, SE, E, NE, N, NW."""
    pts = SETS[k]
    np.testing.assert_array_equal(G.extremes16(pts)[0::2], F.extremes(pts))


def _circle16(rng, n_inner, dup=()):
    """Interior points (radius < R/2), then one point on a circle of radius R
    at the angle of each direction of DIRS, then copies of some of them."""
    c, R = float(1 << 23), float(1 << 20)
    ang = rng.uniform(0, 2 * math.pi, n_inner)
    rad = rng.uniform(0, R / 2, n_inner)
    inner = np.stack([np.rint(c + rad * np.cos(ang)), np.rint(c + rad * np.sin(ang))], 1)
    ring = []
    for a, b in G.DIRS:
        t = math.atan2(b, a)
        ring.append((round(c + R * math.cos(t)), round(c + R * math.sin(t))))
    ring = np.array(ring, np.float64)
    pts = np.concatenate([inner, ring, ring[list(dup)]]).astype(np.float32)
    return pts, n_inner


def test_known_extremes_on_a_circle():
    """On a circle, the point at direction k's own angle is the unique
    maximiser of that direction among the circle points (the next direction is
    at least 18.4 degrees away: a margin of 0.05 R against rounding of 1), and
    every interior point lies below it.  Later copies never win a tie."""
    rng = np.random.default_rng(16)
    pts, base = _circle16(rng, 3000, dup=(3, 9, 14))
    np.testing.assert_array_equal(G.extremes16(pts), base + np.arange(16))
    lab = G.labels16(pts)
    assert (lab[:base] == 0).all()            # strictly inside the 16-gon
    # vertices are on its boundary: W, S, E, N lie on the quadrilateral (no
    # queue); the three between two of them are in that arc's queue
    np.testing.assert_array_equal(lab[base:base + 16], [0, 1, 1, 1, 0, 2, 2, 2, 0, 3, 3, 3, 0, 4, 4, 4])


def test_ties_take_the_lowest_index():
    """A copy of a circle point placed BEFORE the original wins its direction."""
    rng = np.random.default_rng(17)
    pts, base = _circle16(rng, 100)
    pts = np.concatenate([pts[base + 5:base + 6], pts])   # copy of V_5 at index 0
    ext = G.extremes16(pts)
    assert ext[5] == 0
    np.testing.assert_array_equal(np.delete(ext, 5), np.delete(base + 1 + np.arange(16), 5))


@pytest.mark.parametrize("k", range(len(SETS)))
def test_inside16_matches_hull_of_the_16_extremes(k):
    """The polygon V_0..V_15 taken in direction order has the strict interior
    of the convex hull of the 16 points (C oracle): the order is
    counter-clockwise and the polygon convex."""
    pts = SETS[k]
    ext = G.extremes16(pts)
    np.testing.assert_array_equal(G.inside16(pts, ext), _strictly_inside_hull_of(pts, ext))


@pytest.mark.parametrize("k", range(len(SETS)))
def test_16gon_contains_the_octagon(k):
    pts = SETS[k]
    assert not (F.inside_octagon(pts) & ~G.inside16(pts)).any()


@pytest.mark.parametrize("k", range(len(SETS)))
def test_filter16_keeps_every_hull_vertex(k):
    """No hull vertex is discarded, and the hull of the kept points plus the
    16 extremes is the hull of all points."""
    pts = SETS[k]
    full = oracle.hull(pts)
    lab = G.labels16(pts)
    kept = lab > 0
    kept[G.extremes16(pts)] = True
    assert kept[full].all()
    sel = np.flatnonzero(kept)
    np.testing.assert_array_equal(sel[oracle.hull(pts[sel])], full)


def test_degenerate_polygon_discards_nothing():
    pts = np.array([[0, 0], [10, 3], [5, 1], [4, 1]], np.float32)   # extremes on one line
    _, area2 = G.polygon16(pts)
    assert area2 == 0
    assert not G.inside16(pts).any()
    np.testing.assert_array_equal(G.labels16(pts), F.labels(pts))


def test_survivors_fewer_on_normal_and_distorted():
    """The point of a wider polygon: fewer survivors where the hull is round
    and the octagon leaves a rim (1e6-point samples; the octagon keeps 380 and
    934,941 of them)."""
    n = G.region_counts16(W.normal(1_000_000, 1)).sum()
    assert 0 < n <= 0.5 * F.region_counts(W.normal(1_000_000, 1)).sum()
    d16 = (G.labels16(W.distorted(1_000_000, 5)) > 0).sum()
    d8 = (F.labels(W.distorted(1_000_000, 5)) > 0).sum()
    assert d16 <= 0.75 * d8


def test_planted_direction_error_is_caught(monkeypatch):
    """A plausible mistake planted in the oracle (one direction with a flipped
    sign, which breaks the counter-clockwise order) fails the hull pin."""
    pts = W.normal(20_000, 3)
    dirs = list(G.DIRS)
    dirs[9] = (2, -1)
    monkeypatch.setattr(G, "DIRS", tuple(dirs))
    ext = G.extremes16(pts)
    assert not np.array_equal(G.inside16(pts, ext), _strictly_inside_hull_of(pts, ext))


@pytest.mark.parametrize("k", range(len(SETS)))
def test_sampled16_drop_keeps_the_hull(k):
    """The drop rule for a sample's 16-gon removes no output point (the
    lowest-index copy of each hull vertex), so the hull of what is left is the
    hull of all points; several samples per set, including one that is a
    single tile and one that is every point."""
    pts = SETS[k]
    n = pts.shape[0]
    full = oracle.hull(pts)
    rng = np.random.default_rng(k)
    samples = [G.sample_tiles(n), G.sample_tiles(n, tile=7, every=3), np.arange(min(n, 512)),
               np.arange(n), np.sort(rng.choice(n, size=max(1, n // 10), replace=False))]
    for s in samples:
        drop = G.hull_drop_sampled16(pts, s)
        assert not drop[full].any()
        sel = np.flatnonzero(~drop)
        np.testing.assert_array_equal(sel[oracle.hull(pts[sel])], full)


def test_sampled16_drop_keeps_every_copy_of_a_vertex():
    """A copy of a sample vertex that comes before the sample (lower index)
    is the hull's choice; the rule must not drop it."""
    rng = np.random.default_rng(21)
    pts, base = _circle16(rng, 2000)
    pts = np.concatenate([pts[base + 9:base + 10], pts])   # copy of V_9 at index 0
    sample = np.arange(1 + base, 1 + base + 16)             # the circle points only
    drop = G.hull_drop_sampled16(pts, sample)
    assert not drop[0] and not drop[1 + base + 9]
    assert drop[1:1 + base].all()                          # interior points go
    full = oracle.hull(pts)
    assert 0 in full and (1 + base + 9) not in full


def test_sampled16_drops_most_of_the_distorted_rim():
    """Every 32nd tile of 512 points is enough: with the octagon the hull
    stage keeps about 0.64 of the distorted points (0.935 with the octagon
    alone)."""
    pts = W.distorted(1_000_000, 5)
    keep = ~(F.inside_octagon(pts) | G.hull_drop_sampled16(pts, G.sample_tiles(pts.shape[0])))
    assert 0.6 < keep.mean() < 0.68


@pytest.mark.parametrize("offset", [1000, W.COORD_LIMIT - 100])
def test_known_extremes_on_the_lattice_circle(offset):
    """The twelve lattice points of x^2 + y^2 = 25 (tests/golden), worked by
    hand: in each (+-2, +-1) and (+-1, +-2) direction one of (+-4, +-3),
    (+-3, +-4) is the unique maximum (value 11; the disk interior reaches at
    most 10), the axis directions hit (+-5, 0) and (0, +-5), and each
    diagonal ties between two points (value 7), which goes to the lower index
    (the fixture repeats every vertex later, never earlier)."""
    from tests import golden_io
    pts, _ = golden_io.load("lattice_circle25.txt", offset=offset)
    first = {}
    for i, (a, b) in enumerate(pts.astype(np.int64).tolist()):
        first.setdefault((a - offset, b - offset), i)
    f = first.__getitem__
    want = [f((-5, 0)), f((-4, -3)), min(f((-4, -3)), f((-3, -4))), f((-3, -4)),
            f((0, -5)), f((3, -4)), min(f((3, -4)), f((4, -3))), f((4, -3)),
            f((5, 0)), f((4, 3)), min(f((4, 3)), f((3, 4))), f((3, 4)),
            f((0, 5)), f((-3, 4)), min(f((-3, 4)), f((-4, 3))), f((-4, 3))]
    np.testing.assert_array_equal(G.extremes16(pts), want)
    # every disk-interior point is strictly inside the 16-gon (the twelve
    # circle points span it), the circle points and their copies are not
    lab_in = G.inside16(pts)
    circle = {(5, 0), (4, 3), (3, 4), (0, 5), (-3, 4), (-4, 3), (-5, 0), (-4, -3), (-3, -4), (0, -5),
              (3, -4), (4, -3)}
    on = np.array([(a - offset, b - offset) in circle for a, b in pts.astype(np.int64).tolist()])
    assert not lab_in[on].any() and lab_in[~on].all()

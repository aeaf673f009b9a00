"""Pins of the numpy filter definition (oracle/filter_ref.py): the paper's own
two-kernel Manhattan formulation, the hull oracle (a different algorithm), and
the properties the method relies on."""
import numpy as np
import pytest

import oracle
from oracle import filter_ref as F
from synth import workloads as W


def _point_sets():
    rng = np.random.default_rng(77)
    sets = []
    for span in (2, 3, 5, 9, 100, 1 << 24):
        for n in (1, 2, 3, 17, 400):
            sets.append(rng.integers(0, span, (n, 2)).astype(np.float32))
    sets.append(W.normal(100_000, 3))
    sets.append(W.ring(50_000, 4))
    sets.append(W.uniform(50_000, 5))
    sets += [v for k, v in W.degenerate_suite().items() if v.shape[0] > 0]
    return sets


SETS = _point_sets()


@pytest.mark.parametrize("k", range(len(SETS)))
def test_extremes_equal_paper_manhattan_two_step(k):
    """Sec. 3 finds the corner points by minimum Manhattan distance to the
    corners of the axis-extreme box, in a second kernel; the x +/- y form must
    select the same indices (lowest index on ties)."""
    pts = SETS[k]
    np.testing.assert_array_equal(F.extremes(pts), F.extremes_manhattan(pts))


def test_extremes_known_octagon_with_ties():
    # Lattice octagon with vertices (2,0),(4,0),(6,2),(6,4),(4,6),(2,6),(0,4),(0,2)
    # plus interior fill; ties everywhere.  By hand: min x = 0 at (0,2),(0,4):
    # the lower index wins, etc.
    verts = [(2, 0), (4, 0), (6, 2), (6, 4), (4, 6), (2, 6), (0, 4), (0, 2)]
    fill = [(x, y) for x in range(1, 6) for y in range(1, 6)
            if 3 <= x + y <= 9 and -3 <= x - y <= 3]
    pts = np.array(fill + verts, np.float32)
    base = len(fill)
    idx = {v: base + i for i, v in enumerate(verts)}
    got = F.extremes(pts)
    # W: x=0 -> (0,4) listed before (0,2); SW: min x+y = 2 at (2,0),(0,2) -> (2,0)
    # S: y=0 -> (2,0); SE: max x-y = 4 at (4,0),(6,2) -> (4,0); E: x=6 -> (6,2)
    # NE: max x+y = 10 at (6,4),(4,6) -> (6,4); N: y=6 -> (4,6); NW: min x-y=-4 at (2,6),(0,4) -> (2,6)
    want = [idx[(0, 4)], idx[(2, 0)], idx[(2, 0)], idx[(4, 0)], idx[(6, 2)],
            idx[(6, 4)], idx[(4, 6)], idx[(2, 6)]]
    np.testing.assert_array_equal(got, want)


def _strictly_inside_hull_of(pts, vertex_idx):
    """Independent strict-inside test: hull of the 8 extremes by the C oracle,
    then cross > 0 against every edge of that strictly convex polygon."""
    a = np.asarray(pts, np.float32)
    sub = a[vertex_idx]
    h = oracle.hull(sub)
    x = a[:, 0].astype(np.int64)
    y = a[:, 1].astype(np.int64)
    if h.size < 3:
        return np.zeros(x.size, bool)
    hx = sub[h, 0].astype(np.int64)
    hy = sub[h, 1].astype(np.int64)
    inside = np.ones(x.size, bool)
    for i in range(h.size):
        j = (i + 1) % h.size
        inside &= (hx[j] - hx[i]) * (y - hy[i]) - (hy[j] - hy[i]) * (x - hx[i]) > 0
    return inside


@pytest.mark.parametrize("k", range(len(SETS)))
def test_octagon_inside_matches_hull_of_extremes(k):
    pts = SETS[k]
    ext = F.extremes(pts)
    np.testing.assert_array_equal(F.inside_octagon(pts, ext), _strictly_inside_hull_of(pts, ext))


@pytest.mark.parametrize("k", range(len(SETS)))
def test_filter_keeps_every_hull_vertex(k):
    """No hull vertex is ever discarded, and the hull of the kept points plus
    the 8 extremes is the hull of all points (indices mapped back)."""
    pts = SETS[k]
    full = oracle.hull(pts)
    ext = F.extremes(pts)
    lab = F.labels(pts)
    kept = lab > 0
    kept[ext] = True
    assert kept[full].all()
    sel = np.flatnonzero(kept)
    sub = oracle.hull(pts[sel])
    np.testing.assert_array_equal(sel[sub], full)


@pytest.mark.parametrize("k", range(len(SETS)))
def test_queues_follow_hull_order(k):
    """Heaphull builds the hull per queue and joins them (Alg. 1): the hull
    vertices in queue 1 lie on the CCW arc W->S, queue 2 on S->E, queue 3 on
    E->N, queue 4 on N->W."""
    pts = SETS[k]
    full = oracle.hull(pts)
    if full.size < 3:
        return
    lab = F.labels(pts)
    ext = F.extremes(pts)
    a = np.asarray(pts, np.float32).astype(np.int64)
    hx, hy = a[full, 0], a[full, 1]
    h = full.size

    def boundary_pos(i):
        # position of point i along the CCW boundary: p for vertex p, p + 0.5
        # for a point inside edge (p, p+1)
        px, py = a[i]
        for p in range(h):
            if hx[p] == px and hy[p] == py:
                return float(p)
        for p in range(h):
            q = (p + 1) % h
            c = (hx[q] - hx[p]) * (py - hy[p]) - (hy[q] - hy[p]) * (px - hx[p])
            if c == 0 and min(hx[p], hx[q]) <= px <= max(hx[p], hx[q]) \
                    and min(hy[p], hy[q]) <= py <= max(hy[p], hy[q]):
                return p + 0.5
        raise AssertionError("extreme point not on the hull boundary")

    quad = [boundary_pos(ext[j]) for j in (0, 2, 4, 6)]
    for v_pos, v in enumerate(full):
        q = int(lab[v])
        if q == 0:
            continue
        a0, a1 = quad[q - 1], quad[q % 4]
        span = (a1 - a0) % h
        off = (v_pos - a0) % h
        assert 0 < off < span, (q, v_pos, a0, a1)


def test_discard_rate_normal_exceeds_99_9_percent():
    """Sec. 4 reports more than 99.99% discarded on normal data; with this
    project's parameters the bar is 99.9%."""
    pts = W.normal(1_000_000, 1)
    lab = F.labels(pts)
    assert (lab == 0).mean() > 0.999


def test_ring_keeps_almost_everything():
    pts = W.ring(200_000, 2)
    assert (F.labels(pts) > 0).mean() > 0.99


def test_degenerate_octagon_discards_nothing():
    # all 8 extremes on one line but a point off it (slope 3/10 case)
    pts = np.array([[0, 0], [10, 3], [5, 1], [4, 1]], np.float32)
    ext = F.extremes(pts)
    _, area2 = F.octagon(pts, ext)
    assert area2 == 0
    assert not F.inside_octagon(pts, ext).any()
    np.testing.assert_array_equal(F.labels(pts), [0, 0, 2, 2])


def test_planted_sign_error_is_caught(monkeypatch):
    """A plausible mistake planted in the oracle (a transposed orientation)
    must fail the pins above."""
    pts = W.normal(20_000, 3)
    good = F.inside_octagon(pts)
    orig = F.orient
    monkeypatch.setattr(F, "orient", lambda ax, ay, bx, by, px, py: -orig(ax, ay, bx, by, px, py))
    bad = F.inside_octagon(pts)
    assert not np.array_equal(good, bad)
    assert not np.array_equal(bad, _strictly_inside_hull_of(pts, F.extremes(pts)))

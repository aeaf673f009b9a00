"""The star polygon that filters dense data (points near a circle, where
almost every point survives the octagon), through the C ABI: on every input
the hull stays bit-exact with the oracle, and on the ring and distorted
workloads the polygon is built and cuts the records the hull stage sees.

The inputs stress what the polygon's construction and test rely on: lattice
duplicates of its vertices, points on its edges and spokes, a centre far from
the middle of the data, arcs that do not go round the centre, gaps, and
convex position."""
import math

import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _hull_and_counters(lib, pts):
    d = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float32)).cuda()
    out_idx = torch.full((max(pts.shape[0], 1),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    lib.ch_hull(d.data_ptr(), pts.shape[0], out_idx.data_ptr(), out_n.data_ptr(), s)
    h = int(out_n.item())
    return out_idx[:max(h, 0)].cpu().numpy(), lib.ch_hull_counters(s)


def _check(lib, pts):
    got, c = _hull_and_counters(lib, pts)
    np.testing.assert_array_equal(got, oracle.hull(pts))
    return c


def _ring(n, seed, cx, cy, rx, ry, width, a0=0.0, a1=2 * math.pi):
    rng = np.random.default_rng(seed)
    th = rng.uniform(a0, a1, n)
    u = rng.uniform(0.0, width, n)
    x = np.rint(cx + (rx - u) * np.cos(th))
    y = np.rint(cy + (ry - u) * np.sin(th))
    return np.clip(np.stack([x, y], 1), 0, (1 << 24) - 1).astype(np.float32)


@pytest.mark.parametrize("kind,n,seed", [("ring", 2_000_003, 21), ("distorted", 2_000_001, 22)])
def test_dense_workloads_build_the_polygon_and_stay_exact(lib, kind, n, seed):
    pts = W.make(kind, n, seed)
    c = _check(lib, pts)
    assert c["two_pass"] == 1 and c["star_vertices"] > 1000, c
    assert c["records"] < n // 10, c   # most points fell inside the polygon


def test_duplicates_of_every_point(lib):
    base = W.ring(700_000, 23)
    pts = np.concatenate([base, base[::-1], base[:1000]])   # each vertex twice, a later copy first
    c = _check(lib, pts)
    assert c["star_vertices"] > 0, c


def test_off_centre_ellipse(lib):
    # a flat ellipse near one corner: the centre of the sample octagon is far
    # from the middle of the point cloud's angular spread
    pts = _ring(1_500_000, 24, 2_000_000, 15_000_000, 1_900_000, 190_000, 300)
    _check(lib, pts)


@pytest.mark.parametrize("a0,a1", [(0.0, math.pi), (0.3, 1.9 * math.pi), (-0.2, 0.4)])
def test_arcs_that_do_not_go_round(lib, a0, a1):
    pts = _ring(1_200_000, 25, 1 << 23, 1 << 23, (1 << 23) - 2, (1 << 23) - 2, 64, a0, a1)
    _check(lib, pts)


def test_ring_with_gaps(lib):
    pts = _ring(1_500_000, 26, 1 << 23, 1 << 23, 6_000_000, 6_000_000, 40)
    ang = np.arctan2(pts[:, 1] - (1 << 23), pts[:, 0] - (1 << 23))
    keep = (np.floor((ang + math.pi) / (2 * math.pi) * 12).astype(int) % 2) == 0   # six gaps of 30 degrees
    _check(lib, pts[keep])


def test_square_annulus(lib):
    # dense points near the four sides of a square: long collinear hull edges
    rng = np.random.default_rng(27)
    m = 400_000
    t = rng.integers(1_000_000, 15_000_001, m)
    d = rng.integers(0, 50, m)
    side = rng.integers(0, 4, m)
    x = np.where(side == 0, 1_000_000 + d, np.where(side == 1, 15_000_000 - d, t))
    y = np.where(side == 2, 1_000_000 + d, np.where(side == 3, 15_000_000 - d, t))
    pts = np.stack([x, y], 1).astype(np.float32)
    _check(lib, pts)


def test_lattice_circle_with_fill(lib):
    # every lattice point of a thin annulus, repeated and shuffled: many points
    # on the polygon's edges, spokes and vertices
    r0, r1 = 3000, 3004
    xs = np.arange(-r1, r1 + 1)
    X, Y = np.meshgrid(xs, xs)
    rr = X * X + Y * Y
    ring = np.stack([X[(rr >= r0 * r0) & (rr <= r1 * r1)], Y[(rr >= r0 * r0) & (rr <= r1 * r1)]], 1)
    pts = np.concatenate([ring] * 6) + (1 << 22)
    pts = pts[np.random.default_rng(28).permutation(pts.shape[0])].astype(np.float32)
    assert pts.shape[0] > 131072 * 3
    _check(lib, pts)


def test_convex_position_dense(lib):
    # all points are hull vertices (a parabola arc), more than the star pass's
    # minimum size: nothing may be dropped
    x = np.arange(0, 5792, dtype=np.int64)
    arc = np.stack([x * 64, x * (x + 1) // 2], 1)
    pts = np.concatenate([arc] * 60)
    pts = pts[np.random.default_rng(29).permutation(pts.shape[0])].astype(np.float32)
    _check(lib, pts)

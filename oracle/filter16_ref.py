"""The 16-direction filter polygon, written out plainly in numpy int64.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Among related work (Sec. 2) the paper cites a GPU filter that discards the
points inside a convex polygon of 16 extreme points; it gives neither the
directions nor the rule.  The reading used here keeps Alg. 2's rules and
only widens the polygon:

* ``DIRS``: 16 outward directions (a, b), in counter-clockwise order of their
  angle, starting at W.  The even ones are the 8 directions of Alg. 2's
  octagon (multiples of 45 degrees); the odd ones are the integer directions
  between them, (+-2, +-1) and (+-1, +-2) (angles 26.57 + k 90 and
  63.43 + k 90 degrees):

      k  0 W (-1, 0)    1 (-2,-1)    2 SW (-1,-1)   3 (-1,-2)
         4 S ( 0,-1)    5 ( 1,-2)    6 SE ( 1,-1)   7 ( 2,-1)
         8 E ( 1, 0)    9 ( 2, 1)   10 NE ( 1, 1)  11 ( 1, 2)
        12 N ( 0, 1)   13 (-1, 2)   14 NW (-1, 1)  15 (-2, 1)

* ``extremes16``: V_k = argmax over the points of a_k x + b_k y, the lowest
  index on ties (as findExtremes, Alg. 2).  V_0, V_2, ..., V_14 are the
  octagon's W, SW, ..., NW.  The V_k lie on the hull boundary in weakly
  counter-clockwise order, so they span a convex polygon inside the hull.
* ``inside16``: a point is discarded when it lies strictly inside that
  polygon (strictly left of every edge of non-zero length); a polygon of zero
  area discards nothing (the octagon's rule, Alg. 1 / 2).
* ``labels16``: the label array of Alg. 2 against this polygon: 0 for a
  discarded point, else the queue 1..4 of the quadrilateral rule over
  W = V_0, S = V_4, E = V_8, N = V_12 (unchanged from the octagon).

Every key |a x + b y| is below 3 * 2^24 and every orientation product below
2^50, so int64 holds all of it exactly.
"""
from __future__ import annotations

import numpy as np

from . import filter_ref

DIRS = ((-1, 0), (-2, -1), (-1, -1), (-1, -2), (0, -1), (1, -2), (1, -1), (2, -1),
        (1, 0), (2, 1), (1, 1), (1, 2), (0, 1), (-1, 2), (-1, 1), (-2, 1))


def _ints(pts):
    a = np.asarray(pts, dtype=np.float32).reshape(-1, 2)
    return a[:, 0].astype(np.int64), a[:, 1].astype(np.int64)


def extremes16(pts) -> np.ndarray:
    """Indices V_0..V_15 (int64[16]) of the points extreme in DIRS; lowest index on ties."""
    x, y = _ints(pts)
    # np.argmax returns the first (lowest-index) maximiser
    return np.array([np.argmax(a * x + b * y) for a, b in DIRS], dtype=np.int64)


def polygon16(pts, ext=None):
    """Vertex coordinates (16, 2) int64 and twice the signed area."""
    x, y = _ints(pts)
    if ext is None:
        ext = extremes16(pts)
    vx, vy = x[ext], y[ext]
    area2 = int(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy))
    return np.stack([vx, vy], 1), area2


def inside16(pts, ext=None) -> np.ndarray:
    """Boolean mask of the points strictly inside the 16-direction polygon."""
    x, y = _ints(pts)
    if x.size == 0:
        return np.zeros(0, bool)
    v, area2 = polygon16(pts, ext)
    if area2 == 0:
        return np.zeros(x.size, bool)
    inside = np.ones(x.size, bool)
    for k in range(16):
        ax, ay = v[k]
        bx, by = v[(k + 1) % 16]
        if ax == bx and ay == by:
            continue
        inside &= filter_ref.orient(ax, ay, bx, by, x, y) > 0
    return inside


def labels16(pts) -> np.ndarray:
    """0 = strictly inside the 16-direction polygon (or in no queue), else the queue 1..4."""
    ext = extremes16(pts)
    lab = filter_ref.regions(pts, ext[0::2])   # W, SW, S, SE, E, NE, N, NW
    lab[inside16(pts, ext)] = 0
    return lab


def region_counts16(pts) -> np.ndarray:
    lab = labels16(pts)
    return np.array([(lab == r).sum() for r in range(1, 5)], dtype=np.int64)


def sample_tiles(n, tile=512, every=32):
    """Indices of a strided sample: the first of every `every` tiles of `tile`
    consecutive points (about n / every points)."""
    starts = np.arange(0, n, tile * every)
    if starts.size == 0:
        return np.zeros(0, np.int64)
    return np.concatenate([np.arange(s, min(s + tile, n)) for s in starts]).astype(np.int64)


def hull_drop_sampled16(pts, sample_idx) -> np.ndarray:
    """Points the hull stage may drop given the 16-direction polygon P of a
    sample's extremes (vertices V_k = extremes16 of the sample, as indices
    into pts): every point strictly inside P, and every point on P's boundary
    whose coordinates are not those of a vertex.

    Why this is safe: P's vertices are input points, so P lies in the hull.
    A point strictly inside P is strictly inside the hull.  A point on an
    edge of P at no vertex lies strictly between two input points, so it is
    no strictly convex hull vertex, and neither is any point sharing its
    coordinates.  Copies of a vertex's coordinates are kept: the sample's
    vertex has the lowest index within the sample only, and the hull must
    report the lowest index of all copies.  A polygon of zero area drops
    nothing."""
    x, y = _ints(pts)
    drop = np.zeros(x.size, bool)
    sample_idx = np.asarray(sample_idx, np.int64)
    if x.size == 0 or sample_idx.size == 0:
        return drop
    ext = sample_idx[extremes16(np.asarray(pts, np.float32).reshape(-1, 2)[sample_idx])]
    v, area2 = polygon16(pts, ext)
    if area2 == 0:
        return drop
    closed = np.ones(x.size, bool)
    strict = np.ones(x.size, bool)
    for k in range(16):
        ax, ay = v[k]
        bx, by = v[(k + 1) % 16]
        if ax == bx and ay == by:
            continue
        o = filter_ref.orient(ax, ay, bx, by, x, y)
        closed &= o >= 0
        strict &= o > 0
    at_vertex = np.zeros(x.size, bool)
    for vx, vy in {(int(a), int(b)) for a, b in v}:
        at_vertex |= (x == vx) & (y == vy)
    return strict | (closed & ~at_vertex)

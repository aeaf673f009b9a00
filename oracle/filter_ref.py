"""The paper's filtering stage written out plainly in numpy int64.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Alg. 2 (GPUfilter) and Sec. 3:

* ``extremes``            -- findExtremes: the 8 directional extreme points.
  The four axis extremes W, E, S, N are argmin/argmax of x and y (Sec. 3,
  first step).  The four corner points are, per Sec. 3, the points of minimum
  Manhattan distance to the corners of the box spanned by the axis extremes;
  because every point lies inside that box, the Manhattan distance to corner
  (xmax, ymax) is (xmax - x) + (ymax - y), so the minimiser is argmax(x + y);
  likewise argmin(x + y), argmax(x - y) and argmin(x - y).  ``extremes`` uses
  the x +/- y form; ``extremes_manhattan`` is the paper's literal two-step form
  and serves as a pin of the first.  Ties take the lowest index (numpy's
  argmin/argmax return the first occurrence).
* ``inside_octagon``      -- "P[j] is outside the convex octagon CP(E)"
  (Alg. 1 and Alg. 2): a point is discarded when it lies strictly inside the
  octagon W, SW, S, SE, E, NE, N, NW (counter-clockwise).  Zero-length edges
  are skipped; an octagon of zero area discards nothing.
* ``regions``             -- findQueue (Alg. 2): the queue of a kept point.
  The paper gives no formula; the reading used is the quadrilateral rule:
  queue 1 (lower-left) if the point is strictly right of W->S, else 2 if
  strictly right of S->E, else 3 if strictly right of E->N, else 4 if
  strictly right of N->W; none otherwise.
* ``labels``              -- the array Q[1..n] of Alg. 2: 0 for a discarded
  point (strictly inside the octagon, or in no queue), else its queue 1..4.
"""
from __future__ import annotations

import numpy as np

# Order of the 8 extremes, counter-clockwise around the octagon.
NAMES = ("W", "SW", "S", "SE", "E", "NE", "N", "NW")


def _ints(pts):
    a = np.asarray(pts, dtype=np.float32).reshape(-1, 2)
    return a[:, 0].astype(np.int64), a[:, 1].astype(np.int64)


def extremes(pts) -> np.ndarray:
    """Indices of W, SW, S, SE, E, NE, N, NW (int64[8]); lowest index on ties."""
    x, y = _ints(pts)
    s = x + y
    d = x - y
    return np.array([
        np.argmin(x),  # W
        np.argmin(s),  # SW
        np.argmin(y),  # S
        np.argmax(d),  # SE
        np.argmax(x),  # E
        np.argmax(s),  # NE
        np.argmax(y),  # N
        np.argmin(d),  # NW
    ], dtype=np.int64)


def extremes_manhattan(pts) -> np.ndarray:
    """Paper-literal two-kernel form (Sec. 3): axis extremes first, then for each
    corner of their bounding box the point of minimum Manhattan distance."""
    x, y = _ints(pts)
    w, e, s, n = np.argmin(x), np.argmax(x), np.argmin(y), np.argmax(y)
    xmin, xmax, ymin, ymax = x[w], x[e], y[s], y[n]
    dist = lambda cx, cy: np.abs(x - cx) + np.abs(y - cy)  # noqa: E731
    sw = np.argmin(dist(xmin, ymin))
    se = np.argmin(dist(xmax, ymin))
    ne = np.argmin(dist(xmax, ymax))
    nw = np.argmin(dist(xmin, ymax))
    return np.array([w, sw, s, se, e, ne, n, nw], dtype=np.int64)


def orient(ax, ay, bx, by, px, py):
    """Twice the signed area of (a, b, p); > 0 when p is left of a->b."""
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax)


def octagon(pts, ext=None):
    """Vertex coordinates (8, 2) int64 and twice the signed area."""
    x, y = _ints(pts)
    if ext is None:
        ext = extremes(pts)
    vx, vy = x[ext], y[ext]
    area2 = int(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy))
    return np.stack([vx, vy], 1), area2


def inside_octagon(pts, ext=None) -> np.ndarray:
    """Boolean mask of the points strictly inside the octagon CP(E)."""
    x, y = _ints(pts)
    if x.size == 0:
        return np.zeros(0, bool)
    v, area2 = octagon(pts, ext)
    if area2 == 0:
        return np.zeros(x.size, bool)
    inside = np.ones(x.size, bool)
    for k in range(8):
        ax, ay = v[k]
        bx, by = v[(k + 1) % 8]
        if ax == bx and ay == by:
            continue
        inside &= orient(ax, ay, bx, by, x, y) > 0
    return inside


def regions(pts, ext=None) -> np.ndarray:
    """Queue of every point by the quadrilateral rule: 1..4, or 0 for none."""
    x, y = _ints(pts)
    if x.size == 0:
        return np.zeros(0, np.int8)
    if ext is None:
        ext = extremes(pts)
    quad = [ext[0], ext[2], ext[4], ext[6]]  # W, S, E, N
    out = np.zeros(x.size, np.int8)
    for r in range(4):
        a, b = quad[r], quad[(r + 1) % 4]
        hit = (orient(x[a], y[a], x[b], y[b], x, y) < 0) & (out == 0)
        out[hit] = r + 1
    return out


def labels(pts) -> np.ndarray:
    """The label array Q of Alg. 2: 0 = discarded, 1..4 = queue."""
    ext = extremes(pts)
    lab = regions(pts, ext)
    lab[inside_octagon(pts, ext)] = 0
    return lab


def region_counts(pts) -> np.ndarray:
    lab = labels(pts)
    return np.array([(lab == r).sum() for r in range(1, 5)], dtype=np.int64)

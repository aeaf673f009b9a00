"""Brute-force convex hull for tiny inputs.  TEST INFRASTRUCTURE ONLY.

Table I lists brute force as the simplest hull algorithm.  This version tests
every ordered pair of distinct points as a candidate counter-clockwise edge
(O(n^3) work): (i, j) is a hull edge when every point k is strictly left of
i->j or lies on the closed segment [i, j].  Walking those edges from the
lexicographically smallest point gives the strictly convex hull; points in
the interior of an edge never start an edge, so they are excluded.  It shares
no code with ``andrew.c`` and serves to pin it.
"""
from __future__ import annotations

import numpy as np


def hull(pts) -> np.ndarray:
    a = np.asarray(pts, dtype=np.float32).reshape(-1, 2)
    n = a.shape[0]
    if n == 0:
        return np.zeros(0, np.int32)
    x = a[:, 0].astype(np.int64)
    y = a[:, 1].astype(np.int64)
    # Representative of each coordinate: its lowest index.
    first = {}
    for i in range(n):
        first.setdefault((int(x[i]), int(y[i])), i)
    rep = np.array(sorted(first.values()), dtype=np.int64)
    px, py = x[rep], y[rep]
    m = rep.size
    if m == 1:
        return rep.astype(np.int32)
    # cross[i, j, k] = orientation of (p_i, p_j, p_k)
    dx = px[None, :] - px[:, None]          # (i, j): p_j - p_i
    dy = py[None, :] - py[:, None]
    kx = px[None, :] - px[:, None]          # (i, k): p_k - p_i
    ky = py[None, :] - py[:, None]
    cross = dx[:, :, None] * ky[:, None, :] - dy[:, :, None] * kx[:, None, :]
    # k on the closed segment [i, j] when collinear and within its bounding box
    lo_x = np.minimum(px[:, None], px[None, :])[:, :, None]
    hi_x = np.maximum(px[:, None], px[None, :])[:, :, None]
    lo_y = np.minimum(py[:, None], py[None, :])[:, :, None]
    hi_y = np.maximum(py[:, None], py[None, :])[:, :, None]
    on_seg = (cross == 0) & (px[None, None, :] >= lo_x) & (px[None, None, :] <= hi_x) \
        & (py[None, None, :] >= lo_y) & (py[None, None, :] <= hi_y)
    ok = np.all((cross > 0) | on_seg, axis=2)
    np.fill_diagonal(ok, False)
    start = min(range(m), key=lambda i: (px[i], py[i]))
    out = [start]
    cur = start
    for _ in range(m + 1):
        nxt = np.flatnonzero(ok[cur])
        if nxt.size == 0:
            break
        # With collinear degenerate input several j may qualify from the same
        # point; the true edge goes to the farthest one.
        far = max(nxt, key=lambda j: (px[j] - px[cur]) ** 2 + (py[j] - py[cur]) ** 2)
        if far == start:
            break
        out.append(far)
        cur = far
    return rep[np.array(out)].astype(np.int32)

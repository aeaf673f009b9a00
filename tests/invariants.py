"""Properties that determine the hull output uniquely, checkable at any size.

A list of input points that (1) is strictly convex counter-clockwise, (2)
contains every input point (inside or on the boundary), (3) starts at the
lexicographically smallest point and (4) names each coordinate by its lowest
index, is exactly the expected output.  ``check_hull`` verifies all four with
O(n log h) numpy work, so it also serves at 1e8 points.
"""
import numpy as np


def _xy(pts):
    a = np.asarray(pts, dtype=np.float32).reshape(-1, 2)
    return a[:, 0].astype(np.int64), a[:, 1].astype(np.int64)


def _cross(ox, oy, ax, ay, bx, by):
    return (ax - ox) * (by - oy) - (ay - oy) * (bx - ox)


def check_hull(pts, idx, chunk=1 << 22):
    x, y = _xy(pts)
    n = x.size
    idx = np.asarray(idx, dtype=np.int64)
    h = idx.size
    if n == 0:
        assert h == 0, "empty input must give an empty hull"
        return
    assert h >= 1, "non-empty input gives an empty hull"
    assert np.all((idx >= 0) & (idx < n)), "index out of range"
    assert np.unique(idx).size == h, "repeated index"
    hx, hy = x[idx], y[idx]
    # (3) lexicographic minimum of all points
    lx = x.min()
    ly = y[x == lx].min()
    assert hx[0] == lx and hy[0] == ly, "hull does not start at the lex-min point"
    # (4) lowest index per coordinate
    key = x * (1 << 25) + y
    hkey = hx * (1 << 25) + hy
    assert np.unique(hkey).size == h, "repeated coordinate"
    mask = np.isin(key, hkey)
    sel = np.flatnonzero(mask)
    order = np.argsort(key[sel], kind="stable")
    ks = key[sel][order]
    first = np.ones(ks.size, bool)
    first[1:] = ks[1:] != ks[:-1]
    lowest = dict(zip(ks[first].tolist(), sel[order][first].tolist()))
    for k, i in zip(hkey.tolist(), idx.tolist()):
        assert lowest[k] == i, f"vertex {i} is not the lowest index of its coordinate ({lowest[k]})"
    if h == 1:
        assert np.all((x == hx[0]) & (y == hy[0])), "single-vertex hull but points differ"
        return
    if h == 2:
        # all points collinear and between the two (lex-min, lex-max) ends
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            c = _cross(hx[0], hy[0], hx[1], hy[1], x[s:e], y[s:e])
            assert np.all(c == 0), "two-vertex hull but points are not collinear"
        kx = x * (1 << 25) + y
        assert hkey[0] == kx.min() and hkey[1] == kx.max(), "two-vertex hull must be [lex-min, lex-max]"
        return
    # (1) strict convexity, counter-clockwise
    px, py = np.roll(hx, 1), np.roll(hy, 1)
    nx, ny = np.roll(hx, -1), np.roll(hy, -1)
    turn = _cross(px, py, hx, hy, nx, ny)
    assert np.all(turn > 0), f"not strictly convex CCW at positions {np.flatnonzero(turn <= 0)[:10]}"
    # (2) containment by binary search over the fan from vertex 0
    ox, oy = hx[0], hy[0]
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        qx, qy = x[s:e], y[s:e]
        # find the largest i in [1, h-1] with cross(o, H_i, q) >= 0
        lo = np.ones(qx.size, np.int64)
        hi = np.full(qx.size, h - 1, np.int64)
        c1 = _cross(ox, oy, hx[1], hy[1], qx, qy)
        cl = _cross(ox, oy, hx[h - 1], hy[h - 1], qx, qy)
        assert np.all(c1 >= 0), "point right of the first fan edge"
        assert np.all(cl <= 0), "point left of the last fan edge"
        while True:
            active = hi - lo > 1
            if not active.any():
                break
            mid = (lo + hi) // 2
            c = _cross(ox, oy, hx[mid], hy[mid], qx, qy)
            go = c >= 0
            lo = np.where(active & go, mid, lo)
            hi = np.where(active & ~go, mid, hi)
        a = lo
        b = np.minimum(lo + 1, h - 1)
        ce = _cross(hx[a], hy[a], hx[b], hy[b], qx, qy)
        bad = ce < 0
        assert not bad.any(), f"point {s + np.flatnonzero(bad)[0]} lies outside the hull"

"""The batched path's star polygons (ch_hull_batched): dense sets of at least
32768 points get a polygon from their own points after the octagon, and sets
whose records one block still cannot hold get a second one from those
records.  Every set's hull stays bit-exact with the oracle; the per-set
counters (ch_batched_counters) show which sets took the polygon and how far
it cut their records.

The inputs stress what the polygons rely on: a centre far from the middle
of the points, arcs that do not go round the centre, gaps, duplicates of
rim points, lattice points on edges and spokes, convex position, and dense
sets next to sparse ones and to sets below the polygon's minimum size."""
import math

import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ring(n, seed, cx, cy, rx, ry, width, a0=0.0, a1=2 * math.pi):
    rng = np.random.default_rng(seed)
    th = rng.uniform(a0, a1, n)
    u = rng.uniform(0.0, width, n)
    x = np.rint(cx + (rx - u) * np.cos(th))
    y = np.rint(cy + (ry - u) * np.sin(th))
    return np.clip(np.stack([x, y], 1), 0, (1 << 24) - 1).astype(np.float32)


def _run(lib, sets):
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([s.shape[0] for s in sets])
    pts = np.ascontiguousarray(np.concatenate(sets).astype(np.float32))
    d_pts = torch.from_numpy(pts).cuda()
    d_off = torch.from_numpy(offsets).cuda()
    out_idx = torch.full((int(offsets[-1]),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((len(sets),), -99, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st = lib.load().ch_hull_batched(d_pts.data_ptr(), d_off.data_ptr(), len(sets), out_idx.data_ptr(),
                                    out_n.data_ptr(), offsets.ctypes.data, s)
    assert st == 0
    ns = out_n.cpu().tolist()
    idx = out_idx.cpu().numpy()
    for i, q in enumerate(sets):
        want = oracle.hull(q)
        assert ns[i] == want.size, i
        np.testing.assert_array_equal(idx[offsets[i]:offsets[i] + ns[i]], want, err_msg=str(i))
    return lib.ch_batched_counters(len(sets), s)


def test_dense_sets_take_the_polygon(lib):
    sets = [W.ring(400_000, 41), W.normal(300_000, 42), W.ring(40_000, 43), W.uniform(200_000, 44),
            W.ring(20_000, 45), W.distorted(250_000, 46), W.ring(1_000_000, 47)]
    c = _run(lib, sets)
    for i in (0, 2, 5, 6):   # dense, at least 32768 points
        assert c[i]["star_vertices"] > 1000, (i, c[i])
    for i in (0, 6):         # large rings: a few percent of the points reach the hull stage
        assert c[i]["records"] < sets[i].shape[0] // 10, (i, c[i])
    assert c[1]["star_vertices"] == 0 and c[3]["star_vertices"] == 0   # sparse sets keep the octagon alone
    # a ring under the first polygon's minimum size whose records one block
    # cannot hold gets its polygon from those records
    assert c[4]["star_vertices"] > 0 and c[4]["records"] <= 8192, c[4]
    assert all(x["status"] == 0 for x in c)


def test_off_centre_and_partial_rings(lib):
    sets = [_ring(300_000, 51, 2_000_000, 15_000_000, 1_900_000, 190_000, 300),     # flat ellipse near a corner
            _ring(200_000, 52, 1 << 23, 1 << 23, (1 << 23) - 2, (1 << 23) - 2, 64, 0.0, math.pi),
            _ring(200_000, 53, 1 << 23, 1 << 23, (1 << 23) - 2, (1 << 23) - 2, 64, -0.2, 0.4),
            _ring(250_000, 54, 1 << 23, 1 << 23, (1 << 23) - 2, (1 << 23) - 2, 64, 0.3, 1.9 * math.pi)]
    g = _ring(300_000, 55, 1 << 23, 1 << 23, 6_000_000, 6_000_000, 40)
    ang = np.arctan2(g[:, 1] - (1 << 23), g[:, 0] - (1 << 23))
    sets.append(g[(np.floor((ang + math.pi) / (2 * math.pi) * 12).astype(int) % 2) == 0])   # six gaps
    _run(lib, sets)


def test_duplicates_lattice_and_convex_position(lib):
    base = W.ring(120_000, 61)
    dup = np.concatenate([base, base[::-1], base[:777]])   # every rim point twice, a later copy first
    r0, r1 = 3000, 3004
    xs = np.arange(-r1, r1 + 1)
    X, Y = np.meshgrid(xs, xs)
    rr = X * X + Y * Y
    lat = np.stack([X[(rr >= r0 * r0) & (rr <= r1 * r1)], Y[(rr >= r0 * r0) & (rr <= r1 * r1)]], 1)
    lat = np.concatenate([lat] * 3) + (1 << 22)
    lat = lat[np.random.default_rng(62).permutation(lat.shape[0])].astype(np.float32)
    x = np.arange(0, 5792, dtype=np.int64)
    arc = np.stack([x * 64, x * (x + 1) // 2], 1)
    conv = np.concatenate([arc] * 8)
    conv = conv[np.random.default_rng(63).permutation(conv.shape[0])].astype(np.float32)
    c = _run(lib, [dup, W.normal(5000, 64), lat, conv, W.ring(50_000, 65)])
    assert c[0]["star_vertices"] > 0, c[0]

"""The largest inputs: one hull of CH_MAX_POINTS = 2^31 - 16 points (17 GB of
float32 pairs) through ch_hull, at an aligned and at an 8- but not 16-byte
aligned base address; and a batch of the most sets ch_hull_batched takes
(2^20), nearly all of them tiny.

It covers the streaming passes' point and tile numbering at the top of the
int32 index range, the ragged tail after the last warp tile, and the lowest
index rule (Alg. 1's output convention) for equal points that lie far apart.

For the single hull the expected result is fixed by construction.  Every
random point lies in a box strictly inside a planted polygon, so the hull of
all the points is the hull of the planted points.  The oracle computes that
hull from the planted points alone, kept in index order, so its lowest-index
rule picks the same copy as it would among all the points."""
import math

import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

C = 1 << 23                # centre of the coordinate domain [0, 2^24)
R_BOX = 1 << 22            # the random points: integers in [C - R_BOX, C + R_BOX)
R_POLY = (1 << 23) - 1000  # circumradius of the planted polygon
NEEDED_BYTES = 125 * 10**9  # points, output, the library's workspace and headroom


def _polygon(k=12, phase=0.1):
    a = phase + 2 * math.pi * np.arange(k) / k
    return np.stack([np.rint(C + R_POLY * np.cos(a)), np.rint(C + R_POLY * np.sin(a))], 1).astype(np.int64)


def _box_strictly_inside(poly):
    lo, hi = C - R_BOX, C + R_BOX - 1
    corners = [(lo, lo), (hi, lo), (hi, hi), (lo, hi)]
    k = poly.shape[0]
    for j in range(k):
        ax, ay = poly[j]
        bx, by = poly[(j + 1) % k]
        for px, py in corners:
            if (bx - ax) * (py - ay) - (by - ay) * (px - ax) <= 0:
                return False
    return True


def _expected(planted, offset, n):
    """The oracle's hull of the planted points that fall in the view
    [offset, offset + n) of the buffer, as view indices."""
    idx = np.array(sorted(i for i in planted if offset <= i < offset + n), dtype=np.int64)
    pts = np.array([planted[i] for i in idx], dtype=np.float32)
    return (idx[oracle.hull(pts)] - offset).astype(np.int64)


def test_largest_single_hull(lib):
    n = lib.CH_MAX_POINTS
    lib.ch_release()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < NEEDED_BYTES:
        pytest.skip(f"needs {NEEDED_BYTES / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")

    poly = _polygon()
    assert _box_strictly_inside(poly)
    tiles = n // 512
    tail = tiles * 512                     # first point of the ragged tail (aligned view)
    # buffer positions of the planted vertices; the buffer holds n + 1 points,
    # view A is [0, n) (aligned, no head point), view B is [1, n + 1) (one
    # head point before the first 16-byte boundary)
    where = {
        0: [0, 1],                         # A: the first point; B: its first point too
        1: [n - 1, n],                     # A: the last point; B: the last two
        2: [511, 512],                     # both sides of a warp-tile boundary
        3: [tail],                         # first point of A's tail
        4: [1000, (1 << 31) - (1 << 20)],  # equal points 2^31 apart: the lower index wins
        5: [tail - 1],                     # last point of A's last full tile
        6: [1 << 30],
        7: [(1 << 30) + 1, (1 << 30) + 7],
    }
    rng = np.random.default_rng(29)
    used = {p for ps in where.values() for p in ps}
    for v in range(8, poly.shape[0]):
        p = int(rng.integers(2, n - 1))
        while p in used:
            p = int(rng.integers(2, n - 1))
        where[v] = [p]
        used.add(p)
    planted = {p: (float(poly[v, 0]), float(poly[v, 1])) for v, ps in where.items() for p in ps}

    buf = torch.empty((n + 1, 2), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2209)
    buf.random_(C - R_BOX, C + R_BOX, generator=gen)
    pos = torch.tensor(sorted(planted), dtype=torch.int64, device="cuda")
    val = torch.tensor([planted[p] for p in sorted(planted)], dtype=torch.float32, device="cuda")
    buf[pos] = val
    out_idx = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    try:
        for offset in (0, 1):
            view = buf[offset:offset + n]
            want = _expected(planted, offset, n)
            for _ in range(2):   # the first call and a replay of its captured graph
                out_n.fill_(-99)
                lib.ch_hull(view.data_ptr(), n, out_idx.data_ptr(), out_n.data_ptr(), s)
                h = int(out_n.item())
                assert h == want.size, (offset, h, want.size)
                np.testing.assert_array_equal(out_idx[:h].cpu().numpy().astype(np.int64), want)
        assert want.size == poly.shape[0]
    finally:
        del buf, out_idx, out_n, pos, val
        torch.cuda.synchronize()
        lib.ch_release()
        torch.cuda.empty_cache()


def test_batched_largest_set_count(lib):
    """2^20 sets: empty, one-point and tiny sets on a 4 x 4 grid (duplicates
    and collinear runs everywhere, some at the top of the coordinate domain),
    every 4096th set a few thousand points of the three workload kinds, and
    rings of 40,000 points (star polygons) first, in the middle and last.
    Every set's local index list equals the oracle's."""
    k = 1 << 20
    rng = np.random.default_rng(31)
    sizes = rng.choice([0, 1, 2, 3, 4, 5, 8], size=k, p=[0.05, 0.15, 0.2, 0.2, 0.15, 0.15, 0.1])
    sets = [None] * k
    kinds = ("uniform", "normal", "ring")
    for i in range(k):
        if i in (0, k // 2, k - 1):
            sets[i] = W.make("ring", 40_000, 100 + i % 7)
        elif i % 4096 == 4095:
            sets[i] = W.make(kinds[(i // 4096) % 3], 2000 + (i // 4096) * 16, i)
        else:
            g = rng.integers(0, 4, (int(sizes[i]), 2))
            if i % 5 == 0:
                g = (1 << 24) - 1 - g   # the top corner of the domain
            sets[i] = g.astype(np.float32)
    offsets = np.zeros(k + 1, np.int64)
    offsets[1:] = np.cumsum([s.shape[0] for s in sets])
    pts = np.ascontiguousarray(np.concatenate(sets))
    d_pts = torch.from_numpy(pts).cuda()
    d_off = torch.from_numpy(offsets).cuda()
    out_idx = torch.full((int(offsets[-1]),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((k,), -99, dtype=torch.int64, device="cuda")
    st = lib.load().ch_hull_batched(d_pts.data_ptr(), d_off.data_ptr(), k, out_idx.data_ptr(), out_n.data_ptr(),
                                    offsets.ctypes.data, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    ns = out_n.cpu().numpy()
    idx = out_idx.cpu().numpy()
    bad = []
    for i in range(k):
        want = oracle.hull(sets[i])
        got = idx[offsets[i]:offsets[i] + max(int(ns[i]), 0)]
        if ns[i] != want.size or not np.array_equal(got, want):
            bad.append(i)
            if len(bad) >= 5:
                break
    assert not bad, [(i, int(ns[i]), sets[i].shape[0]) for i in bad]
    c = lib.ch_batched_counters(k, torch.cuda.current_stream().cuda_stream)
    for i in (0, k // 2, k - 1):
        assert c[i]["star_vertices"] > 0, (i, c[i])


def test_batched_largest_total(lib):
    """A batch of CH_MAX_POINTS points in all (the most one call takes),
    starting 8 bytes past a 16-byte boundary: two sets of about 2^30 points
    each (random points in a box strictly inside a planted 12-gon, copies of
    the vertices at the set's first and last points and 2^29 apart) among
    1002 tiny sets, the last of them in the batch's ragged tail.  Every set's
    local index list equals the oracle's (for the two large sets, on their
    planted points alone, as in the single-hull test)."""
    n = lib.CH_MAX_POINTS
    lib.ch_release()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < NEEDED_BYTES:
        pytest.skip(f"needs {NEEDED_BYTES / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    rng = np.random.default_rng(37)
    tiny = [rng.integers(0, 6, (int(m), 2)).astype(np.float32) for m in rng.integers(0, 9, 1002)]
    tiny[0] = np.array([[3, 3], [1, 2], [3, 3]], np.float32)
    tiny[-1] = np.array([[7, 1], [2, 9]], np.float32)
    n_tiny = sum(t.shape[0] for t in tiny)
    n_a = (1 << 30) + 3
    n_b = n - n_a - n_tiny
    # set order: tiny[0], A, tiny[1..1000], B, tiny[1001]
    sizes = [tiny[0].shape[0], n_a] + [t.shape[0] for t in tiny[1:-1]] + [n_b, tiny[-1].shape[0]]
    k = len(sizes)
    offsets = np.zeros(k + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    assert offsets[-1] == n
    ia, ib = 1, k - 2
    poly = _polygon()
    assert _box_strictly_inside(poly)
    planted = {}
    for set_i, extra in ((ia, 0), (ib, 5)):
        m = sizes[set_i]
        where = [[0, 1 << 29], [m - 1], [511 - extra], [m // 2, m // 2 + 1]]
        used = {p for ps in where for p in ps}
        while len(where) < poly.shape[0]:
            p = int(rng.integers(2, m - 2))
            if p not in used:
                where.append([p])
                used.add(p)
        planted[set_i] = {p: (float(poly[v, 0]), float(poly[v, 1])) for v, ps in enumerate(where) for p in ps}

    buf = torch.empty((n + 1, 2), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2210)
    buf.random_(C - R_BOX, C + R_BOX, generator=gen)
    view = buf[1:]   # 8 bytes past a 16-byte boundary: one head point
    tiny_sets = [0] + list(range(2, k - 2)) + [k - 1]
    for t, set_i in zip(tiny, tiny_sets):
        if t.shape[0]:
            view[int(offsets[set_i]):int(offsets[set_i + 1])] = torch.from_numpy(t).cuda()
    for set_i, pl in planted.items():
        pos = torch.tensor([int(offsets[set_i]) + p for p in sorted(pl)], dtype=torch.int64, device="cuda")
        view[pos] = torch.tensor([pl[p] for p in sorted(pl)], dtype=torch.float32, device="cuda")
    d_off = torch.from_numpy(offsets).cuda()
    out_idx = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((k,), -99, dtype=torch.int64, device="cuda")
    try:
        st = lib.load().ch_hull_batched(view.data_ptr(), d_off.data_ptr(), k, out_idx.data_ptr(), out_n.data_ptr(),
                                        offsets.ctypes.data, torch.cuda.current_stream().cuda_stream)
        assert st == 0
        ns = out_n.cpu().numpy()
        for set_i in range(k):
            if set_i in planted:
                pl = planted[set_i]
                idx = np.array(sorted(pl), dtype=np.int64)
                want = idx[oracle.hull(np.array([pl[p] for p in idx], np.float32))]
            else:
                want = oracle.hull(tiny[tiny_sets.index(set_i)])
            o = int(offsets[set_i])
            assert ns[set_i] == want.size, (set_i, int(ns[set_i]), want.size)
            got = out_idx[o:o + want.size].cpu().numpy().astype(np.int64)
            np.testing.assert_array_equal(got, want, err_msg=str(set_i))
        assert planted[ia] and ns[ia] == poly.shape[0] and ns[ib] == poly.shape[0]
    finally:
        del buf, view, d_off, out_idx, out_n
        torch.cuda.synchronize()
        lib.ch_release()
        torch.cuda.empty_cache()

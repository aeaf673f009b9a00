"""ch_hull_noalloc, the allocation-free entry point, called through the C ABI.

Each call must give exactly what ch_hull gives on the same points (hull
indices are integers: the tolerance is equality), on two calls in a row with
different inputs, and sizes beyond its fixed scratch are refused up front.
Named to run last, after every other GPU test, and passes alone as well."""
import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_POINTS = 8000   # CH_NOALLOC_MAX_POINTS in ch.h


def _run(fn, pts, n):
    out_idx = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    st = fn(pts.data_ptr(), n, out_idx.data_ptr(), out_n.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, st
    torch.cuda.synchronize()
    h = int(out_n.item())
    return h, out_idx[:max(h, 0)].cpu().numpy()


def _same_as_ch_hull(native, host_pts):
    n = host_pts.shape[0]
    pts = torch.from_numpy(np.ascontiguousarray(host_pts, dtype=np.float32)).cuda()
    want = _run(native.ch_hull, pts, n)
    got = _run(native.ch_hull_noalloc, pts, n)
    assert got[0] == want[0]
    np.testing.assert_array_equal(got[1], want[1])
    return got


def test_two_calls_in_a_row_match_ch_hull(lib):
    native = lib.load()
    a = W.make("normal", MAX_POINTS, 31)
    b = W.make("ring", 5003, 32)
    ha = _same_as_ch_hull(native, a)
    hb = _same_as_ch_hull(native, b)
    np.testing.assert_array_equal(ha[1], oracle.hull(a))
    np.testing.assert_array_equal(hb[1], oracle.hull(b))


def _u_arc(m, seed):
    """m lattice points in strictly convex position (a narrow U, slopes -m/2 ..
    m/2, x step 1500), shuffled: every point is a hull vertex."""
    i = np.arange(m, dtype=np.int64)
    y = np.concatenate([[0], np.cumsum(i[:-1] - m // 2)])
    pts = np.stack([i * 1500, y - y.min() + 5], 1)
    return pts[np.random.default_rng(seed).permutation(m)].astype(np.float32)


def _parabola(m, seed):
    """m points of y = x (x + 1) / 2, x step 64 (m <= 5792 keeps y < 2^24),
    shuffled, plus a copy of every tenth point at the end: all hull vertices,
    each duplicate named by its first index."""
    x = np.arange(m, dtype=np.int64)
    pts = np.stack([x * 64, x * (x + 1) // 2], 1)[np.random.default_rng(seed).permutation(m)]
    return np.concatenate([pts, pts[::10]]).astype(np.float32)


def test_all_points_on_the_hull_take_the_sort_fallback(lib):
    """Sets whose hull has thousands of vertices overflow the one-block
    quickhull's chain capacity, so the kernel sorts its records in the static
    scratch and joins the chains from there (the branch no smaller hull
    reaches).  Two different such sets in a row, each against ch_hull and the
    oracle."""
    native = lib.load()
    a = _u_arc(MAX_POINTS, 41)
    b = _parabola(5000, 42)
    assert b.shape[0] <= MAX_POINTS
    for pts in (a, b, a):
        want = oracle.hull(pts)
        assert want.size >= 5000
        got = _same_as_ch_hull(native, pts)
        np.testing.assert_array_equal(got[1], want)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 17, 512, 4097, MAX_POINTS])
def test_sizes_match_ch_hull(lib, n):
    rng = np.random.default_rng(n + 5)
    _same_as_ch_hull(lib.load(), rng.integers(0, 1 << 24, (n, 2)).astype(np.float32))


@pytest.mark.parametrize("name", ["identical", "horizontal", "diagonal", "square_extremes", "dense_duplicates",
                                  "collinear_plus_one"])
def test_degenerate_inputs_match_ch_hull(lib, name):
    pts = W.degenerate_suite()[name]
    if pts.shape[0] <= MAX_POINTS:
        _same_as_ch_hull(lib.load(), pts)


def test_bad_coordinate_reports_erange(lib):
    pts = W.uniform(1000, 7)
    pts[10, 0] = 0.5
    h, _ = _run(lib.load().ch_hull_noalloc, torch.from_numpy(pts).cuda(), pts.shape[0])
    assert h == lib.CH_ERANGE


def test_larger_than_scratch_is_refused(lib):
    native = lib.load()
    pts = torch.zeros((MAX_POINTS + 1, 2), dtype=torch.float32, device="cuda")
    out_idx = torch.zeros(MAX_POINTS + 1, dtype=torch.int32, device="cuda")
    out_n = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    st = native.ch_hull_noalloc(pts.data_ptr(), MAX_POINTS + 1, out_idx.data_ptr(), out_n.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == lib.CH_EINVAL
    torch.cuda.synchronize()
    assert int(out_n.item()) == -99   # nothing was enqueued

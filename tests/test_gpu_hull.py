"""Parity of the CUDA hull (through the C ABI) with the CPU oracle: bit-exact
index lists on seeded workloads at sizes spanning many tiles with ragged
tails, on the degenerate suite, on lattice polygons, and on misaligned input."""
import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests import golden_io
from tests.invariants import check_hull

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_hull(ch, pts, offset_points=0):
    """Run ch_hull on pts; offset_points > 0 places the points at a base
    address that is 8- but not 16-byte aligned."""
    n = pts.shape[0]
    buf = torch.zeros((n + offset_points, 2), dtype=torch.float32, device="cuda")
    buf[offset_points:] = torch.from_numpy(pts).cuda()
    view = buf[offset_points:]
    out_idx = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    ch.ch_hull(view.data_ptr(), n, out_idx.data_ptr(), out_n.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
    h = int(out_n.item())
    return h, out_idx[:max(h, 0)].cpu().numpy()


def assert_same(ch, pts, offset_points=0):
    h, got = gpu_hull(ch, pts, offset_points)
    want = oracle.hull(pts)
    assert h == want.size, f"size {h} != {want.size}"
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("kind,n,seed", [
    ("uniform", 1_000_000, 0),           # the uniform 1e6 workload exactly
    ("normal", 2_000_003, 1),
    ("ring", 1_000_001, 2),
    ("normal", 4097, 5),
    ("ring", 70_000, 6),
    ("uniform", 513, 7),
    ("uniform", 511, 8),
    ("ring", 4096 * 3 + 17, 9),
    ("distorted", 1_000_003, 5),         # the circumference with 2% distortion
    ("distorted", 30_000, 10),
])
def test_hull_matches_oracle(lib, kind, n, seed):
    assert_same(lib, W.make(kind, n, seed))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 255, 256, 257, 1023, 1024, 1025, 3000])
@pytest.mark.parametrize("misaligned", [0, 1])
def test_small_and_ragged_sizes(lib, n, misaligned):
    rng = np.random.default_rng(n)
    pts = rng.integers(0, 1 << 24, (n, 2)).astype(np.float32)
    assert_same(lib, pts, misaligned)
    dup = rng.integers(0, 6, (n, 2)).astype(np.float32)
    assert_same(lib, dup, misaligned)


@pytest.mark.parametrize("name", list(W.degenerate_suite().keys()))
def test_degenerate_suite(lib, name):
    pts = W.degenerate_suite()[name]
    assert_same(lib, pts)
    assert_same(lib, pts, 1)


@pytest.mark.parametrize("name", golden_io.FIXTURES)
def test_lattice_polygons(lib, name):
    pts, expected = golden_io.load(name, offset=1 << 23)
    h, got = gpu_hull(lib, pts)
    np.testing.assert_array_equal(got, expected)


def test_large_duplicate_runs(lib):
    # runs of equal queue key longer than a sort/chain tile
    rng = np.random.default_rng(3)
    base = rng.integers(0, 1 << 24, (2000, 2))
    pts = np.repeat(base, 37, axis=0)
    rng.shuffle(pts)
    corner = np.array([[0, 0]] * 10000 + [[1 << 23, 0]] * 9000)
    pts = np.concatenate([pts, corner, pts[:5000]]).astype(np.float32)
    assert_same(lib, pts)


def test_points_in_convex_position(lib):
    # every point is a hull vertex: parabola lattice points
    x = np.arange(0, 4000, dtype=np.int64)
    y = (x - 2000) ** 2 // 4 + 10
    pts = np.stack([x * 4000, y], 1)
    pts = np.concatenate([pts, np.stack([x * 4000, np.full_like(x, 16_000_000)], 1)])
    rng = np.random.default_rng(1)
    pts = pts[rng.permutation(pts.shape[0])].astype(np.float32)
    assert_same(lib, pts)


def test_out_of_domain_reports_erange(lib):
    pts = W.uniform(10_000, 1)
    for bad in (np.nan, -1.0, 0.5, 16777216.0, np.inf):
        p = pts.copy()
        p[1234, 1] = bad
        h, _ = gpu_hull(lib, p)
        assert h == lib.CH_ERANGE


def test_workspace_reuse_and_determinism(lib):
    pts = W.ring(300_000, 12)
    small = W.normal(1000, 3)
    a = gpu_hull(lib, pts)[1]
    b = gpu_hull(lib, small)[1]
    c = gpu_hull(lib, pts)[1]
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(b, oracle.hull(small))
    for _ in range(5):
        np.testing.assert_array_equal(gpu_hull(lib, pts)[1], a)


def test_metamorphic_translation(lib):
    pts = W.ring(200_000, 4).astype(np.int64) // 2
    a = gpu_hull(lib, pts.astype(np.float32))[1]
    b = gpu_hull(lib, (pts + [12345, 6789]).astype(np.float32))[1]
    np.testing.assert_array_equal(a, b)


def test_host_entry_point(lib):
    import ctypes
    pts = np.ascontiguousarray(W.normal(500_000, 2))
    out = np.empty(pts.shape[0], np.int32)
    n = ctypes.c_int64()
    lib.ch_hull_host(pts.ctypes.data, pts.shape[0], out.ctypes.data, ctypes.addressof(n), 0)
    np.testing.assert_array_equal(out[:n.value], oracle.hull(pts))


def test_tensor_helper(lib):
    pts = W.uniform(100_000, 3)
    got = lib.hull(torch.from_numpy(pts).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.hull(pts))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["normal_1e8", "ring_1e8", "distorted_1e8"])
def test_full_size_workloads(lib, name):
    """The 1e8-point normal, ring and distorted workloads in the benchmark's launch shape,
    checked bit-exactly against the oracle and by the defining invariants."""
    pts = W.single(name)
    h, got = gpu_hull(lib, pts)
    want = oracle.hull(pts)
    np.testing.assert_array_equal(got, want)
    check_hull(pts, got)


def test_repeated_calls_replay_graph(lib):
    """Calls repeated with the same buffers replay a cached CUDA graph; the
    results must follow the current contents of the buffers, and a larger
    call on the same stream (workspace regrowth) must stay correct."""
    stream = torch.cuda.Stream()
    a = W.normal(300_000, 21)
    b = W.ring(300_000, 22)
    pts = torch.from_numpy(a).cuda()
    out_idx = torch.empty(pts.shape[0], dtype=torch.int32, device="cuda")
    out_n = torch.empty(1, dtype=torch.int64, device="cuda")
    want_a, want_b = oracle.hull(a), oracle.hull(b)
    with torch.cuda.stream(stream):
        for rep in range(6):
            src = a if rep % 2 == 0 else b
            pts.copy_(torch.from_numpy(src).cuda())
            lib.ch_hull(pts.data_ptr(), pts.shape[0], out_idx.data_ptr(), out_n.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            h = int(out_n.item())
            np.testing.assert_array_equal(out_idx[:h].cpu().numpy(), want_a if rep % 2 == 0 else want_b)
        big = W.uniform(2_000_000, 23)
        got = lib.hull(torch.from_numpy(big).cuda(), stream=stream).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.hull(big))


def _u_arc(m, seed):
    """m lattice points in strictly convex position forming a narrow U (slopes
    -m/2 .. m/2): near the bottom the points crowd into a few u-buckets, whose
    chains overflow, so the call takes the radix-sort fallback."""
    i = np.arange(m, dtype=np.int64)
    s = i - m // 2
    y = np.concatenate([[0], np.cumsum(s[:-1])])
    pts = np.stack([i * 1500, y - y.min() + 5], 1)
    rng = np.random.default_rng(seed)
    return pts[rng.permutation(m)].astype(np.float32)


def test_sort_fallback_when_bucket_chains_overflow(lib):
    pts = _u_arc(11_000, 1)
    assert oracle.hull(pts).size == pts.shape[0]
    assert_same(lib, pts)
    # a repeat replays the captured graph, through its conditional node
    assert_same(lib, pts)

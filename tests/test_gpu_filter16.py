"""Parity of ch_filter16 (the filter with the 16-direction polygon) with its
numpy definition: the 16 extreme indices, the label array and the queue
sizes, bit-exact."""
import numpy as np
import pytest

from oracle import filter16_ref as G
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_filter16(ch, pts, misaligned=0, labels=True):
    n = pts.shape[0]
    buf = torch.zeros((n + misaligned, 2), dtype=torch.float32, device="cuda")
    buf[misaligned:] = torch.from_numpy(pts).cuda()
    v = buf[misaligned:]
    ext = torch.empty(16, dtype=torch.int32, device="cuda")
    lab = torch.full((max(n, 1),), 255, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(4, dtype=torch.int64, device="cuda")
    ch.ch_filter16(v.data_ptr(), n, ext.data_ptr(), lab.data_ptr() if labels else None, cnt.data_ptr(),
                   torch.cuda.current_stream().cuda_stream)
    return ext.cpu().numpy(), lab[:n].cpu().numpy(), cnt.cpu().numpy()


CASES = [("normal", 1_000_037, 1), ("distorted", 300_000, 5), ("ring", 300_000, 2),
         ("uniform", 1_000_000, 0), ("normal", 513, 3), ("uniform", 7, 4)]


@pytest.mark.parametrize("kind,n,seed", CASES)
@pytest.mark.parametrize("misaligned", [0, 1])
def test_filter16_matches_definition(lib, kind, n, seed, misaligned):
    pts = W.make(kind, n, seed)
    ext, lab, cnt = gpu_filter16(lib, pts, misaligned)
    np.testing.assert_array_equal(ext, G.extremes16(pts))
    want = G.labels16(pts)
    np.testing.assert_array_equal(lab, want)
    np.testing.assert_array_equal(cnt, [(want == r).sum() for r in range(1, 5)])


@pytest.mark.parametrize("name", [k for k, v in W.degenerate_suite().items() if v.shape[0] > 0])
def test_filter16_degenerate(lib, name):
    pts = W.degenerate_suite()[name]
    ext, lab, cnt = gpu_filter16(lib, pts)
    np.testing.assert_array_equal(ext, G.extremes16(pts))
    np.testing.assert_array_equal(lab, G.labels16(pts))


def test_filter16_ties_lowest_index(lib):
    # exact ties in every direction, spread over the array and over blocks
    rng = np.random.default_rng(1)
    pts = rng.integers(100, 200, (400_000, 2))
    for j, (x, y) in enumerate([(100, 100), (199, 199), (100, 199), (199, 100), (150, 100), (100, 150)]):
        pts[j::991 + 2 * j] = [x, y]
    pts = pts.astype(np.float32)
    ext, lab, _ = gpu_filter16(lib, pts)
    np.testing.assert_array_equal(ext, G.extremes16(pts))
    np.testing.assert_array_equal(lab, G.labels16(pts))


def test_filter16_even_directions_equal_ch_filter(lib):
    pts = W.normal(200_000, 9)
    ext16, _, _ = gpu_filter16(lib, pts)
    v = torch.from_numpy(pts).cuda()
    ext8 = torch.empty(8, dtype=torch.int32, device="cuda")
    lib.ch_filter(v.data_ptr(), pts.shape[0], ext8.data_ptr(), None, None, torch.cuda.current_stream().cuda_stream)
    np.testing.assert_array_equal(ext16[0::2], ext8.cpu().numpy())


def test_filter16_counts_without_labels(lib):
    pts = W.distorted(100_000, 6)
    ext, _, cnt = gpu_filter16(lib, pts, labels=False)
    np.testing.assert_array_equal(cnt, G.region_counts16(pts))


def test_filter16_empty(lib):
    ext = torch.zeros(16, dtype=torch.int32, device="cuda")
    cnt = torch.ones(4, dtype=torch.int64, device="cuda")
    lib.ch_filter16(8, 0, ext.data_ptr(), None, cnt.data_ptr(), 0)
    torch.cuda.synchronize()
    assert ext.cpu().tolist() == [-1] * 16
    assert cnt.cpu().tolist() == [0] * 4


@pytest.mark.parametrize("bad", [0.5, float(1 << 24), -1.0, float("nan")])
def test_filter16_rejects_bad_coordinates(lib, bad):
    pts = W.uniform(10_000, 7)
    pts[4321, 1] = bad
    ext, _, cnt = gpu_filter16(lib, pts)
    assert ext.tolist() == [-1] * 16
    assert cnt.tolist() == [lib.CH_ERANGE] * 4

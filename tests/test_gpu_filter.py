"""Parity of the CUDA filter stage with the numpy definition of Alg. 2:
the 8 extreme indices, the label array Q, and the queue sizes (bit-exact)."""
import numpy as np
import pytest

from oracle import filter_ref as F
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_filter(ch, pts, misaligned=0, fn="ch_filter"):
    n = pts.shape[0]
    buf = torch.zeros((n + misaligned, 2), dtype=torch.float32, device="cuda")
    buf[misaligned:] = torch.from_numpy(pts).cuda()
    v = buf[misaligned:]
    ext = torch.empty(8, dtype=torch.int32, device="cuda")
    lab = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    cnt = torch.empty(4, dtype=torch.int64, device="cuda")
    getattr(ch, fn)(v.data_ptr(), n, ext.data_ptr(), lab.data_ptr(), cnt.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    return ext.cpu().numpy(), lab[:n].cpu().numpy(), cnt.cpu().numpy()


CASES = [("normal", 1_000_000, 1), ("ring", 300_000, 2), ("uniform", 1_000_000, 0),
         ("normal", 513, 3), ("uniform", 7, 4)]


FILTERS = ["ch_filter", "ch_filter_manhattan"]


@pytest.mark.parametrize("fn", FILTERS)
@pytest.mark.parametrize("kind,n,seed", CASES)
@pytest.mark.parametrize("misaligned", [0, 1])
def test_filter_matches_definition(lib, kind, n, seed, misaligned, fn):
    pts = W.make(kind, n, seed)
    ext, lab, cnt = gpu_filter(lib, pts, misaligned, fn)
    np.testing.assert_array_equal(ext, F.extremes(pts))
    if fn == "ch_filter_manhattan":   # the paper's two-step form, written out in the oracle
        np.testing.assert_array_equal(ext, F.extremes_manhattan(pts))
    want = F.labels(pts)
    np.testing.assert_array_equal(lab, want)
    np.testing.assert_array_equal(cnt, [(want == r).sum() for r in range(1, 5)])


@pytest.mark.parametrize("fn", FILTERS)
@pytest.mark.parametrize("name", [k for k, v in W.degenerate_suite().items() if v.shape[0] > 0])
def test_filter_degenerate(lib, name, fn):
    pts = W.degenerate_suite()[name]
    ext, lab, cnt = gpu_filter(lib, pts, 0, fn)
    np.testing.assert_array_equal(ext, F.extremes(pts))
    np.testing.assert_array_equal(lab, F.labels(pts))


@pytest.mark.parametrize("fn", FILTERS)
def test_filter_ties_lowest_index(lib, fn):
    # many exact ties on every extreme direction, far apart in the array
    rng = np.random.default_rng(0)
    pts = rng.integers(100, 200, (300_000, 2))
    pts[::1000] = [100, 100]
    pts[5::997] = [199, 199]
    pts[7::991] = [100, 199]
    pts[11::983] = [199, 100]
    pts = pts.astype(np.float32)
    ext, lab, cnt = gpu_filter(lib, pts, 0, fn)
    np.testing.assert_array_equal(ext, F.extremes(pts))
    np.testing.assert_array_equal(lab, F.labels(pts))


@pytest.mark.parametrize("fn", FILTERS)
def test_filter_empty(lib, fn):
    ext = torch.zeros(8, dtype=torch.int32, device="cuda")
    cnt = torch.ones(4, dtype=torch.int64, device="cuda")
    getattr(lib, fn)(8, 0, ext.data_ptr(), None, cnt.data_ptr(), 0)
    assert ext.cpu().tolist() == [-1] * 8
    assert cnt.cpu().tolist() == [0] * 4


def test_manhattan_reports_erange(lib):
    pts = W.uniform(100_000, 5)
    pts[777, 0] = 2.5
    ext, lab, cnt = gpu_filter(lib, pts, 0, "ch_filter_manhattan")
    assert ext.tolist() == [-1] * 8
    assert cnt.tolist() == [lib.CH_ERANGE] * 4

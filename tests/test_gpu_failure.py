"""Failure detection on the GPU without a fault: the library's bounded device
waits, made to run out on purpose (a flag nothing sets, a copy barrier with
no copy), give up with CH_ETIMEOUT; the context stays usable afterwards."""
import time

import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1], ids=["lookback_poll", "copy_barrier"])
def test_bounded_wait_gives_up_and_context_survives(lib, which):
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    st = lib.load().ch_selftest_timeout(which, stream)
    elapsed = time.perf_counter() - t0
    assert st == lib.CH_ETIMEOUT, lib.ch_strerror(st)
    assert elapsed < 30.0
    # the context is intact: a hull right after matches the oracle
    pts = W.normal(200_000, 3)
    got = lib.hull(torch.from_numpy(pts).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.hull(pts))


def test_selftest_rejects_unknown_wait(lib):
    assert lib.load().ch_selftest_timeout(7, torch.cuda.current_stream().cuda_stream) == lib.CH_EINVAL

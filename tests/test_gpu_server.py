"""Continuous-batching server: each request's result equals the oracle (and
ch_hull) whether it runs alone or in a mix of concurrent requests; admission
and ticket errors are reported with status codes."""
import time

import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _wait(lib, srv, tickets, caps, timeout=120.0):
    out = {}
    t0 = time.time()
    pending = set(tickets)
    while pending and time.time() - t0 < timeout:
        for t in list(pending):
            buf = np.empty(max(caps[t], 1), np.int32)
            st, n = lib.ch_poll(srv, t, buf.ctypes.data, caps[t])
            if st == lib.CH_PENDING:
                continue
            assert st == lib.CH_OK, lib.ch_strerror(st)
            out[t] = buf[:n].copy()
            pending.discard(t)
        time.sleep(0.001)
    assert not pending, f"{len(pending)} requests not served in time"
    return out


def test_server_mix_matches_oracle(lib):
    srv = lib.ch_server_create(2 << 30, 0)
    try:
        plan_sizes = [1000, 250_000, 3, 70_000, 1_000_000, 5000, 12, 400_000, 999, 150_000] * 3
        kinds = ["normal", "uniform", "ring"]
        reqs = [np.ascontiguousarray(W.make(kinds[i % 3], n, 100 + i)) for i, n in enumerate(plan_sizes)]
        tickets, caps = [], {}
        for i, p in enumerate(reqs):
            st, t = lib.ch_submit(srv, p.ctypes.data, p.shape[0])
            assert st == lib.CH_OK
            tickets.append(t)
            caps[t] = p.shape[0]
            if i % 7 == 0:
                time.sleep(0.002)   # arrivals while earlier batches run
        res = _wait(lib, srv, tickets, caps)
        for t, p in zip(tickets, reqs):
            np.testing.assert_array_equal(res[t], oracle.hull(p))
        # alone: the same request submitted by itself gives the same answer
        p = reqs[4]
        st, t = lib.ch_submit(srv, p.ctypes.data, p.shape[0])
        alone = _wait(lib, srv, [t], {t: p.shape[0]})[t]
        np.testing.assert_array_equal(alone, res[tickets[4]])
        stats = lib.ch_server_stats(srv)
        assert stats["completed"] == len(reqs) + 1
        assert stats["p99_ms"] >= stats["p50_ms"] > 0
        # the per-batch trace accounts for every request and point
        trace = lib.ch_server_trace(srv)
        assert sum(b[1] for b in trace) == len(reqs) + 1
        assert sum(b[2] for b in trace) == sum(p.shape[0] for p in reqs) + p.shape[0]
        for b in trace:
            assert b[1] >= 1 and min(b[3], b[4], b[5]) >= 0.0 and b[6] > 0.0
    finally:
        lib.ch_server_destroy(srv)


def test_server_errors(lib):
    srv = lib.ch_server_create(256 << 20, 0)
    try:
        st, _ = lib.ch_poll(srv, 987654321, None, 0)
        assert st == lib.CH_EINVAL
        # a request that can never fit the budget is refused before it is read
        st, _ = lib.ch_submit(srv, 4096, 100_000_000)
        assert st == lib.CH_ENOMEM
        bad = np.array([[1.5, 2.0], [3.0, 4.0], [5.0, 1.0]], np.float32)
        st, t = lib.ch_submit(srv, bad.ctypes.data, 3)
        assert st == lib.CH_OK
        t0 = time.time()
        while True:
            buf = np.empty(3, np.int32)
            st, n = lib.ch_poll(srv, t, buf.ctypes.data, 3)
            if st != lib.CH_PENDING or time.time() - t0 > 30:
                break
            time.sleep(0.001)
        assert st == lib.CH_ERANGE and n == lib.CH_ERANGE
    finally:
        lib.ch_server_destroy(srv)


def _convex_position(m, seed):
    """m lattice points that are all hull vertices (a strictly convex arc),
    shuffled: bucket chains overflow and the set takes the single-hull path."""
    x = np.arange(m, dtype=np.int64)
    y = x * (x + 1) // 2   # strictly convex: the slopes x + 1 increase (m <= 5792 keeps y < 2^24)
    pts = np.stack([x * 64, y], 1)
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(pts[rng.permutation(m)].astype(np.float32))


def test_server_set_left_to_single_hull_path(lib):
    """A request whose bucket chains overflow is finished by the single-hull
    path after the batch (no host wait inside the batch), in a mix."""
    srv = lib.ch_server_create(2 << 30, 0)
    try:
        conv = _convex_position(5000, 3)
        assert oracle.hull(conv).size == conv.shape[0]
        reqs = [np.ascontiguousarray(W.normal(20_000, 5)), conv, np.ascontiguousarray(W.ring(30_000, 6)), conv]
        tickets, caps = [], {}
        for p in reqs:
            st, t = lib.ch_submit(srv, p.ctypes.data, p.shape[0])
            assert st == lib.CH_OK
            tickets.append(t)
            caps[t] = p.shape[0]
        res = _wait(lib, srv, tickets, caps)
        for t, p in zip(tickets, reqs):
            np.testing.assert_array_equal(res[t], oracle.hull(p))
    finally:
        lib.ch_server_destroy(srv)


def test_submit_reads_the_buffer_until_poll_answers(lib):
    """ch_submit does not copy: the buffer is read when the request joins a
    batch.  Once ch_poll has answered, the caller may reuse the buffer: the
    same buffer refilled with other points gives that set's hull."""
    srv = lib.ch_server_create(1 << 30, 0)
    try:
        buf = np.ascontiguousarray(W.ring(200_000, 31))
        first = buf.copy()
        st, t = lib.ch_submit(srv, buf.ctypes.data, buf.shape[0])
        assert st == lib.CH_OK
        got1 = _wait(lib, srv, [t], {t: buf.shape[0]})[t]
        buf[:] = W.normal(200_000, 32)   # reuse after the answer
        st, t2 = lib.ch_submit(srv, buf.ctypes.data, buf.shape[0])
        assert st == lib.CH_OK
        got2 = _wait(lib, srv, [t2], {t2: buf.shape[0]})[t2]
        np.testing.assert_array_equal(got1, oracle.hull(first))
        np.testing.assert_array_equal(got2, oracle.hull(buf))
    finally:
        lib.ch_server_destroy(srv)

"""Whole workload configurations against the oracle, through the C ABI.

* the batched configuration exactly as the benchmark runs it: 4096 sets of
  log-uniform size in [100, 1e6] drawn from the uniform / normal / ring
  generators (seed 3), one ch_hull_batched call, every set's local index
  list equal to the oracle's hull of that set;
* a served mix drawn from the serving configuration's own plan (Poisson
  arrivals, sizes log-uniform in [1e3, 1e7], 50% normal / 40% uniform / 10%
  ring), every request with its own points, submitted at its arrival time
  into a server with the configuration's 16 GB budget, each result equal to
  the oracle's;
* the radix-sort fallback of the single hull (taken when a bucket chain
  overflows) on input full of duplicate hull vertices, interior duplicates
  and collinear boundary runs, where its run de-duplication of equal
  (queue, u) keys decides which index names a vertex.

The oracle runs in host threads (its C code releases the GIL), so the
comparison of 4.4e8 points takes seconds on a many-core host."""
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle_many(sets):
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(oracle.hull, sets))


@pytest.mark.slow
def test_batched_configuration_matches_oracle_set_by_set(lib):
    pts, off = W.batched(4096)
    k = off.size - 1
    d_pts = torch.from_numpy(pts).cuda()
    d_off = torch.from_numpy(off).cuda()
    out_idx = torch.full((int(off[-1]),), -7, dtype=torch.int32, device="cuda")
    out_n = torch.full((k,), -99, dtype=torch.int64, device="cuda")
    st = lib.load().ch_hull_batched(d_pts.data_ptr(), d_off.data_ptr(), k, out_idx.data_ptr(), out_n.data_ptr(),
                                    off.ctypes.data, torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.ch_strerror(st)
    ns = out_n.cpu().numpy()
    idx = out_idx.cpu().numpy()
    del d_pts, out_idx
    want = _oracle_many([pts[off[i]:off[i + 1]] for i in range(k)])
    bad = [i for i in range(k)
           if ns[i] != want[i].size or not np.array_equal(idx[off[i]:off[i] + ns[i]], want[i])]
    assert not bad, f"{len(bad)} of {k} sets differ, first {bad[:5]}"


@pytest.mark.slow
def test_served_mix_from_the_serving_plan_matches_oracle(lib):
    arrivals, sizes, names = W.serving_plan()
    r = 240   # the plan's first requests: about 2.6e8 points, sizes up to ~1e7
    reqs = [np.ascontiguousarray(W.make(str(names[i]), int(sizes[i]), 7000 + i)) for i in range(r)]
    assert max(int(s) for s in sizes[:r]) > 5_000_000
    srv = lib.ch_server_create(16 << 30, 0)
    try:
        tickets = []
        t0 = time.perf_counter()
        for i in range(r):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            while True:
                st, t = lib.ch_submit(srv, reqs[i].ctypes.data, reqs[i].shape[0])
                if st != lib.CH_EBUSY:
                    break
                time.sleep(0.0005)
            assert st == lib.CH_OK, lib.ch_strerror(st)
            tickets.append(t)
        got = {}
        deadline = time.time() + 300
        pending = set(range(r))
        while pending and time.time() < deadline:
            for i in list(pending):
                buf = np.empty(max(reqs[i].shape[0], 1), np.int32)
                st, h = lib.ch_poll(srv, tickets[i], buf.ctypes.data, reqs[i].shape[0])
                if st == lib.CH_PENDING:
                    continue
                assert st == lib.CH_OK, lib.ch_strerror(st)
                got[i] = buf[:h].copy()
                pending.discard(i)
            time.sleep(0.001)
        assert not pending, f"{len(pending)} requests not served"
    finally:
        lib.ch_server_destroy(srv)
    want = _oracle_many(reqs)
    bad = [i for i in range(r) if not np.array_equal(got[i], want[i])]
    assert not bad, f"{len(bad)} of {r} requests differ, first {bad[:5]}"


def _u_arc_with_runs(m, seed):
    """A narrow U of m lattice points in strictly convex position (slopes
    -m/2 .. m/2, x step 1500: its bucket chains overflow, so the single hull
    takes the radix-sort fallback), with
      * every fifth vertex repeated three more times at shuffled positions
        (a later copy must never name the vertex),
      * interior points just above the arc, some of them repeated,
      * lattice points on the closing chord between the two end vertices
        (collinear boundary points, excluded from the hull), and
      * extra copies of both end vertices."""
    i = np.arange(m, dtype=np.int64)
    y = np.concatenate([[0], np.cumsum(i[:-1] - m // 2)])
    arc = np.stack([i * 1500, y - y.min() + 5], 1)
    rng = np.random.default_rng(seed)
    dups = np.repeat(arc[::5], 3, axis=0)
    above = arc[1:-1:3] + np.array([0, 7])
    inner = np.concatenate([above, above[::4]])
    a, b = arc[0], arc[-1]
    g = int(np.gcd(abs(int(b[0] - a[0])), abs(int(b[1] - a[1]))))
    steps = np.arange(1, g, max(1, g // 200))
    chord = a + np.outer(steps, (b - a) // g)
    ends = np.array([a, b, a, b])
    pts = np.concatenate([arc, dups, inner, chord, ends])
    return pts[rng.permutation(pts.shape[0])].astype(np.float32)


def test_sort_fallback_with_duplicate_and_collinear_runs(lib):
    for m, seed in ((11_000, 1), (10_501, 2)):
        pts = _u_arc_with_runs(m, seed)
        want = oracle.hull(pts)
        assert want.size == m   # the arc's vertices, each named once
        d = torch.from_numpy(pts).cuda()
        out_idx = torch.full((pts.shape[0],), -7, dtype=torch.int32, device="cuda")
        out_n = torch.full((1,), -99, dtype=torch.int64, device="cuda")
        for _ in range(2):   # direct launch, then the captured graph's replay
            lib.ch_hull(d.data_ptr(), pts.shape[0], out_idx.data_ptr(), out_n.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
            h = int(out_n.item())
            assert h == want.size
            np.testing.assert_array_equal(out_idx[:h].cpu().numpy(), want)
            c = lib.ch_hull_counters(torch.cuda.current_stream().cuda_stream)
            assert c["stage"] == 2, c   # the call really took the radix-sort fallback

"""The data-parallel form of the filter's exchange step, run as two CPU ranks
(gloo): each rank holds one shard of the points, finds its shard's extremes
as packed (key, lowest global index) values, one all-reduce (max) gives the
global extremes, each rank keeps the points of its shard that are not
strictly inside the global octagon, and the gathered survivors' hull equals
the oracle's hull of all points.  This is the exchange a sharded single hull
would need (one GPU per rank); on one GPU the library runs replicas only."""
import os
import socket

import numpy as np
import pytest

import oracle
from oracle import filter_ref as F
from synth import workloads as W

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _packed_extremes(pts, first_index):
    """Per direction W, SW, S, SE, E, NE, N, NW: (key, 2^31 - 1 - global index)
    packed so that the maximum is the winner (minima by complemented key)."""
    x = pts[:, 0].astype(np.int64)
    y = pts[:, 1].astype(np.int64)
    keys = [-x, -(x + y), -y, x - y, x, x + y, y, -(x - y)]
    idx = np.arange(pts.shape[0], dtype=np.int64) + first_index
    out = np.zeros(8, np.int64)
    for d, k in enumerate(keys):
        packed = ((k + (1 << 26)) << 31) | ((1 << 31) - 1 - idx)   # key biased non-negative (< 2^27)
        out[d] = packed.max() if packed.size else -1
    return out


def _rank(rank, world, port, pts, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = pts.shape[0]
        bounds = np.linspace(0, n, world + 1).astype(np.int64)
        lo, hi = int(bounds[rank]), int(bounds[rank + 1])
        shard = pts[lo:hi]
        t = torch.from_numpy(_packed_extremes(shard, lo))
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ext = ((1 << 31) - 1) - (t.numpy() & ((1 << 31) - 1))   # global indices of the 8 extremes
        # filter the shard against the global octagon: the 8 extreme points are
        # appended so the oracle's octagon can name them by index
        aug = np.concatenate([shard, pts[ext]])
        inside = F.inside_octagon(aug, np.arange(shard.shape[0], shard.shape[0] + 8))[:shard.shape[0]]
        keep = np.nonzero(~inside)[0] + lo
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([keep.size], dtype=torch.int64))
        m = max(int(s.item()) for s in sizes)
        buf = torch.full((m,), -1, dtype=torch.int64)
        buf[:keep.size] = torch.from_numpy(keep)
        parts = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(parts, buf)
        if rank == 0:
            got = np.concatenate([p.numpy()[:int(s.item())] for p, s in zip(parts, sizes)])
            q.put((ext.tolist(), got))
    finally:
        dist.destroy_process_group()


def _run(pts, world=2):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, pts, q)) for r in range(world)]
    for p in procs:
        p.start()
    ext, survivors = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return np.array(ext), survivors


@pytest.mark.parametrize("kind,n,seed", [("normal", 20_000, 1), ("ring", 5_000, 2), ("uniform", 7_777, 3)])
def test_sharded_exchange_gives_the_oracle_hull(kind, n, seed):
    pts = W.make(kind, n, seed)
    ext, survivors = _run(pts)
    np.testing.assert_array_equal(ext, F.extremes(pts))           # same extremes as one rank
    assert np.all(np.diff(survivors) > 0)                        # gathered in global order
    sub = pts[survivors]
    hull_sub = survivors[oracle.hull(sub)]
    np.testing.assert_array_equal(hull_sub, oracle.hull(pts))
    if kind == "normal":
        assert survivors.size < n // 10                          # the exchange moves few points

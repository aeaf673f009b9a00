"""Seeded synthetic point sets shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This module only draws random numbers and lays them out; it contains none of
the hull or filter arithmetic.  Every generator returns an ``(n, 2)`` float32
array in AoS order (x0, y0, x1, y1, ...) whose values are integers in
``[0, 2**24)`` -- the input domain of the library (the paper only says
"floating point values", Alg. 2; integer-valued float32 keeps every
predicate exact).

Workload shapes follow the paper's evaluation (Sec. 4): an average case drawn
from a normal distribution (Tables III-IV), the worst case with points on a
circumference (Table V), and sizes from 1e4 to 1e8.  The paper does not give
its distribution parameters, so the parameters below are this project's
stand-ins:

* uniform:  integers uniform in the square [0, 2**24)^2
* normal:   isotropic normal centred at (2**23, 2**23), sigma 2**21, rounded
            half-to-even and clamped to [0, 2**24 - 1]
* ring:     angle uniform in [0, 2 pi), radius 2**23 - u with u uniform in
            [0, 64), centred at (2**23, 2**23), rounded and clamped
* distorted: the circumference with "2% distortion": radius 2**23 (1 - 0.02 u),
            u uniform in [0, 1), otherwise as ring
* batched:  4096 instances, sizes log-uniform in [100, 1e6], each drawn from
            one of the three generators above
* serving:  Poisson arrivals at 20,000 req/s, sizes log-uniform in
            [1e3, 1e7], mix 50% normal / 40% uniform / 10% ring
"""
from __future__ import annotations

import math

import numpy as np

COORD_LIMIT = 1 << 24          # exclusive upper bound of a coordinate
CENTER = float(1 << 23)
SIGMA = float(1 << 21)
RING_RADIUS = float(1 << 23)
RING_WIDTH = 64.0

GENERATORS = ("uniform", "normal", "ring")


def _clip_round(a: np.ndarray) -> np.ndarray:
    np.rint(a, out=a)
    np.clip(a, 0.0, float(COORD_LIMIT - 1), out=a)
    return a


def uniform(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, COORD_LIMIT, size=(n, 2), dtype=np.int64).astype(np.float32)


def normal(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.empty((n, 2), dtype=np.float32)
    # Chunked so that a 1e8-point draw does not need 1.6 GB of float64 at once;
    # the stream of draws is identical to one rng.normal(..., (n, 2)) call.
    step = 1 << 22
    for s in range(0, n, step):
        e = min(n, s + step)
        a = rng.normal(CENTER, SIGMA, size=(e - s, 2))
        out[s:e] = _clip_round(a)
    return out


def ring(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=n)
    u = rng.uniform(0.0, RING_WIDTH, size=n)
    out = np.empty((n, 2), dtype=np.float32)
    step = 1 << 22
    for s in range(0, n, step):
        e = min(n, s + step)
        r = RING_RADIUS - u[s:e]
        out[s:e, 0] = _clip_round(CENTER + r * np.cos(theta[s:e]))
        out[s:e, 1] = _clip_round(CENTER + r * np.sin(theta[s:e]))
    return out


DISTORTION = 0.02


def distorted(n: int, seed: int) -> np.ndarray:
    """The paper's worst case with "2% distortion" (Sec. 4; parameters not
    given): points near the circle of radius 2**23 about (2**23, 2**23), the
    radius jittered inward by up to 2% of it (angle uniform in [0, 2 pi),
    radius R (1 - 0.02 U[0, 1))), rounded and clamped."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=n)
    f = rng.uniform(0.0, 1.0, size=n)
    out = np.empty((n, 2), dtype=np.float32)
    step = 1 << 22
    for s in range(0, n, step):
        e = min(n, s + step)
        r = RING_RADIUS * (1.0 - DISTORTION * f[s:e])
        out[s:e, 0] = _clip_round(CENTER + r * np.cos(theta[s:e]))
        out[s:e, 1] = _clip_round(CENTER + r * np.sin(theta[s:e]))
    return out


def make(kind: str, n: int, seed: int) -> np.ndarray:
    if kind == "uniform":
        return uniform(n, seed)
    if kind == "normal":
        return normal(n, seed)
    if kind == "ring":
        return ring(n, seed)
    if kind == "distorted":
        return distorted(n, seed)
    raise ValueError(f"unknown generator {kind!r}")


# The five workload configurations (single hulls, batched, served).
SINGLE = {
    "uniform_1e6": ("uniform", 1_000_000, 0),
    "normal_1e8": ("normal", 100_000_000, 1),
    "ring_1e8": ("ring", 100_000_000, 2),
    "distorted_1e8": ("distorted", 100_000_000, 5),
}


def single(name: str, n: int | None = None) -> np.ndarray:
    kind, n0, seed = SINGLE[name]
    return make(kind, n0 if n is None else n, seed)


def batched_plan(k: int = 4096, seed: int = 3, lo: int = 100, hi: int = 1_000_000):
    """Sizes and generator kinds of the batched workload, plus per-instance seeds."""
    rng = np.random.default_rng(seed)
    sizes = [int(np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(k)]
    kinds = [GENERATORS[int(rng.integers(0, 3))] for _ in range(k)]
    seeds = np.random.SeedSequence(seed).spawn(k)
    inst_seeds = [int(s.generate_state(1)[0]) for s in seeds]
    return sizes, kinds, inst_seeds


def batched(k: int = 4096, seed: int = 3, lo: int = 100, hi: int = 1_000_000):
    """Packed batched workload: (points (N, 2) float32, offsets int64[k+1])."""
    sizes, kinds, inst_seeds = batched_plan(k, seed, lo, hi)
    offsets = np.zeros(k + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    pts = np.empty((int(offsets[-1]), 2), dtype=np.float32)
    for i in range(k):
        pts[offsets[i]:offsets[i + 1]] = make(kinds[i], sizes[i], inst_seeds[i])
    return pts, offsets


def serving_plan(rate: float = 20_000.0, seconds: float = 10.0, seed: int = 4,
                 lo: int = 1_000, hi: int = 10_000_000):
    """Poisson request stream: arrival times (s), sizes, generator kinds."""
    rng = np.random.default_rng(seed)
    count = int(rng.poisson(rate * seconds))
    arrivals = np.sort(rng.uniform(0.0, seconds, size=count))
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    mix = rng.uniform(0.0, 1.0, size=count)
    kinds = np.where(mix < 0.5, 0, np.where(mix < 0.9, 1, 2))  # normal, uniform, ring
    names = np.array(["normal", "uniform", "ring"])[kinds]
    return arrivals, sizes, names


# Small structured inputs (edge cases of the method, used by both sides' tests).

def degenerate_suite(seed: int = 7):
    """Named small inputs covering the degenerate cases of the hull."""
    rng = np.random.default_rng(seed)
    M = COORD_LIMIT - 1
    cases = {}
    cases["empty"] = np.zeros((0, 2), np.float32)
    cases["one"] = np.array([[5, 7]], np.float32)
    cases["two"] = np.array([[9, 1], [3, 4]], np.float32)
    cases["two_same"] = np.array([[3, 3], [3, 3]], np.float32)
    cases["identical"] = np.full((1000, 2), 12345, np.float32)
    t = rng.integers(0, 1 << 20, 777)
    cases["horizontal"] = np.stack([t, np.full_like(t, 99)], 1).astype(np.float32)
    cases["vertical"] = np.stack([np.full_like(t, 4242), t], 1).astype(np.float32)
    cases["diagonal"] = np.stack([t + 5, t + 17], 1).astype(np.float32)
    cases["antidiagonal"] = np.stack([t, (1 << 21) - t], 1).astype(np.float32)
    cases["slope_1_3"] = np.stack([3 * t[:300], t[:300] + 11], 1).astype(np.float32)
    corners = np.array([[0, 0], [M, 0], [M, M], [0, M]], np.float32)
    fill = rng.integers(0, M + 1, (2000, 2)).astype(np.float32)
    cases["square_extremes"] = np.concatenate([fill, corners, corners, fill[:10]])
    dup = rng.integers(0, 50, (3000, 2)).astype(np.float32)
    cases["dense_duplicates"] = dup
    cases["border_lines"] = np.concatenate([
        np.stack([np.zeros(500), rng.integers(0, M + 1, 500)], 1),
        np.stack([np.full(500, M), rng.integers(0, M + 1, 500)], 1),
        np.stack([rng.integers(0, M + 1, 500), np.zeros(500)], 1),
        np.stack([rng.integers(0, M + 1, 500), np.full(500, M)], 1),
        rng.integers(0, M + 1, (500, 2)),
    ]).astype(np.float32)
    rng.shuffle(cases["border_lines"])
    tri = []
    for a in range(0, 301, 3):
        tri.append([a, 0])
        tri.append([0, a])
        tri.append([a, 300 - a])
    cases["triangle_edges"] = (np.array(tri, np.float32) + 1000)
    cases["tiny_random"] = rng.integers(0, 8, (37, 2)).astype(np.float32)
    cases["collinear_plus_one"] = np.concatenate([
        np.stack([3 * t[:200], t[:200]], 1), [[1500, 490]]]).astype(np.float32)
    return cases

"""Planted mistakes in a COPY of the oracle (compiled on the CPU) must be
caught by the pins: brute force, lattice polygons and degenerate closed
forms.  Shows the pins would notice a dropped term, a wrong sign, an
off-by-one or a lost tie rule in the oracle."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import brute
from synth import workloads as W
from tests import golden_io

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "andrew.c")

MUTANTS = {
    "keeps_collinear": ("cross3(&h[k - 2], &h[k - 1], &p[i]) <= 0", "cross3(&h[k - 2], &h[k - 1], &p[i]) < 0"),
    "transposed_operand": ("(b->y - o->y) - (a->y - o->y)", "(b->y - a->y) - (a->y - o->y)"),
    "keeps_last_duplicate": ("p[m - 1].y == p[i].y) continue;", "p[m - 1].y == p[i].y) { p[m - 1] = p[i]; continue; }"),
    "upper_chain_off_by_one": ("const int64_t lower_len = k + 1;", "const int64_t lower_len = k;"),
    "repeats_first_point": ("--k; /* the last point repeats the first */", "/* mutated */"),
    "sign_flipped_pop": ("cross3(&h[k - 2], &h[k - 1], &p[i]) <= 0", "cross3(&h[k - 2], &h[k - 1], &p[i]) >= 0"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    lib.oracle_hull.restype = ctypes.c_int64
    lib.oracle_hull.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return lib


def _run(lib, pts):
    a = np.ascontiguousarray(pts, np.float32)
    out = np.empty(max(a.shape[0], 1) + 1, np.int32)
    h = lib.oracle_hull(a.ctypes.data, a.shape[0], out.ctypes.data)
    return out[:max(h, 0)].copy()


def _pins_pass(lib):
    rng = np.random.default_rng(1)
    for span in (4, 9, 300):
        for _ in range(10):
            pts = rng.integers(0, span, (int(rng.integers(3, 80)), 2)).astype(np.float32)
            if not np.array_equal(_run(lib, pts), brute.hull(pts)):
                return False
    for name in golden_io.FIXTURES:
        pts, exp = golden_io.load(name)
        if not np.array_equal(_run(lib, pts), exp):
            return False
    for pts in W.degenerate_suite().values():
        if pts.shape[0] and len({tuple(p) for p in pts.tolist()}) <= 250:
            if not np.array_equal(_run(lib, pts), brute.hull(pts)):
                return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_unmutated_copy_passes(tmp_path):
    lib = _build(tmp_path, "identity", "int64_t oracle_hull", "int64_t oracle_hull")
    assert _pins_pass(lib)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    assert not _pins_pass(lib), f"pins did not catch mutant {name}"

"""CPU oracle for the convex-hull hot path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports, links or calls anything here, and nothing here
imports the product package.

Contents
--------
* ``hull(pts)``       -- Andrew's monotone chain in plain C with int64
                         orientation (``andrew.c``); the definition the GPU
                         hull must reach bit-exactly.
* ``filter_ref``      -- the paper's filtering stage (Alg. 2) written out in
                         numpy int64: the 8 extremes, the octagon test and the
                         four-queue labelling.
* ``filter16_ref``    -- the same filter with a 16-direction polygon (the 8
                         octagon directions and the 8 integer directions
                         between them), in numpy int64.
* ``brute``           -- an O(n^3) edge-test hull for tiny inputs, used to
                         pin ``hull`` itself.
* ``heaphull_cpu(pts, threads)`` -- the paper's heaphull on the host's cores
                         (``heaphull_cpu.c``: parallel extremes and octagon
                         filter, parallel sort, Andrew's chains): the CPU
                         comparator the benchmark times; checked against
                         ``hull`` by the tests, not a definition itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "andrew.c"), os.path.join(_HERE, "heaphull_cpu.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORACLE_ERANGE = -2


def build(force: bool = False) -> str:
    """Compile ``andrew.c`` and ``heaphull_cpu.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src) for src in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, *_SRCS, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_hull.restype = ctypes.c_int64
            lib.oracle_hull.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            lib.oracle_check.restype = ctypes.c_int
            lib.oracle_check.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            lib.cpu_heaphull.restype = ctypes.c_int64
            lib.cpu_heaphull.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
            _lib = lib
    return _lib


def _as_points(pts) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pts, dtype=np.float32))
    if a.ndim == 1:
        a = a.reshape(-1, 2)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("points must have shape (n, 2)")
    return a


def hull(pts) -> np.ndarray:
    """CCW index list of the strictly convex hull vertices, from the lex-min vertex.

    Raises ``ValueError`` when a coordinate is not an integer in [0, 2**24).
    """
    a = _as_points(pts)
    n = a.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    h = _load().oracle_hull(a.ctypes.data, n, out.ctypes.data)
    if h == ORACLE_ERANGE:
        raise ValueError("coordinate outside the integer domain [0, 2**24)")
    if h < 0:
        raise MemoryError("oracle allocation failed")
    return out[:h].copy()


def heaphull_cpu(pts, threads: int = 1) -> np.ndarray:
    """The CPU heaphull comparator on ``threads`` POSIX threads; same output
    convention and errors as ``hull``."""
    a = _as_points(pts)
    n = a.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    h = _load().cpu_heaphull(a.ctypes.data, n, out.ctypes.data, int(threads))
    if h == ORACLE_ERANGE:
        raise ValueError("coordinate outside the integer domain [0, 2**24)")
    if h < 0:
        raise MemoryError("heaphull_cpu allocation failed")
    return out[:h].copy()


def check(pts) -> bool:
    """True when every coordinate is an integer-valued float in [0, 2**24)."""
    a = _as_points(pts)
    return _load().oracle_check(a.ctypes.data, a.shape[0]) == 0


from . import brute, filter16_ref, filter_ref  # noqa: E402,F401

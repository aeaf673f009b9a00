"""ctypes binding of libconvhull.so: the C ABI of include/ch.h, same names,
argument marshalling only.  Pointers are passed as integers (device or host
addresses as the header states); every computation happens in the library.

The library is loaded from this package's _build/ directory.  There is no
fallback: if the shared library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libconvhull.so")

CH_OK = 0
CH_PENDING = 1
CH_EINVAL = -1
CH_ERANGE = -2
CH_ENOMEM = -3
CH_ECUDA = -4
CH_ETIMEOUT = -5
CH_EBUSY = -6
CH_MAX_POINTS = 0x7FFFFFF0   # largest point count of one hull (indices are int32)

_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_INT = ctypes.c_int
_SZ = ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/ch.h
SIGNATURES = {
    "ch_hull": (_INT, [_P, _I64, _P, _P, _P]),
    "ch_hull_batched": (_INT, [_P, _P, _I32, _P, _P, _P, _P]),
    "ch_filter": (_INT, [_P, _I64, _P, _P, _P, _P]),
    "ch_filter16": (_INT, [_P, _I64, _P, _P, _P, _P]),
    "ch_filter_manhattan": (_INT, [_P, _I64, _P, _P, _P, _P]),
    "ch_hull_host": (_INT, [_P, _I64, _P, _P, _P]),
    "ch_hull_noalloc": (_INT, [_P, _I64, _P, _P, _P]),
    "ch_batched_config": (_INT, [_I64, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "ch_reserve": (_INT, [_I64, _I32, _P]),
    "ch_workspace_bytes": (_SZ, [_I64]),
    "ch_hull_counters": (_INT, [_P, ctypes.POINTER(_I64), _INT]),
    "ch_batched_counters": (_INT, [_P, _I32, ctypes.POINTER(_I64)]),
    "ch_release": (_INT, []),
    "ch_selftest_timeout": (_INT, [_INT, _P]),
    "ch_strerror": (ctypes.c_char_p, [_INT]),
    "ch_profile_enable": (_INT, [_INT]),
    "ch_profile_reset": (_INT, []),
    "ch_profile_read": (_INT, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_I64),
                               ctypes.POINTER(ctypes.c_double), _INT]),
    "ch_server_create": (_INT, [_SZ, _INT, ctypes.POINTER(_P)]),
    "ch_submit": (_INT, [_P, _P, _I64, ctypes.POINTER(ctypes.c_uint64)]),
    "ch_poll": (_INT, [_P, ctypes.c_uint64, _P, _I64, ctypes.POINTER(_I64)]),
    "ch_server_stats": (_INT, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "ch_server_trace": (_INT, [_P, _P, _I64]),
    "ch_server_destroy": (_INT, [_P]),
}


class CHError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else strerror(status))


def load(path: str | None = None):
    """Load libconvhull.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libconvhull.so not built at {p}; run paper_2209_12310_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def strerror(status: int) -> str:
    try:
        return load().ch_strerror(int(status)).decode()
    except Exception:  # library missing: keep the message usable
        return f"status {status}"


def _check(status: int, what: str) -> int:
    if status < 0:
        raise CHError(status, what)
    return status


def ch_hull(pts, n, out_idx, out_n, stream=0):
    return _check(load().ch_hull(pts, n, out_idx, out_n, stream), "ch_hull")


def ch_hull_batched(pts, offsets, k, out_idx, out_n, host_offsets=None, stream=0):
    return _check(load().ch_hull_batched(pts, offsets, k, out_idx, out_n, host_offsets, stream),
                  "ch_hull_batched")


def ch_batched_config(total_points, k):
    """(threads, points per thread) of ch_hull_batched's tile kernels for this
    size class on the current device; (0, 0) before it has been tuned."""
    t, p = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().ch_batched_config(int(total_points), int(k), ctypes.byref(t), ctypes.byref(p)),
           "ch_batched_config")
    return t.value, p.value


def ch_filter(pts, n, out_ext8, out_labels=None, out_counts4=None, stream=0):
    return _check(load().ch_filter(pts, n, out_ext8, out_labels, out_counts4, stream), "ch_filter")


def ch_filter_manhattan(pts, n, out_ext8, out_labels=None, out_counts4=None, stream=0):
    return _check(load().ch_filter_manhattan(pts, n, out_ext8, out_labels, out_counts4, stream),
                  "ch_filter_manhattan")


def ch_filter16(pts, n, out_ext16, out_labels=None, out_counts4=None, stream=0):
    return _check(load().ch_filter16(pts, n, out_ext16, out_labels, out_counts4, stream), "ch_filter16")


def ch_hull_host(pts, n, out_idx, out_n, stream=0):
    return _check(load().ch_hull_host(pts, n, out_idx, out_n, stream), "ch_hull_host")


def ch_reserve(n, k=1, stream=0):
    return _check(load().ch_reserve(n, k, stream), "ch_reserve")


def ch_batched_counters(k, stream=0):
    """Per-set counters of the most recent ch_hull_batched of k sets on
    `stream`: a list of dicts (records, star vertices, status, hull stage)."""
    out = (_I64 * (4 * max(k, 1)))()
    _check(load().ch_batched_counters(stream, k, out), "ch_batched_counters")
    return [{"records": int(out[4 * i]), "star_vertices": int(out[4 * i + 1]), "status": int(out[4 * i + 2]),
             "stage": int(out[4 * i + 3])} for i in range(k)]


def ch_hull_counters(stream=0):
    """Counters of the most recent ch_hull on `stream`: raw survivors, records,
    mode (two streaming passes), hull stage (0 one block, 1 buckets, 2 sort),
    status, vertices of the star polygon (0: none built)."""
    out = (_I64 * 8)()
    k = _check(load().ch_hull_counters(stream, out, 8), "ch_hull_counters")
    names = ("raw", "records", "two_pass", "stage", "status", "star_vertices")
    return {names[i]: int(out[i]) for i in range(min(k, 8, len(names)))}


def ch_workspace_bytes(n):
    return int(load().ch_workspace_bytes(n))


def ch_release():
    return _check(load().ch_release(), "ch_release")


def ch_strerror(status):
    return strerror(status)


def ch_profile_enable(on=True):
    return _check(load().ch_profile_enable(1 if on else 0), "ch_profile_enable")


def ch_profile_reset():
    return _check(load().ch_profile_reset(), "ch_profile_reset")


def ch_profile_read():
    """{kernel name: (launches, total_ms)} of the device-timed statistics."""
    lib = load()
    cap = 64
    names = (ctypes.c_char_p * cap)()
    launches = (_I64 * cap)()
    ms = (ctypes.c_double * cap)()
    k = lib.ch_profile_read(names, launches, ms, cap)
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(k, cap))}


def ch_server_create(budget_bytes, device=0):
    h = _P()
    _check(load().ch_server_create(budget_bytes, device, ctypes.byref(h)), "ch_server_create")
    return h.value


def ch_submit(srv, pts_host, n):
    t = ctypes.c_uint64()
    st = load().ch_submit(srv, pts_host, n, ctypes.byref(t))
    return st, t.value


def ch_poll(srv, ticket, out_idx_host, cap):
    n = _I64()
    st = load().ch_poll(srv, ticket, out_idx_host, cap, ctypes.byref(n))
    return st, n.value


def ch_server_stats(srv):
    p50, p99, pps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    done = _I64()
    _check(load().ch_server_stats(srv, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(pps),
                                  ctypes.byref(done)), "ch_server_stats")
    return {"p50_ms": p50.value, "p99_ms": p99.value, "points_per_s": pps.value,
            "completed": done.value}


def ch_server_trace(srv):
    """The server's retired batches: a list of 8-tuples (formation ms, requests,
    points, copy-in ms, hull ms, index-copy ms, host ms, sets redone)."""
    lib = load()
    n = _check(lib.ch_server_trace(srv, None, 0), "ch_server_trace")
    buf = (ctypes.c_double * (8 * max(n, 1)))()
    n = min(n, _check(lib.ch_server_trace(srv, ctypes.addressof(buf), n), "ch_server_trace"))
    return [tuple(buf[8 * i:8 * i + 8]) for i in range(n)]


def ch_server_destroy(srv):
    return _check(load().ch_server_destroy(srv), "ch_server_destroy")

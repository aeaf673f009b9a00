"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/ch.h declares; host-side argument checks answer without
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ch.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ch_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def native():
    from paper_2209_12310_gb300 import build as pkg_build
    path = pkg_build()
    assert os.path.exists(path)
    import paper_2209_12310_gb300 as ch
    return ch.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ch_hull", "ch_hull_batched", "ch_filter", "ch_submit", "ch_poll",
                 "ch_server_create", "ch_server_destroy", "ch_workspace_bytes", "ch_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(native):
    lib = ctypes.CDLL(native._name)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_names_match_header():
    from paper_2209_12310_gb300 import _native
    assert sorted(_native.SIGNATURES) == _declared()


def test_host_side_checks_without_gpu(native):
    import paper_2209_12310_gb300 as ch
    assert native.ch_hull(None, -1, None, None, None) == ch.CH_EINVAL
    assert native.ch_hull(8, 10, 0, 0, None) == ch.CH_EINVAL          # null outputs
    assert native.ch_hull(12, 10, 64, 64, None) == ch.CH_EINVAL        # pts not 8-byte aligned
    assert native.ch_filter(None, -5, None, None, None, None) == ch.CH_EINVAL
    assert native.ch_filter16(None, -5, None, None, None, None) == ch.CH_EINVAL
    assert native.ch_filter16(8, 10, None, None, None, None) == ch.CH_EINVAL      # null out_ext16
    assert native.ch_filter16(12, 10, 64, None, None, None) == ch.CH_EINVAL       # pts not 8-byte aligned
    assert native.ch_filter16(None, 10, 64, None, None, None) == ch.CH_EINVAL     # null pts, n > 0
    assert native.ch_hull_batched(None, None, -1, None, None, None, None) == ch.CH_EINVAL
    assert native.ch_hull_batched(None, None, 0, None, None, None, None) == ch.CH_OK
    assert native.ch_hull_batched(None, None, (1 << 20) + 1, None, None, None, None) == ch.CH_EINVAL  # k > 2^20
    assert native.ch_batched_counters(None, 4, None) == ch.CH_EINVAL                 # null out
    assert native.ch_batched_counters(None, 0, (ctypes.c_int64 * 4)()) == ch.CH_EINVAL  # k < 1
    assert native.ch_filter_manhattan(None, -5, None, None, None, None) == ch.CH_EINVAL
    assert native.ch_filter_manhattan(8, 10, None, None, None, None) == ch.CH_EINVAL  # null out_ext8
    assert native.ch_poll(None, 1, None, 0, None) == ch.CH_EINVAL
    assert native.ch_submit(None, None, 1, None) == ch.CH_EINVAL
    assert ch.ch_strerror(ch.CH_ERANGE).startswith("coordinate")


def test_point_count_limit_without_gpu(native):
    """One point past CH_MAX_POINTS is refused by every entry point that
    takes a point count, before any device work (the pointers are never
    dereferenced)."""
    import paper_2209_12310_gb300 as ch
    text = open(HEADER).read()
    assert int(re.search(r"#define CH_MAX_POINTS \(\(int64_t\)(0x[0-9A-Fa-f]+)\)", text).group(1), 16) == ch.CH_MAX_POINTS
    over = ch.CH_MAX_POINTS + 1
    assert native.ch_hull(8, over, 64, 64, None) == ch.CH_EINVAL
    assert native.ch_hull_host(8, over, 64, 64, None) == ch.CH_EINVAL
    assert native.ch_filter(8, over, 64, None, None, None) == ch.CH_EINVAL
    assert native.ch_filter16(8, over, 64, None, None, None) == ch.CH_EINVAL
    assert native.ch_filter_manhattan(8, over, 64, None, None, None) == ch.CH_EINVAL


def test_workspace_size_is_linear(native):
    import paper_2209_12310_gb300 as ch
    a = ch.ch_workspace_bytes(1_000_000)
    b = ch.ch_workspace_bytes(2_000_000)
    assert 20 * 1_000_000 < a < 80 * 1_000_000
    assert 1.8 < b / a < 2.2


def test_no_fallback_without_the_library():
    """Without libconvhull.so the binding raises instead of computing
    anything, and the tensor helpers refuse host tensors (no CPU path)."""
    import subprocess
    import sys
    code = (
        "import paper_2209_12310_gb300 as ch, paper_2209_12310_gb300._native as n\n"
        "n.LIB_PATH = '/nonexistent/libconvhull.so'\n"
        "try:\n"
        "    ch.load()\n"
        "except RuntimeError as e:\n"
        "    assert 'not built' in str(e)\n"
        "else:\n"
        "    raise SystemExit('loaded a library that does not exist')\n"
        "import torch\n"
        "try:\n"
        "    ch.hull(torch.zeros((3, 2)))\n"
        "except TypeError:\n"
        "    print('refused')\n"
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "refused"

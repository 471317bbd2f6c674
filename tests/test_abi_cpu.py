"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/squaresort.h, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "squaresort.h")


@pytest.fixture(scope="module")
def sq():
    from paper_2407_14801_gb300 import build

    build.build()
    import paper_2407_14801_gb300 as sq

    return sq


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(sq_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sq_sort", "sq_skew_transpose", "sq_sort_batch", "sq_serve_submit", "sq_serve_poll",
                     "sq_serve_create", "sq_serve_destroy", "sq_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(sq):
    lib = ctypes.CDLL(sq.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_limits(sq):
    assert sq.max_leaf("u32") == 65536 and sq.max_leaf("u64") == 65536 and sq.max_leaf("f32") == 65536
    assert sq.max_n("u32") == 16385 ** 2 >= 1 << 28
    assert sq.max_n("u64") == 8193 ** 2 >= 1 << 26


def test_rejects_bad_arguments_without_a_device(sq):
    L = sq.lib()
    assert L.sq_sort(None, None, 10, 7, 0, None) == 1  # bad dtype
    assert L.sq_sort(None, None, 10, 0, 0, None) == 1  # NULL keys
    assert L.sq_sort(None, None, sq.max_n("u32") + 1, 0, 0, None) == 1
    assert b"exceeds" in L.sq_last_error()
    opts = sq.SortOpts(1, 0, None, None)  # cutoff 1 is below the minimum
    assert L.sq_sort_ex(ctypes.c_void_p(8), None, 10, 0, 0, None, ctypes.byref(opts)) == 1
    assert L.sq_skew_transpose(None, 4, 4, None) == 1
    buf = sq.SkewBuf(0, 20, None, None, None, None, None, None, 4, None)
    assert L.sq_skew_transpose(ctypes.byref(buf), 4, 4, None) == 1  # n > rows*cols
    assert L.sq_sort_batch(None, 3, None) == 1
    assert L.sq_set_cutoff(0, 1) == 1 and L.sq_set_cutoff(0, 70000) == 1
    assert L.sq_set_cutoff(0, 300) == 0 and L.sq_get_cutoff(0) == 300
    assert L.sq_set_cutoff(0, 0) == 0 and L.sq_get_cutoff(0) == 65536
    assert L.sq_sort(None, None, 0, 0, 0, None) == 0  # empty sort is a no-op


def test_launch_mode_without_a_device(sq):
    L = sq.lib()
    assert L.sq_get_launch_mode() == 2  # auto
    assert L.sq_set_launch_mode(5) == 1 and b"launch mode" in L.sq_last_error()
    assert L.sq_set_launch_mode(0) == 0 and L.sq_get_launch_mode() == 0
    assert L.sq_set_launch_mode(2) == 0

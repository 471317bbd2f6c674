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
    assert sq.max_n("u32") == 2**32 - 1  # (65535 + 1)^2 capped to 32-bit sizes: cluster-sorted pivot samples
    assert sq.max_n("f32") == 8193 ** 2
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


def test_appendix_variant_refusals_without_a_device(sq):
    """The variant takes integer keys, a cutoff of at least 8 and n below
    (16384 + 1)^2 for uint32 keys; the checks come before any device work."""
    L = sq.lib()

    def ex(dtype, n, cutoff, variant):
        opts = sq.SortOpts(cutoff, 0, None, None, variant)
        return L.sq_sort_ex(ctypes.c_void_p(8), None, n, dtype, 0, None, ctypes.byref(opts))

    assert ex(2, 10, 16, 1) == 1 and b"integer" in L.sq_last_error()  # SQ_F32
    assert ex(0, 10, 7, 1) == 1 and b"cutoff" in L.sq_last_error()
    assert ex(0, 10, 16, 2) == 1 and b"variant" in L.sq_last_error()
    assert ex(0, 16385**2, 16, 1) == 1 and b"appendix" in L.sq_last_error()
    assert ex(1, sq.max_n("u64"), 16, 1) == 1
    assert sq.VARIANTS == {"algorithm1": 0, "appendix": 1}


def test_skew_transpose_keeps_the_one_cta_pivot_limit(sq):
    """Sorts of uint32 keys reach 2^32 - 1 (cluster-sorted pivot samples),
    but the stand-alone SkewTranspose takes k up to 16385 buckets for uint32
    and 8193 otherwise; the check comes before any device work."""
    L = sq.lib()
    dummy = ctypes.c_void_p(8)
    for dtype, kmax in ((0, 16385), (1, 8193), (2, 8193)):
        buf = sq.SkewBuf(dtype, 4, dummy, dummy, dummy, dummy, dummy, dummy, kmax + 1, dummy)
        assert L.sq_skew_transpose(ctypes.byref(buf), 2, 2, None) == 1
        assert b"k = " in L.sq_last_error()
        assert L.sq_skew_transpose_noalloc(ctypes.byref(buf), 2, 2, None) == 1


def test_launch_mode_without_a_device(sq):
    L = sq.lib()
    assert L.sq_get_launch_mode() == 2  # auto
    assert L.sq_set_launch_mode(5) == 1 and b"launch mode" in L.sq_last_error()
    assert L.sq_set_launch_mode(0) == 0 and L.sq_get_launch_mode() == 0
    assert L.sq_set_launch_mode(2) == 0


def test_binding_structs_match_the_header(tmp_path):
    """Every structure the binding passes through the C ABI (ctypes, and the
    numpy records of batch descriptors) lays its fields out exactly as the C
    compiler does for the header's struct."""
    import shutil
    import subprocess

    import paper_2407_14801_gb300 as sq

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [(sq.TraceRec, "sq_trace_rec"), (sq.SortOpts, "sq_sort_opts"), (sq.SkewBuf, "sq_skew_buf"),
             (sq.SortDesc, "sq_sort_desc"), (sq.ServeOpts, "sq_serve_opts"), (sq.Stats, "sq_stats")]
    lines = []
    for cls, cname in pairs:
        fields = [f for f, _ in cls._fields_]
        fmt = " ".join(["%zu"] * (1 + len(fields)))
        args = ", ".join([f"sizeof({cname})"] + [f"offsetof({cname}, {f})" for f in fields])
        lines.append(f'  printf("{fmt}\\n", {args});')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "squaresort.h"\nint main(void) {\n' +
                   "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    for (cls, cname), line in zip(pairs, out):
        got = list(map(int, line.split()))
        want = [ctypes.sizeof(cls)] + [getattr(cls, f).offset for f, _ in cls._fields_]
        assert got == want, (cname, got, want)
    rec = sq._desc_dtype()  # the batch descriptors' numpy record
    desc = list(map(int, out[3].split()))
    assert rec.itemsize == desc[0]
    assert [rec.fields[f][1] for f, _ in sq.SortDesc._fields_] == desc[1:]

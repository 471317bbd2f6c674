"""GB300 SquareSort: Python binding of ``libsquaresort.so``.

Argument marshalling only: every step of the sort runs in the library's CUDA
kernels.  The functions mirror the C ABI in ``include/squaresort.h``
(``sq_sort``, ``sq_skew_transpose``, ``sq_sort_batch``, ``sq_serve_*``).
PyTorch supplies device memory and streams.  If the compiled library is
missing this module raises on first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LIB_PATH = _build.LIB
TUNING_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")

SQ_U32, SQ_U64, SQ_F32 = 0, 1, 2
DTYPES = {"u32": SQ_U32, "u64": SQ_U64, "f32": SQ_F32}
STATUS = {0: "SQ_OK", 1: "SQ_ERR_INVALID", 2: "SQ_ERR_NOMEM", 3: "SQ_ERR_BUDGET", 4: "SQ_ERR_TIMEOUT",
          5: "SQ_ERR_CUDA", 6: "SQ_PENDING", 7: "SQ_ERR_ATTEMPTS", 8: "SQ_ERR_INTERNAL"}
SQ_OK, SQ_PENDING = 0, 6
FAMILIES = ["leaf", "plan", "pivots", "count", "scan", "bstart", "skew", "expand", "aux"]


class SquareSortError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class TraceRec(ctypes.Structure):
    _fields_ = [("off", ctypes.c_uint64), ("n", ctypes.c_uint64), ("m", ctypes.c_uint64),
                ("hash", ctypes.c_uint64), ("depth", ctypes.c_uint32), ("kind", ctypes.c_uint32),
                ("attempts", ctypes.c_uint32), ("index", ctypes.c_uint32)]


class SortOpts(ctypes.Structure):
    _fields_ = [("cutoff", ctypes.c_uint32), ("trace_cap", ctypes.c_uint32),
                ("trace", ctypes.POINTER(TraceRec)), ("trace_count", ctypes.POINTER(ctypes.c_uint32)),
                ("variant", ctypes.c_uint32)]


# sq_variant: Algorithm 1, or the variant the paper prints in its appendix
VARIANTS = {"algorithm1": 0, "appendix": 1}


class SkewBuf(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("n", ctypes.c_uint64), ("keys_in", ctypes.c_void_p),
                ("vals_in", ctypes.c_void_p), ("keys_out", ctypes.c_void_p), ("vals_out", ctypes.c_void_p),
                ("pivot_keys", ctypes.c_void_p), ("pivot_vals", ctypes.c_void_p), ("k", ctypes.c_uint64),
                ("bucket_start_out", ctypes.c_void_p)]


class SortDesc(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("dtype", ctypes.c_int), ("seed", ctypes.c_uint64)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("cutoff", ctypes.c_uint32), ("device", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 9), ("ms", ctypes.c_double * 9), ("bytes", ctypes.c_double * 9),
                ("rounds", ctypes.c_uint64), ("nodes", ctypes.c_uint64), ("sorts", ctypes.c_uint64)]


_lib = None


def _bind(lib):
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "sq_sort": (i32, [vp, vp, u64, i32, u64, vp]),
        "sq_sort_ex": (i32, [vp, vp, u64, i32, u64, vp, ctypes.POINTER(SortOpts)]),
        "sq_sync": (i32, [vp]),
        "sq_skew_transpose": (i32, [ctypes.POINTER(SkewBuf), u64, u64, vp]),
        "sq_skew_transpose_noalloc": (i32, [ctypes.POINTER(SkewBuf), u64, u64, vp]),
        "sq_sort_batch": (i32, [ctypes.POINTER(SortDesc), u32, vp]),
        "sq_serve_create": (i32, [ctypes.POINTER(vp), u64, ctypes.POINTER(ServeOpts)]),
        "sq_serve_submit": (i32, [vp, ctypes.POINTER(SortDesc), ctypes.POINTER(u64)]),
        "sq_serve_poll": (i32, [vp, u64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]),
        "sq_serve_destroy": (i32, [vp]),
        "sq_last_error": (ctypes.c_char_p, []),
        "sq_max_n": (u64, [i32]),
        "sq_max_leaf": (u32, [i32]),
        "sq_set_cutoff": (i32, [i32, u32]),
        "sq_get_cutoff": (u32, [i32]),
        "sq_set_cutoff_table": (i32, [i32, ctypes.POINTER(u32), u32]),
        "sq_cutoff_for": (u32, [i32, u64]),
        "sq_set_launch_mode": (i32, [i32]),
        "sq_get_launch_mode": (i32, []),
        "sq_stats_get": (None, [ctypes.POINTER(Stats)]),
        "sq_stats_reset": (None, []),
        "sq_set_profiling": (None, [i32]),
        "sq_set_radix_classes": (i32, [i32, u32]),
        "sq_get_radix_classes": (u32, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def lib():
    """The loaded C library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2407_14801_gb300.build.build()")
        _lib = _bind(ctypes.CDLL(LIB_PATH))
        if os.environ.get("SQ_NO_TUNING", "") != "1":
            load_tuning()
    return _lib


def _check(status: int):
    if status != SQ_OK:
        raise SquareSortError(status, lib().sq_last_error().decode(errors="replace"))


def _dtype_of(t, dtype: str | None) -> int:
    if dtype is not None:
        return DTYPES[dtype]
    name = str(t.dtype)
    if name.endswith(("int32", "uint32")):
        return SQ_U32
    if name.endswith(("int64", "uint64")):
        return SQ_U64
    if name.endswith("float32"):
        return SQ_F32
    raise TypeError(f"unsupported key dtype {t.dtype}")


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)  # numpy


def _numel(t):
    return t.numel() if hasattr(t, "numel") else t.size


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream) if torch.cuda.is_available() else None
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


# ----------------------------------------------------------------- sq_sort --

def sq_sort(keys, vals=None, seed: int = 0, dtype: str | None = None, cutoff: int = 0, stream=None,
            trace_cap: int = 0, variant: str = "algorithm1"):
    """Sort (keys, vals) in place (CUDA tensors, or CPU tensors / numpy arrays,
    which the library stages through device memory).  Returns the list of
    per-node trace records when ``trace_cap`` > 0, else None.  ``variant``:
    "algorithm1" or "appendix" (integer keys, cutoff >= 8)."""
    n = _numel(keys)
    if vals is not None and _numel(vals) != n:
        raise ValueError("keys and vals differ in length")
    if variant not in VARIANTS:
        raise ValueError(f"variant {variant!r}: one of {sorted(VARIANTS)}")
    opts = None
    recs = None
    cnt = ctypes.c_uint32(0)
    if cutoff or trace_cap or VARIANTS[variant]:
        recs = (TraceRec * max(trace_cap, 1))()
        opts = SortOpts(cutoff, trace_cap, ctypes.cast(recs, ctypes.POINTER(TraceRec)) if trace_cap else None,
                        ctypes.pointer(cnt), VARIANTS[variant])
    st = lib().sq_sort_ex(_ptr(keys), _ptr(vals), n, _dtype_of(keys, dtype), seed & (2**64 - 1), _stream(stream),
                          ctypes.byref(opts) if opts is not None else None)
    _check(st)
    if trace_cap:
        return [dict(off=r.off, n=r.n, m=r.m, hash=r.hash, depth=r.depth, kind=r.kind, index=r.index,
                     attempts=r.attempts) for r in recs[: min(cnt.value, trace_cap)]]
    return None


sort = sq_sort


def sq_sync(stream=None):
    """Waits for the stream (default: torch's current stream) and raises the
    first error latched by an asynchronous sort on it (graph launch mode)."""
    _check(lib().sq_sync(_stream(stream)))


sync = sq_sync


def sq_skew_transpose(keys_in, vals_in, rows: int, cols: int, pivot_keys, pivot_vals, k: int, keys_out, vals_out,
                      bucket_start_out, dtype: str | None = None, stream=None):
    """Stand-alone SkewTranspose of ``cols`` sorted columns of height <= rows
    into k buckets (CUDA tensors); bucket_start_out: k+1 int64 on the GPU."""
    buf = SkewBuf(_dtype_of(keys_in, dtype), _numel(keys_in), _ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                  _ptr(vals_out), _ptr(pivot_keys), _ptr(pivot_vals), k, _ptr(bucket_start_out))
    _check(lib().sq_skew_transpose(ctypes.byref(buf), rows, cols, _stream(stream)))


skew_transpose = sq_skew_transpose


def sq_skew_transpose_noalloc(keys_in, vals_in, rows: int, cols: int, pivot_keys, pivot_vals, k: int, keys_out,
                              vals_out, bucket_start_out, dtype: str | None = None, stream=None):
    """sq_skew_transpose with its scratch in the library's fixed 64 MiB
    device array instead of freshly allocated memory (for callers that cannot
    allocate device memory there).  Calls whose GPU work overlaps race on that
    array."""
    buf = SkewBuf(_dtype_of(keys_in, dtype), _numel(keys_in), _ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                  _ptr(vals_out), _ptr(pivot_keys), _ptr(pivot_vals), k, _ptr(bucket_start_out))
    _check(lib().sq_skew_transpose_noalloc(ctypes.byref(buf), rows, cols, _stream(stream)))


skew_transpose_noalloc = sq_skew_transpose_noalloc


# sq_sort_desc as a numpy record (keys, vals, n, dtype, 4 bytes of padding,
# seed): a batch's descriptors are built as one array rather than field by
# field through ctypes (4096 instances: a few ms less per call).
_DESC_DTYPE = None
_DTYPE_CODE = {}


def _desc_dtype():
    global _DESC_DTYPE
    if _DESC_DTYPE is None:
        import numpy as np

        _DESC_DTYPE = np.dtype([("keys", "<u8"), ("vals", "<u8"), ("n", "<u8"), ("dtype", "<i4"), ("pad", "<i4"),
                                ("seed", "<u8")])
        assert _DESC_DTYPE.itemsize == ctypes.sizeof(SortDesc)
    return _DESC_DTYPE


def _addr(t):
    if t is None:
        return 0
    return t.data_ptr() if hasattr(t, "data_ptr") else t.ctypes.data  # numpy


def _code(t):
    c = _DTYPE_CODE.get(t.dtype)
    if c is None:
        c = _DTYPE_CODE[t.dtype] = _dtype_of(t, None)
    return c


def sq_sort_batch(items, stream=None):
    """Sort many independent instances together.  items: iterable of
    (keys, vals_or_None, seed) CUDA tensors; each is sorted in place."""
    import numpy as np

    items = list(items)
    mask = 2**64 - 1
    code = _DTYPE_CODE
    rows = []
    try:
        for k, v, seed in items:  # tensors (the common case, kept lean)
            c = code.get(k.dtype)
            if c is None:
                c = _code(k)
            rows.append((k.data_ptr(), 0 if v is None else v.data_ptr(), k.numel(), c, 0, seed & mask))
    except AttributeError:  # numpy arrays among them
        rows = [(_addr(k), _addr(v), _numel(k), _code(k), 0, seed & mask) for k, v, seed in items]
    descs = np.array(rows or [(0, 0, 0, 0, 0, 0)], dtype=_desc_dtype())
    _check(lib().sq_sort_batch(descs.ctypes.data_as(ctypes.POINTER(SortDesc)), len(items), _stream(stream)))


sort_batch = sq_sort_batch


class Server:
    """Continuous-batching sort server over an HBM budget (sq_serve_*).
    Requests are host numpy arrays sorted in place."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 0, cutoff: int = 0, device: int = 0):
        self._h = ctypes.c_void_p()
        self._keep = {}
        _check(lib().sq_serve_create(ctypes.byref(self._h), hbm_budget_bytes,
                                     ctypes.byref(ServeOpts(max_inflight, cutoff, device))))

    def submit(self, keys, vals=None, seed: int = 0, dtype: str | None = None) -> int:
        if dtype is None:
            dtype = {"uint32": "u32", "int32": "u32", "uint64": "u64", "int64": "u64", "float32": "f32"}[
                str(keys.dtype)]
        d = SortDesc(_ptr(keys), _ptr(vals), keys.size, DTYPES[dtype], seed & (2**64 - 1))
        t = ctypes.c_uint64(0)
        _check(lib().sq_serve_submit(self._h, ctypes.byref(d), ctypes.byref(t)))
        self._keep[t.value] = (keys, vals)  # buffers must outlive the request
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (status, latency_s)."""
        res = ctypes.c_int(0)
        lat = ctypes.c_double(0)
        st = lib().sq_serve_poll(self._h, ticket, ctypes.byref(res), ctypes.byref(lat))
        if st == SQ_PENDING:
            return None
        _check(st)
        self._keep.pop(ticket, None)
        return res.value, lat.value

    def close(self):
        if self._h:
            _check(lib().sq_serve_destroy(self._h))
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------- utilities --

def max_n(dtype: str) -> int:
    return int(lib().sq_max_n(DTYPES[dtype]))


def max_leaf(dtype: str) -> int:
    return int(lib().sq_max_leaf(DTYPES[dtype]))


def set_cutoff(dtype: str, cutoff: int):
    _check(lib().sq_set_cutoff(DTYPES[dtype], cutoff))


def get_cutoff(dtype: str) -> int:
    return int(lib().sq_get_cutoff(DTYPES[dtype]))


def set_cutoff_table(dtype: str, table: dict | list):
    """Cutoffs by size: entry i (a list index or a dict key) applies to sorts
    of floor(log2 n) == i keys; 0 or absent entries use the default cutoff."""
    if isinstance(table, dict):
        arr = [0] * 64
        for lg, c in table.items():
            arr[int(lg)] = int(c)
        while arr and arr[-1] == 0:
            arr.pop()
    else:
        arr = [int(c) for c in table]
    buf = (ctypes.c_uint32 * max(1, len(arr)))(*arr)
    _check(lib().sq_set_cutoff_table(DTYPES[dtype], buf, len(arr)))


LAUNCH_MODES = {"host": 0, "graph": 1, "auto": 2}


def set_launch_mode(mode: str):
    """'host' (a host round trip per recursion round), 'graph' (all rounds in
    one CUDA-graph launch) or 'auto' (currently host rounds everywhere)."""
    _check(lib().sq_set_launch_mode(LAUNCH_MODES[mode]))


def get_launch_mode() -> str:
    m = int(lib().sq_get_launch_mode())
    return {v: k for k, v in LAUNCH_MODES.items()}[m]


RADIX_CLASSES_ALL = 0x7FC


def set_radix_classes(dtype: str, mask: int):
    """Leaf classes (bit c: class c) sorted by the radix base case for a key
    type; the others are merge sorted.  uint64 keys take no radix classes."""
    _check(lib().sq_set_radix_classes(DTYPES[dtype], mask))


def get_radix_classes(dtype: str) -> int:
    return int(lib().sq_get_radix_classes(DTYPES[dtype]))


def cutoff_for(dtype: str, n: int) -> int:
    """The cutoff a sort of n keys uses when the call gives none."""
    return int(lib().sq_cutoff_for(DTYPES[dtype], n))


def load_tuning(path: str | None = None) -> bool:
    """Applies a cutoff table written by paper_2407_14801_gb300.autotune
    (default: tuning.json beside this file).  False if there is none."""
    import json

    path = path or TUNING_PATH
    if not os.path.exists(path):
        return False
    with open(path) as f:
        doc = json.load(f)
    for dtype, table in doc.get("cutoff_by_log2n", {}).items():
        set_cutoff_table(dtype, {int(k): int(v) for k, v in table.items()})
    for dtype, mask in doc.get("radix_classes", {}).items():
        set_radix_classes(dtype, int(mask))
    return True


def stats() -> dict:
    s = Stats()
    lib().sq_stats_get(ctypes.byref(s))
    return dict(launches={f: int(s.launches[i]) for i, f in enumerate(FAMILIES)},
                ms={f: float(s.ms[i]) for i, f in enumerate(FAMILIES)},
                bytes={f: float(s.bytes[i]) for i, f in enumerate(FAMILIES)},
                rounds=int(s.rounds), nodes=int(s.nodes), sorts=int(s.sorts))


def reset_stats():
    lib().sq_stats_reset()


def set_profiling(on: bool):
    lib().sq_set_profiling(1 if on else 0)

"""SquareSort CPU oracle -- TEST INFRASTRUCTURE ONLY.

A thin ctypes wrapper around ``squaresort_oracle.c``, a plain single-threaded
C statement of SquareSort (Algorithms 1-3 of Koucky & Matejka, Section 2).
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA path never does, and this
package never imports the CUDA path.

Every function takes and returns numpy arrays.  Keys are uint32, uint64 or
float32 (float32 is handled by its bit pattern); vals are the uint32 payload.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "squaresort_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsqoracle.so")

DTYPES = {"u32": 0, "u64": 1, "f32": 2}
NP_DTYPE = {"u32": np.uint32, "u64": np.uint64, "f32": np.float32}

OK, ERR_INVALID, ERR_NOMEM, ERR_ATTEMPTS = 0, 1, 2, 7
MAX_ATTEMPTS = 256


class NodeRecord(ctypes.Structure):
    """One record per SquareSort call that recursed (n > cutoff)."""

    _fields_ = [
        ("off", ctypes.c_uint64),
        ("n", ctypes.c_uint64),
        ("m", ctypes.c_uint64),
        ("hash", ctypes.c_uint64),
        ("depth", ctypes.c_uint32),
        ("kind", ctypes.c_uint32),
        ("attempts", ctypes.c_uint32),
        ("index", ctypes.c_uint32),
    ]


def build(force: bool = False, extra_flags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile the oracle with gcc into a shared library; returns its path.

    ``extra_flags`` / ``out`` let a test compile a deliberately broken copy
    (``-D`` switches) to check that the pins catch it.
    """
    out = out or _LIB
    if not force and not extra_flags and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", out, _SRC, *extra_flags]
    subprocess.run(cmd, check=True)
    return out


_lib = None


def _bind(lib):
    u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
    lib.sqo_ordinal.restype = u64
    lib.sqo_ordinal.argtypes = [i32, u64]
    lib.sqo_less.restype = i32
    lib.sqo_less.argtypes = [i32, u64, u32, u64, u32]
    lib.sqo_fmix64.restype = u64
    lib.sqo_fmix64.argtypes = [u64]
    lib.sqo_root_hash.restype = u64
    lib.sqo_root_hash.argtypes = [u64]
    lib.sqo_child_hash.restype = u64
    lib.sqo_child_hash.argtypes = [u64, i32, u64]
    lib.sqo_pivot_draw.restype = u64
    lib.sqo_pivot_draw.argtypes = [u64, u64, u64]
    lib.sqo_scale.restype = u64
    lib.sqo_scale.argtypes = [u64, u64]
    lib.sqo_isqrt_ceil.restype = u64
    lib.sqo_isqrt_ceil.argtypes = [u64]
    lib.sqo_sort.restype = i32
    lib.sqo_sort.argtypes = [i32, vp, vp, u64, u64, u64, i32, vp, u64, ctypes.POINTER(u64), vp, vp]
    if hasattr(lib, "sqo_sort_appendix"):
        lib.sqo_sort_appendix.restype = i32
        lib.sqo_sort_appendix.argtypes = [i32, vp, vp, u64, u64, u64, vp, u64, ctypes.POINTER(u64), vp, vp]
    if hasattr(lib, "sqo_isqrt_floor"):
        lib.sqo_isqrt_floor.restype = u64
        lib.sqo_isqrt_floor.argtypes = [u64]
    lib.sqo_skew_transpose.restype = i32
    lib.sqo_skew_transpose.argtypes = [i32, vp, vp, u64, u64, u64, vp, vp, u64, vp, vp, vp, i32]
    lib.sqo_node_buckets.restype = u32
    lib.sqo_node_buckets.argtypes = [vp, u64, u64, vp]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  A ``path`` loads a
    separately built copy (used by the planted-mistake tests)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _key_bits(keys: np.ndarray, dtype: str) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=NP_DTYPE[dtype])
    return keys.view(np.uint32) if dtype == "f32" else keys


# ------------------------------------------------------------------ helpers --

def ordinal(dtype: str, key_bits: int, lib=None) -> int:
    return int((lib or load()).sqo_ordinal(DTYPES[dtype], int(key_bits)))


def less(dtype: str, ka: int, va: int, kb: int, vb: int, lib=None) -> bool:
    return bool((lib or load()).sqo_less(DTYPES[dtype], int(ka), int(va), int(kb), int(vb)))


def fmix64(z: int, lib=None) -> int:
    return int((lib or load()).sqo_fmix64(z & (2**64 - 1)))


def root_hash(seed: int, lib=None) -> int:
    return int((lib or load()).sqo_root_hash(seed & (2**64 - 1)))


def child_hash(h: int, kind: int, i: int, lib=None) -> int:
    return int((lib or load()).sqo_child_hash(h, kind, i))


def pivot_draw(h: int, attempt: int, r: int, lib=None) -> int:
    return int((lib or load()).sqo_pivot_draw(h, attempt, r))


def scale(u: int, n: int, lib=None) -> int:
    return int((lib or load()).sqo_scale(u, n))


def isqrt_ceil(n: int, lib=None) -> int:
    return int((lib or load()).sqo_isqrt_ceil(n))


def isqrt_floor(n: int, lib=None) -> int:
    return int((lib or load()).sqo_isqrt_floor(n))


# -------------------------------------------------------------- the method --

def sort(keys, vals=None, seed: int = 0, cutoff: int = 16, skew_mode: int = 0, dtype: str = "u32",
         trace_cap: int = 0, root_skew: bool = False, lib=None, variant: str = "algorithm1"):
    """SquareSort (Algorithm 1) of (keys, vals) by (ordinal(key), val).

    Returns ``(keys, vals, trace, root_skew)``: sorted copies, the list of
    per-node records (empty unless ``trace_cap``), and the root's array right
    after its SkewTranspose as ``(keys, vals)`` (or None).
    ``variant="appendix"``: the paper's Appendix listing instead (integer keys;
    floor(sqrt n) columns with a long last one, pivots sampled from the input,
    "<=" buckets; ``skew_mode`` is Algorithm 3 there).
    """
    lib = lib or load()
    kb = _key_bits(keys, dtype).copy()
    n = kb.shape[0]
    vv = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    trace = (NodeRecord * max(trace_cap, 1))()
    cnt = ctypes.c_uint64(0)
    rk = np.empty_like(kb) if root_skew else None
    rv = np.empty(n, dtype=np.uint32) if root_skew else None
    if variant == "appendix":
        st = lib.sqo_sort_appendix(DTYPES[dtype], _ptr(kb), _ptr(vv), n, seed & (2**64 - 1), cutoff,
                                   ctypes.cast(trace, ctypes.c_void_p) if trace_cap else None, trace_cap,
                                   ctypes.byref(cnt), _ptr(rk), _ptr(rv))
    elif variant == "algorithm1":
        st = lib.sqo_sort(DTYPES[dtype], _ptr(kb), _ptr(vv), n, seed & (2**64 - 1), cutoff, skew_mode,
                          ctypes.cast(trace, ctypes.c_void_p) if trace_cap else None, trace_cap,
                          ctypes.byref(cnt), _ptr(rk), _ptr(rv))
    else:
        raise ValueError(variant)
    if st != OK:
        raise RuntimeError(f"oracle sort failed with status {st}")
    recs = [dict(off=r.off, n=r.n, m=r.m, hash=r.hash, depth=r.depth, kind=r.kind, index=r.index,
                 attempts=r.attempts)
            for r in trace[: min(cnt.value, trace_cap)]]
    out_keys = kb.view(np.float32) if dtype == "f32" else kb
    skew = None
    if root_skew:
        skew = (rk.view(np.float32) if dtype == "f32" else rk, rv)
    return out_keys, vv, recs, skew


def skew_transpose(keys, vals, rows: int, cols: int, piv_keys, piv_vals, k: int, dtype: str = "u32",
                   mode: int = 0, lib=None):
    """SkewTranspose of ``cols`` sorted columns of height <= ``rows`` into ``k``
    buckets bounded by ``k-1`` sorted pivots.  ``mode`` 0 = Algorithm 3,
    1 = Algorithm 2 (threshold 4), 2 = Algorithm 2 (threshold 10).
    Returns ``(keys_out, vals_out, bucket_start[k+1])``."""
    lib = lib or load()
    kb = _key_bits(keys, dtype)
    n = kb.shape[0]
    vv = np.ascontiguousarray(vals, dtype=np.uint32)
    pk = _key_bits(piv_keys, dtype)
    pvv = np.ascontiguousarray(piv_vals, dtype=np.uint32)
    assert pk.shape[0] == k - 1 and pvv.shape[0] == k - 1
    ko = np.empty_like(kb)
    vo = np.empty(n, dtype=np.uint32)
    bs = np.empty(k + 1, dtype=np.uint64)
    st = lib.sqo_skew_transpose(DTYPES[dtype], _ptr(kb), _ptr(vv), n, rows, cols, _ptr(pk), _ptr(pvv), k,
                                _ptr(ko), _ptr(vo), _ptr(bs), mode)
    if st != OK:
        raise RuntimeError(f"oracle skew_transpose failed with status {st}")
    return (ko.view(np.float32) if dtype == "f32" else ko), vo, bs


def node_buckets(keys_u64, h: int, lib=None):
    """Column sorts + pivot selection + bucket sizes of one node over distinct
    uint64 keys.  Returns ``(sizes[m], attempts)``; attempts 0 = failure."""
    lib = lib or load()
    k = np.ascontiguousarray(keys_u64, dtype=np.uint64)
    n = k.shape[0]
    m = isqrt_ceil(n, lib)
    sizes = np.zeros(m, dtype=np.uint64)
    att = lib.sqo_node_buckets(_ptr(k), n, h, _ptr(sizes))
    return sizes, int(att)

"""The allocation-free SkewTranspose (sq_skew_transpose_noalloc) against the
allocating one (sq_skew_transpose), through the C ABI.

Callers that cannot allocate device memory at the point of use (a device
already held by other frameworks' pools, or a latency-critical path that must
not call cudaMalloc/cudaFree) use the allocation-free variant; its results must
be exactly those of the regular entry point.  Each shape is run twice in a row
through the allocation-free variant, since calls share one scratch array and
the second call must not depend on what the first left behind.  Collected
last, so that a failure here stops a -x run after every other test has run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VIEW = {"u32": np.int32, "u64": np.int64, "f32": np.int32}


@pytest.fixture(scope="module")
def sq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_14801_gb300 import build

    build.build()
    import paper_2407_14801_gb300 as sq

    sq.lib()
    return sq


def ordinal(dtype, keys):
    if dtype == "f32":
        b = keys.astype(np.uint64)
        nan = (b & 0x7FFFFFFF) > 0x7F800000
        return np.where(nan, 0xFFFFFFFF, np.where(b & 0x80000000, b ^ 0xFFFFFFFF, b | 0x80000000))
    return keys


def make_case(rows, cols, n, k, dtype, seed):
    """cols sorted columns (by ordinal(key), val) and k-1 sorted distinct pivots."""
    rng = np.random.default_rng(seed)
    if dtype == "u64":
        keys = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    elif dtype == "f32":
        keys = rng.standard_normal(n).astype(np.float32).view(np.uint32).copy()
    else:
        keys = rng.integers(0, 7, size=n, dtype=np.uint64).astype(np.uint32)  # many ties
    vals = rng.permutation(n).astype(np.uint32)
    ords = ordinal(dtype, keys)
    for i in range(cols):
        a, b = min(i * rows, n), min((i + 1) * rows, n)
        o = np.lexsort((vals[a:b], ords[a:b]))
        keys[a:b], vals[a:b], ords[a:b] = keys[a:b][o], vals[a:b][o], ords[a:b][o]
    order = np.lexsort((vals, ords))
    pidx = order[np.sort(rng.choice(n, size=k - 1, replace=False))]
    return keys, vals, keys[pidx].copy(), vals[pidx].copy()


def run(fn, dev_in, rows, cols, k, dtype):
    ki, vi, pk, pv = dev_in
    ko, vo = torch.empty_like(ki), torch.empty_like(vi)
    bs = torch.empty(k + 1, dtype=torch.int64, device="cuda")
    fn(ki, vi, rows, cols, pk, pv, k, ko, vo, bs, dtype=dtype)
    torch.cuda.synchronize()
    return ko.cpu().numpy(), vo.cpu().numpy(), bs.cpu().numpy()


@pytest.mark.parametrize("dtype", ["u32", "u64", "f32"])
@pytest.mark.parametrize("shape", [(256, 256, 65536, 256), (1000, 37, 36001, 500), (300, 300, 89999, 129),
                                   (2048, 2048, 4194000, 2048), (5, 3, 13, 4)])
def test_noalloc_equals_regular_twice(sq, dtype, shape):
    rows, cols, n, k = shape
    keys, vals, pk, pv = make_case(rows, cols, n, k, dtype, seed=rows + cols + k)
    dev = lambda a, v: torch.from_numpy(np.ascontiguousarray(a).view(v).copy()).cuda()
    dev_in = (dev(keys, VIEW[dtype]), dev(vals, np.int32), dev(pk, VIEW[dtype]), dev(pv, np.int32))
    ref = run(sq.skew_transpose, dev_in, rows, cols, k, dtype)
    first = run(sq.skew_transpose_noalloc, dev_in, rows, cols, k, dtype)
    second = run(sq.skew_transpose_noalloc, dev_in, rows, cols, k, dtype)
    for got in (first, second):
        for a, b in zip(got, ref):
            assert (a == b).all()  # bit-exact: integer work
    assert int(ref[2][-1]) == n


def test_noalloc_refuses_oversized_shapes(sq):
    rows = cols = k = 16384
    buf = sq.SkewBuf(0, rows * cols, ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256),
                     ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256), k, ctypes.c_void_p(256))
    st = sq.lib().sq_skew_transpose_noalloc(ctypes.byref(buf), rows, cols, None)
    assert st == 1  # SQ_ERR_INVALID, before any device work
    assert b"scratch" in sq.lib().sq_last_error()


def _default_pool():
    """The current device's default stream-ordered memory pool, through the
    CUDA driver API (the pool every cudaMallocAsync without a pool uses)."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int(0)
    assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    return cu, pool


USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # CUmemPool_attribute values


def _pool_attr(cu, pool, attr):
    v = ctypes.c_uint64(0)
    assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


def test_noalloc_takes_nothing_from_the_stream_ordered_pool(sq):
    """What the entry point exists for: a warm call draws no memory from the
    device's default pool (where the regular call's stream-ordered scratch
    comes from).  The pool's high watermark is reset before the call and
    must not rise above the pool's use at that moment."""
    rows, cols, n, k = 2048, 2048, 4194000, 2048
    keys, vals, pk, pv = make_case(rows, cols, n, k, "u32", seed=5)
    dev = lambda a, v: torch.from_numpy(np.ascontiguousarray(a).view(v).copy()).cuda()
    dev_in = (dev(keys, np.int32), dev(vals, np.int32), dev(pk, np.int32), dev(pv, np.int32))
    ref = run(sq.skew_transpose, dev_in, rows, cols, k, "u32")
    cu, pool = _default_pool()
    used_high_regular = None
    run(sq.skew_transpose_noalloc, dev_in, rows, cols, k, "u32")  # warm: the array is reserved here
    torch.cuda.synchronize()
    for fn in (sq.skew_transpose, sq.skew_transpose_noalloc):
        used0 = _pool_attr(cu, pool, USED_MEM_CURRENT)
        zero = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0
        got = run(fn, dev_in, rows, cols, k, "u32")
        high = _pool_attr(cu, pool, USED_MEM_HIGH)
        if fn is sq.skew_transpose:
            used_high_regular = high - used0  # the check below can see an allocation
        else:
            assert high <= used0, f"the allocation-free call drew {high - used0} bytes from the pool"
        for a, b in zip(got, ref):
            assert (a == b).all()
    assert used_high_regular > 0

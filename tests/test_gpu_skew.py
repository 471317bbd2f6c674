"""GPU parity of the stand-alone SkewTranspose (sq_skew_transpose) against the
oracle's Algorithm 3 / Algorithm 2 on shapes from 1x1 to hundreds of columns,
ragged last columns, k different from the number of columns, and key
alphabets small enough that most comparisons are decided by the payload."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VIEW = {"u32": np.int32, "u64": np.int64, "f32": np.int32}
NP = {"u32": np.uint32, "u64": np.uint64, "f32": np.uint32}


@pytest.fixture(scope="module")
def sq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_14801_gb300 as sq

    sq.lib()
    return sq


def make(rows, cols, n, k, dtype, alphabet, seed):
    rng = np.random.default_rng(seed)
    if dtype == "f32":
        keys = W.normal_f32(n, seed, 0.05, 0.05, 0.05).view(np.uint32).copy()
        if alphabet:
            keys = (keys % np.uint32(alphabet)) | np.uint32(0x3F800000)
    elif dtype == "u64":
        keys = rng.integers(0, alphabet or (1 << 63), size=n, dtype=np.uint64)
    else:
        keys = rng.integers(0, alphabet or (1 << 32), size=n, dtype=np.uint64).astype(np.uint32)
    vals = rng.permutation(n).astype(np.uint32)
    ords = np.array([oracle.ordinal(dtype, int(b)) for b in keys], dtype=np.uint64)
    for i in range(cols):
        a, b = min(i * rows, n), min((i + 1) * rows, n)
        o = np.lexsort((vals[a:b], ords[a:b]))
        keys[a:b], vals[a:b], ords[a:b] = keys[a:b][o], vals[a:b][o], ords[a:b][o]
    # k-1 sorted distinct pivots drawn from the elements
    order = np.lexsort((vals, ords))
    pidx = order[np.sort(rng.choice(n, size=min(k - 1, n), replace=False))] if n else np.array([], int)
    if len(pidx) < k - 1:
        return None
    return keys, vals, keys[pidx].copy(), vals[pidx].copy()


def run_case(sq, rows, cols, n, k, dtype, alphabet, seed):
    case = make(rows, cols, n, k, dtype, alphabet, seed)
    if case is None:
        return
    keys, vals, pk, pv = case
    okey = keys.view(np.float32) if dtype == "f32" else keys
    ek, ev, eb = oracle.skew_transpose(okey, vals, rows, cols, pk.view(np.float32) if dtype == "f32" else pk, pv,
                                       k, dtype=dtype, mode=1)
    dev = lambda a, v: torch.from_numpy(np.ascontiguousarray(a).view(v).copy()).cuda()
    ki, vi = dev(keys, VIEW[dtype]), dev(vals, np.int32)
    ko, vo = torch.empty_like(ki), torch.empty_like(vi)
    bs = torch.empty(k + 1, dtype=torch.int64, device="cuda")
    sq.skew_transpose(ki, vi, rows, cols, dev(pk, VIEW[dtype]), dev(pv, np.int32), k, ko, vo, bs, dtype=dtype)
    torch.cuda.synchronize()
    gk = ko.cpu().numpy().view(NP[dtype])
    gv = vo.cpu().numpy().view(np.uint32)
    ekb = ek.view(np.uint32) if dtype == "f32" else ek
    assert (gk == ekb).all() and (gv == ev).all(), (rows, cols, n, k, dtype)
    assert (bs.cpu().numpy().astype(np.uint64) == eb).all()


def test_every_small_shape(sq):
    seed = 0
    for rows in range(1, 17):
        for cols in range(1, 17):
            for k in sorted({1, 2, cols, min(cols + 3, 40), 17}):
                seed += 1
                n = rows * cols - (seed % rows)
                run_case(sq, rows, cols, n, k, "u32", 3, seed)


@pytest.mark.parametrize("dtype", ["u32", "u64", "f32"])
@pytest.mark.parametrize("shape", [(256, 256, 65536, 256), (256, 256, 65300, 256), (1000, 37, 36001, 500),
                                   (37, 1000, 36999, 1000), (130, 130, 16900, 64), (130, 130, 16899, 65),
                                   (300, 300, 90000, 129), (64, 200, 12800, 3000)])
@pytest.mark.parametrize("alphabet", [0, 5])
def test_larger_shapes(sq, dtype, shape, alphabet):
    rows, cols, n, k = shape
    if dtype != "u32" and k > 8193:
        pytest.skip("k beyond the pivot capacity of this key type")
    run_case(sq, rows, cols, n, k, dtype, alphabet, rows * 7 + cols + k)


def test_transpose_special_case(sq):
    """Columns holding one element of every bucket: a plain transpose."""
    for m in (1, 2, 3, 64, 65, 127, 300):
        r, c = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        keys = (r * m + c).T.reshape(-1).astype(np.uint32)
        vals = np.arange(m * m, dtype=np.uint32)
        pk = (np.arange(1, m) * m).astype(np.uint32)
        pv = np.zeros(m - 1, dtype=np.uint32)
        dev = lambda a: torch.from_numpy(a.view(np.int32).copy()).cuda()
        ki, vi = dev(keys), dev(vals)
        ko, vo = torch.empty_like(ki), torch.empty_like(vi)
        bs = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        sq.skew_transpose(ki, vi, m, m, dev(pk), dev(pv), m, ko, vo, bs, dtype="u32")
        assert (ko.cpu().numpy().view(np.uint32) == np.arange(m * m)).all()

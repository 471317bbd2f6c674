"""Pins for the oracle's SkewTranspose (Algorithms 2 and 3, Section 2.2).

The brute force below is the operation's definition: a stable partition of
the column-major array by bucket id, where an element's bucket is the number
of pivots it is not below.  Algorithm 3 and Algorithm 2 (thresholds 4 and 10)
must all equal it on every shape up to 16x16, and on the special case where
every column holds one element of every bucket the result is a plain matrix
transpose.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W


def brute_force(keys, vals, rows, cols, pk, pv, k):
    n = keys.size
    piv = list(zip(pk.tolist(), pv.tolist()))
    bucket = np.array([sum(1 for p in piv if p <= (int(a), int(b))) for a, b in zip(keys, vals)],
                      dtype=np.int64)
    order = np.argsort(bucket, kind="stable")
    starts = np.concatenate([[0], np.cumsum(np.bincount(bucket, minlength=k))])
    return keys[order], vals[order], starts


def make_case(rows, cols, n, k, alphabet, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, alphabet, size=n).astype(np.uint32)
    vals = rng.permutation(n).astype(np.uint32)
    for i in range(cols):  # sort every column by (key, val)
        a, b = min(i * rows, n), min((i + 1) * rows, n)
        o = np.lexsort((vals[a:b], keys[a:b]))
        keys[a:b], vals[a:b] = keys[a:b][o], vals[a:b][o]
    # k-1 distinct sorted pivots (any (key, val) pairs; they need not be elements)
    pool = sorted({(int(rng.integers(0, alphabet)), int(rng.integers(0, n + 2))) for _ in range(4 * k)})
    if len(pool) < k - 1:
        return None
    idx = np.sort(rng.choice(len(pool), size=k - 1, replace=False))
    pk = np.array([pool[i][0] for i in idx], dtype=np.uint32)
    pv = np.array([pool[i][1] for i in idx], dtype=np.uint32)
    return keys, vals, pk, pv


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_every_shape_up_to_16(mode):
    seed = 0
    for rows in range(1, 17):
        for cols in range(1, 17):
            for k in sorted({1, 2, 3, 4, 5, cols, min(16, cols + 3), 16}):
                seed += 1
                n_full = rows * cols
                for n in {n_full, max(0, n_full - rows + 1), max(0, n_full - rows)}:
                    case = make_case(rows, cols, n, k, alphabet=3, seed=seed)
                    if case is None:
                        continue
                    keys, vals, pk, pv = case
                    ko, vo, bs = oracle.skew_transpose(keys, vals, rows, cols, pk, pv, k, mode=mode)
                    ek, ev, es = brute_force(keys, vals, rows, cols, pk, pv, k)
                    assert (ko == ek).all() and (vo == ev).all(), (rows, cols, n, k)
                    assert (bs == es).all()


def test_exhaustive_small():
    """All key matrices over {0,1,2} with rows, cols <= 2 and every pivot set."""
    elems = [(a, b) for a in range(3) for b in range(5)]
    for rows, cols in itertools.product([1, 2], [1, 2]):
        n = rows * cols
        for keys_t in itertools.product(range(3), repeat=n):
            keys = np.array(keys_t, dtype=np.uint32)
            vals = np.arange(n, dtype=np.uint32)
            for i in range(cols):
                a, b = i * rows, (i + 1) * rows
                o = np.lexsort((vals[a:b], keys[a:b]))
                keys[a:b], vals[a:b] = keys[a:b][o], vals[a:b][o]
            for k in (1, 2, 3):
                for piv in itertools.combinations(elems, k - 1):
                    pk = np.array([p[0] for p in piv], dtype=np.uint32)
                    pv = np.array([p[1] for p in piv], dtype=np.uint32)
                    ek, ev, es = brute_force(keys, vals, rows, cols, pk, pv, k)
                    for mode in (0, 1):
                        ko, vo, bs = oracle.skew_transpose(keys, vals, rows, cols, pk, pv, k, mode=mode)
                        assert (ko == ek).all() and (vo == ev).all() and (bs == es).all()


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 8, 16, 31, 64])
def test_transpose_special_case(m):
    """Column c holds r*m + c at row r; pivots i*m.  Each column has one
    element of each bucket, so SkewTranspose is the matrix transpose: the
    output is 0, 1, ..., m*m - 1."""
    r, c = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    keys = (r * m + c).T.reshape(-1).astype(np.uint32)  # column-major
    vals = np.arange(m * m, dtype=np.uint32)
    pk = (np.arange(1, m) * m).astype(np.uint32)
    pv = np.zeros(m - 1, dtype=np.uint32)
    for mode in (0, 1, 2):
        ko, vo, bs = oracle.skew_transpose(keys, vals, m, m, pk, pv, m, mode=mode)
        assert (ko == np.arange(m * m)).all()
        assert (bs == np.arange(0, m * m + 1, m)).all()


@pytest.mark.parametrize("dtype", ["u64", "f32"])
def test_wide_and_float_keys(dtype):
    rng = np.random.default_rng(7)
    rows, cols, k = 12, 9, 7
    n = rows * cols - 5
    keys = W.zipf_u64(n, 3) % np.uint64(5) if dtype == "u64" else W.normal_f32(n, 3, 0.1, 0.1, 0.1)
    vals = rng.permutation(n).astype(np.uint32)
    bits = keys.view(np.uint32) if dtype == "f32" else keys
    ords = np.array([oracle.ordinal(dtype, int(b)) for b in bits], dtype=np.uint64)
    for i in range(cols):
        a, b = min(i * rows, n), min((i + 1) * rows, n)
        o = np.lexsort((vals[a:b], ords[a:b]))
        keys[a:b], vals[a:b], ords[a:b] = keys[a:b][o], vals[a:b][o], ords[a:b][o]
    sel = np.sort(rng.choice(n, size=k - 1, replace=False))
    allo = np.lexsort((vals, ords))
    pidx = allo[sel]
    pk, pv = keys[pidx], vals[pidx]
    # expected: stable partition by bucket computed on ordinals
    piv = list(zip(ords[pidx].tolist(), pv.tolist()))
    bucket = np.array([sum(1 for p in piv if p <= (int(a), int(b))) for a, b in zip(ords, vals)])
    order = np.argsort(bucket, kind="stable")
    for mode in (0, 1, 2):
        ko, vo, bs = oracle.skew_transpose(keys, vals, rows, cols, pk, pv, k, dtype=dtype, mode=mode)
        assert (vo == vals[order]).all()
        kb = ko.view(np.uint32) if dtype == "f32" else ko
        assert (kb == bits[order]).all()

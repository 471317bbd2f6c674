"""Pins for the oracle's SquareSort (Algorithm 1).

* The final output is the plain definition of sorting: numpy's lexsort on
  (ordinal(key), val) -- for every dtype, distribution, size and cutoff.
* The root's array after its SkewTranspose is recomputed here from the
  definitions (column spans, column sorts, pivot redraw rule, bucket order,
  stable partition), so the intermediate state of Algorithm 1 is pinned too.
* Per-node invariants from Section 3 (bucket sizes, recursion shape).
"""
import numpy as np
import pytest

import oracle
import workloads as W


def ords_of(dtype, keys):
    if dtype == "f32":
        return np.array([oracle.ordinal("f32", int(b)) for b in keys.view(np.uint32)], dtype=np.uint64)
    return keys.astype(np.uint64)


def check_sorted(dtype, keys, vals, ko, vo):
    o = ords_of(dtype, keys)
    ref = np.lexsort((vals, o))
    kb = (lambda a: a.view(np.uint32)) if dtype == "f32" else (lambda a: a)
    assert (vo == vals[ref]).all()
    assert (kb(ko) == kb(keys)[ref]).all()


@pytest.mark.parametrize("cutoff", [2, 3, 16, 100, 1000])
@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "distinct16"])
def test_u32_matches_library_sort(cutoff, dist):
    for n in [0, 1, 2, 3, 4, 15, 16, 17, 100, 257, 3000]:
        keys = W.U32_DISTRIBUTIONS[dist](n, 1000 + n)
        vals = W.iota(n)
        ko, vo, _, _ = oracle.sort(keys, vals, seed=n, cutoff=cutoff)
        check_sorted("u32", keys, vals, ko, vo)


@pytest.mark.parametrize("cutoff", [2, 16, 256])
def test_ties_resolved_by_val(cutoff):
    rng = np.random.default_rng(1)
    for alphabet in (1, 2, 3):
        n = 2000
        keys = W.small_alphabet_u32(n, alphabet, alphabet)
        vals = rng.permutation(n).astype(np.uint32)  # not iota: order comes from the compare
        ko, vo, _, _ = oracle.sort(keys, vals, seed=alphabet, cutoff=cutoff)
        check_sorted("u32", keys, vals, ko, vo)


@pytest.mark.parametrize("cutoff", [2, 16, 300])
def test_u64_zipf(cutoff):
    n = 5000
    keys = W.zipf_u64(n, 4)
    vals = W.iota(n)
    ko, vo, _, _ = oracle.sort(keys, vals, seed=9, cutoff=cutoff, dtype="u64")
    check_sorted("u64", keys, vals, ko, vo)
    big = W.uniform_u64(n, 5)
    ko, vo, _, _ = oracle.sort(big, vals, seed=9, cutoff=cutoff, dtype="u64")
    check_sorted("u64", big, vals, ko, vo)


@pytest.mark.parametrize("cutoff", [2, 16, 300])
def test_f32_specials(cutoff):
    n = 5000
    keys = W.normal_f32(n, 6, p_inf=0.02, p_negzero=0.02, p_nan=0.02)
    keys[::50] = np.float32(0.0)
    vals = W.iota(n)
    ko, vo, _, _ = oracle.sort(keys, vals, seed=2, cutoff=cutoff, dtype="f32")
    check_sorted("f32", keys, vals, ko, vo)
    nan_bits = ko.view(np.uint32)[np.isnan(ko)]
    assert sorted(nan_bits.tolist()) == sorted(keys.view(np.uint32)[np.isnan(keys)].tolist())


def test_null_vals_uses_position():
    keys = W.distinct16_u32(3000, 3)
    ko, vo, _, _ = oracle.sort(keys, None, seed=1, cutoff=16)
    assert vo is None
    check_sorted("u32", keys, W.iota(3000), ko, W.iota(3000)[np.lexsort((W.iota(3000), keys))])


@pytest.mark.parametrize("skew_mode", [0, 1, 2])
def test_skew_modes_same_result(skew_mode):
    keys = W.uniform_u32(20000, 8)
    vals = W.iota(20000)
    ko, vo, tr, sk = oracle.sort(keys, vals, seed=8, cutoff=64, skew_mode=skew_mode, trace_cap=10000,
                                root_skew=True)
    k0, v0, tr0, sk0 = oracle.sort(keys, vals, seed=8, cutoff=64, skew_mode=0, trace_cap=10000,
                                   root_skew=True)
    check_sorted("u32", keys, vals, ko, vo)
    assert tr == tr0 and (sk[1] == sk0[1]).all()


# ----------------------------------------- the root step, from definitions --

def root_step_from_definitions(keys, vals, seed):
    """Columns, column sorts, pivots (with the redraw rule) and the stable
    partition by bucket, each written from the paper's text."""
    n = keys.size
    m = oracle.isqrt_ceil(n)
    cols = [(min(i * m, n), min((i + 1) * m, n)) for i in range(m)]
    k, v = keys.copy(), vals.copy()
    for a, b in cols:
        o = np.lexsort((v[a:b], k[a:b]))
        k[a:b], v[a:b] = k[a:b][o], v[a:b][o]
    D = list(zip(k.tolist(), v.tolist()))
    mn = min(D[a] for a, b in cols if b > a)
    h = oracle.root_hash(seed)
    for attempt in range(oracle.MAX_ATTEMPTS):
        P = sorted(D[oracle.scale(oracle.pivot_draw(h, attempt, r), n)] for r in range(m - 1))
        if P[0] != mn and all(P[i] != P[i + 1] for i in range(len(P) - 1)):
            break
    else:
        raise AssertionError("no pivot sample accepted")
    bucket = np.array([sum(1 for p in P if p <= e) for e in D])  # e in bucket j iff p_j <= e < p_{j+1}
    order = np.argsort(bucket, kind="stable")
    return k[order], v[order], attempt + 1


@pytest.mark.parametrize("n,cutoff", [(17, 16), (50, 8), (257, 16), (1000, 40), (4096, 64), (5000, 100)])
@pytest.mark.parametrize("dist", ["uniform", "distinct16"])
def test_root_skew_from_definitions(n, cutoff, dist):
    keys = W.U32_DISTRIBUTIONS[dist](n, n + 7)
    vals = np.random.default_rng(n).permutation(n).astype(np.uint32)
    ek, ev, att = root_step_from_definitions(keys, vals, seed=n)
    ko, vo, tr, (sk, sv) = oracle.sort(keys, vals, seed=n, cutoff=cutoff, trace_cap=100000, root_skew=True)
    assert (sk == ek).all() and (sv == ev).all()
    root = [r for r in tr if r["depth"] == 0]
    assert len(root) == 1 and root[0]["attempts"] == att and root[0]["m"] == oracle.isqrt_ceil(n)
    check_sorted("u32", keys, vals, ko, vo)


def test_trace_shape_and_invariants():
    """Every recursing node: n > cutoff, m = ceil(sqrt n), column children have
    n <= parent m, bucket children have n <= parent n - m + 1 (Section 3,
    space bound), hashes follow the path rule."""
    n, cutoff = 30000, 16
    keys = W.uniform_u32(n, 12)
    _, _, tr, _ = oracle.sort(keys, W.iota(n), seed=12, cutoff=cutoff, trace_cap=100000)
    roots = [r for r in tr if r["depth"] == 0]
    assert len(roots) == 1 and roots[0]["hash"] == oracle.root_hash(12) and roots[0]["kind"] == 0
    for r in tr:
        assert r["n"] > cutoff and r["m"] == oracle.isqrt_ceil(r["n"]) and r["attempts"] >= 1
    # The oracle records a node after its column children and before its
    # bucket children, so a column child's parent is the first later record
    # one level up that contains it, and a bucket child's the last earlier one.
    def contains(p, r):
        return p["off"] <= r["off"] and r["off"] + r["n"] <= p["off"] + p["n"]

    for idx, r in enumerate(tr):
        if r["depth"] == 0:
            continue
        if r["kind"] == 1:
            p = next(q for q in tr[idx + 1:] if q["depth"] == r["depth"] - 1 and contains(q, r))
            i = (r["off"] - p["off"]) // p["m"]
            assert r["off"] == p["off"] + i * p["m"]
            assert r["n"] == min(p["m"], p["n"] - i * p["m"])
            assert r["hash"] == oracle.child_hash(p["hash"], 1, i)
        else:
            assert r["kind"] == 2
            p = next(q for q in reversed(tr[:idx]) if q["depth"] == r["depth"] - 1 and contains(q, r))
            assert r["n"] <= p["n"] - p["m"] + 1
            assert r["hash"] == oracle.child_hash(p["hash"], 2, r["index"]) and r["index"] < p["m"]
        if r["kind"] == 1:
            assert r["index"] == i

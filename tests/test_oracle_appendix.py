"""Pins for the oracle's appendix variant (the paper's Appendix listing, which
Section 2.1 says deviates slightly from Algorithm 1), each against something
other than the oracle itself:

  - the final output against numpy's lexsort on (key, val), integer keys;
  - every traced node's shape from its definition: m = floor(sqrt n) (Python's
    math.isqrt), one pivot sample (no redraws), the column children's sizes
    (m each, the last one n - (m-1)m) and their offsets, and the children's
    hashes by the random source restated in Python integers;
  - the root's array right after its SkewTranspose recomputed from the
    listing's steps in Python: m draws with replacement from the input
    before the column sorts, sorted, the largest replaced by +inf, a sample
    equal to its neighbour above replaced by its predecessor, buckets
    { e : pivots[i-1] < e <= pivots[i] }, and the stable partition of the
    column-sorted array by bucket.
A set of planted mistakes (strict bucket bounds, ceil instead of floor, the
last column not extended, pivots sampled after the column sorts, no
duplicate separation) each fails at least one of these pins.
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_rng_restated import F, bucket_child, column_child, draw, position

SRC = os.path.join(os.path.dirname(oracle.__file__), "squaresort_oracle.c")


def lexsorted(keys, vals):
    o = np.lexsort((vals, keys))
    return keys[o], vals[o]


def inputs():
    yield "uniform_u32", W.uniform_u32(50000, 1), "u32"
    yield "alphabet_u32", W.small_alphabet_u32(40000, 2, 7), "u32"
    yield "sorted_u32", W.sorted_u32(30001, 3), "u32"
    yield "reverse_u32", W.reverse_u32(30000, 4), "u32"
    yield "square_u32", W.uniform_u32(4096, 5), "u32"
    yield "zipf_u64", W.zipf_u64(40000, 6), "u64"
    yield "extremes_u32", np.array([0, 0xFFFFFFFF] * 3000, dtype=np.uint32), "u32"


@pytest.mark.parametrize("cutoff", [3, 4, 16, 64, 999])
def test_output_is_lexsort(cutoff):
    for name, keys, dt in inputs():
        for vals in (W.iota(keys.size), np.random.default_rng(7).permutation(keys.size).astype(np.uint32)):
            ok, ov, _, _ = oracle.sort(keys, vals, seed=11, cutoff=cutoff, dtype=dt, variant="appendix")
            ek, ev = lexsorted(keys, vals)
            assert (ok == ek).all() and (ov == ev).all(), (name, cutoff)


def test_float_keys_and_cutoff_2_refused():
    with pytest.raises(RuntimeError):
        oracle.sort(W.normal_f32(1000, 1), W.iota(1000), dtype="f32", cutoff=16, variant="appendix")
    with pytest.raises(RuntimeError):  # floor(sqrt 3) = 1: one column as large as the node
        oracle.sort(W.uniform_u32(1000, 1), W.iota(1000), cutoff=2, variant="appendix")


def test_node_shapes_and_hashes_follow_the_listing():
    for seed, n in [(1, 100000), (2, 65536), (3, 5000), (4, 1000003)]:
        keys = W.uniform_u32(n, 40 + seed)
        _, _, trace, _ = oracle.sort(keys, W.iota(n), seed=seed, cutoff=40, trace_cap=1 << 20, variant="appendix")
        assert trace
        by_depth = {}
        for r in trace:
            by_depth.setdefault(r["depth"], []).append(r)
            assert r["m"] == math.isqrt(r["n"]) and r["attempts"] == 1
        root = [r for r in trace if r["depth"] == 0]
        assert len(root) == 1 and root[0]["hash"] == F(seed) and root[0]["n"] == n
        for r in trace:
            if r["depth"] == 0:
                continue
            cands = [p for p in by_depth[r["depth"] - 1]
                     if p["off"] <= r["off"] and r["off"] + r["n"] <= p["off"] + p["n"]]
            child = column_child if r["kind"] == 1 else bucket_child
            parents = [p for p in cands if child(p["hash"], r["index"]) == r["hash"]]
            assert len(parents) == 1
            p = parents[0]
            if r["kind"] == 1:
                m = p["m"]
                assert r["off"] == p["off"] + r["index"] * m
                want = m if r["index"] + 1 < m else p["n"] - (m - 1) * m
                assert r["n"] == want


def pred(e):
    k, v = e
    if v > 0:
        return (k, v - 1)
    if k > 0:
        return (k - 1, 0xFFFFFFFF)
    return e


def root_skew_from_the_listing(keys, vals, seed):
    """The root's post-SkewTranspose array, restated from the listing."""
    n = keys.size
    m = math.isqrt(n)
    A = list(zip((int(k) for k in keys), (int(v) for v in vals)))
    h = F(seed)
    smp = sorted(A[position(draw(h, 0, r), n)] for r in range(m))
    piv = smp[: m - 1]  # index m-1 becomes +inf
    for r in range(m - 2):
        if piv[r] == piv[r + 1]:
            piv[r] = pred(piv[r])
    D = []
    for i in range(m):
        lo, hi = i * m, (n if i + 1 == m else (i + 1) * m)
        D.extend(sorted(A[lo:hi]))

    def bucket(e):  # the first i with e <= pivots[i]; m-1 if none
        for i, p in enumerate(piv):
            if e <= p:
                return i
        return m - 1

    out = []
    for b in range(m):
        out.extend(e for e in D if bucket(e) == b)
    return out


def test_root_skew_from_the_listing():
    """Small nodes (m draws from a few dozen positions: repeated draws and
    so separated duplicates are frequent) and ties resolved by the payload."""
    checked = dup = 0
    for seed in range(60):
        n = 20 + (seed * 13) % 90
        keys = W.small_alphabet_u32(n, 100 + seed, 6) if seed % 2 else W.uniform_u32(n, 100 + seed)
        vals = np.random.default_rng(seed).permutation(n).astype(np.uint32)
        _, _, _, rs = oracle.sort(keys, vals, seed=seed, cutoff=3, root_skew=True, variant="appendix")
        got = list(zip((int(k) for k in rs[0]), (int(v) for v in rs[1])))
        assert got == root_skew_from_the_listing(keys, vals, seed), seed
        m = math.isqrt(n)
        pos = [position(draw(F(seed), 0, r), n) for r in range(m)]
        dup += len(set(pos)) < len(pos)
        checked += 1
    assert checked == 60 and dup >= 10


MUTANTS = {
    "strict_bounds": ("  if (c->variant) return !elem_less(c->dtype, &pv->p[idx], e); /* appendix: bucket i holds e <= pivot i */",
                      "  if (c->variant) return elem_less(c->dtype, e, &pv->p[idx]);"),
    "ceil_geometry": ("  const uint64_t m = sqo_isqrt_floor(n);", "  const uint64_t m = sqo_isqrt_ceil(n);"),
    "short_last_column": ("    last[i] = (i + 1 < m) ? (i + 1) * m : n;", "    last[i] = (i + 1) * m < n ? (i + 1) * m : n;"),
    "sample_after_sorts": ("  appendix_pivots(c, A, n, m, h, smp);\n", ""),
    "no_separation": ("    if (elem_equal(c->dtype, &smp[r], &smp[r + 1])) smp[r] = elem_pred(smp[r]);", "    ;"),
}


def _battery(lib):
    """A compact run of the pins above against a built copy; returns the
    first failing check's name or None."""
    try:
        for name, keys, dt in list(inputs())[:3]:
            ok, ov, _, _ = oracle.sort(keys, W.iota(keys.size), seed=3, cutoff=16, dtype=dt, lib=lib,
                                       variant="appendix")
            ek, ev = lexsorted(keys, W.iota(keys.size))
            if not ((ok == ek).all() and (ov == ev).all()):
                return "output"
        for seed in range(30):
            n = 20 + (seed * 13) % 90
            keys = W.small_alphabet_u32(n, 100 + seed, 6) if seed % 2 else W.uniform_u32(n, 100 + seed)
            vals = np.random.default_rng(seed).permutation(n).astype(np.uint32)
            _, _, _, rs = oracle.sort(keys, vals, seed=seed, cutoff=3, root_skew=True, lib=lib, variant="appendix")
            got = list(zip((int(k) for k in rs[0]), (int(v) for v in rs[1])))
            if got != root_skew_from_the_listing(keys, vals, seed):
                return "root_skew"
        n = 100000
        _, _, trace, _ = oracle.sort(W.uniform_u32(n, 9), W.iota(n), seed=2, cutoff=40, trace_cap=1 << 20, lib=lib,
                                     variant="appendix")
        for r in trace:
            if r["m"] != math.isqrt(r["n"]):
                return "shape"
    except Exception as e:  # a crash is a caught mistake too
        return f"raised {type(e).__name__}"
    return None


def _build(tmp, name, edit):
    text = open(SRC).read()
    if edit is not None:
        old, new = edit
        assert text.count(old) == 1, f"mutation anchor for {name} not unique"
        text = text.replace(old, new)
    src = os.path.join(tmp, f"{name}.c")
    with open(src, "w") as f:
        f.write(text)
    out = os.path.join(tmp, f"{name}.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", out, src], check=True)
    return oracle.load(out)


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="sqo_appendix_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_pristine_passes_battery(tmpdir_mod):
    assert _battery(_build(tmpdir_mod, "pristine", None)) is None


def _battery_in_child(so_path):
    """The battery in a child process (a planted mistake may crash the
    oracle outright, which also counts as caught)."""
    import sys

    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path[:0] = [%r, %r]\n"
            "import oracle, test_oracle_appendix as t\n"
            "r = t._battery(oracle.load(%r))\n"
            "print('CAUGHT' if r else 'MISSED', r)\n") % (here, os.path.dirname(here), so_path)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    return p.returncode != 0 or "CAUGHT" in p.stdout


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmpdir_mod, name):
    _build(tmpdir_mod, name, MUTANTS[name])
    assert _battery_in_child(os.path.join(tmpdir_mod, f"{name}.so")), name

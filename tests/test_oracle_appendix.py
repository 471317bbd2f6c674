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
    before the column sorts, sorted, the largest replaced by the greatest
    pair (the listing's INT_MAX), a sample equal to its neighbour above
    replaced by its predecessor, buckets
    { e : pivots[i-1] < e <= pivots[i] }, and the stable partition of the
    column-sorted array by bucket.
  - with repeated (key, val) pairs, which buckets recurse: the root's pivots
    and bucket contents recomputed in Python, a bucket whose range holds a
    single pair copied (no trace record), every other bucket above the
    cutoff recursing; and inputs made of one repeated pair (the least, the
    greatest, one in between) sorted at all.
A set of planted mistakes (strict bucket bounds, ceil instead of floor, the
last column not extended, pivots sampled after the column sorts, no
duplicate separation, no monochromatic copy, no copy of bucket 0 at the
least pair, +inf as a flag that the last sample is never compared with)
each fails at least one of these pins.
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


@pytest.mark.parametrize("cutoff", [8, 9, 16, 64, 999])
def test_output_is_lexsort(cutoff):
    for name, keys, dt in inputs():
        for vals in (W.iota(keys.size), np.random.default_rng(7).permutation(keys.size).astype(np.uint32)):
            ok, ov, _, _ = oracle.sort(keys, vals, seed=11, cutoff=cutoff, dtype=dt, variant="appendix")
            ek, ev = lexsorted(keys, vals)
            assert (ok == ek).all() and (ov == ev).all(), (name, cutoff)


def test_float_keys_and_cutoffs_below_8_refused():
    with pytest.raises(RuntimeError):
        oracle.sort(W.normal_f32(1000, 1), W.iota(1000), dtype="f32", cutoff=16, variant="appendix")
    with pytest.raises(RuntimeError):  # floor(sqrt 8) = 2: a node of equal elements could be its own bucket
        oracle.sort(W.uniform_u32(1000, 1), W.iota(1000), cutoff=7, variant="appendix")


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


TOP = {"u32": (0xFFFFFFFF, 0xFFFFFFFF), "u64": (2**64 - 1, 0xFFFFFFFF)}


def root_pivots_from_the_listing(A, seed, dt="u32"):
    """The root's m pivots: m draws from the input, sorted, the largest
    replaced by the greatest pair, a sample equal to the next one lowered to
    its predecessor.  Bucket i is (pivots[i-1], pivots[i]]."""
    n = len(A)
    m = math.isqrt(n)
    h = F(seed)
    smp = sorted(A[position(draw(h, 0, r), n)] for r in range(m))
    smp[m - 1] = TOP[dt]
    for r in range(m - 1):
        if smp[r] == smp[r + 1]:
            smp[r] = pred(smp[r])
    return smp


def root_skew_from_the_listing(keys, vals, seed):
    """The root's post-SkewTranspose array, restated from the listing."""
    n = keys.size
    m = math.isqrt(n)
    A = list(zip((int(k) for k in keys), (int(v) for v in vals)))
    piv = root_pivots_from_the_listing(A, seed)
    D = []
    for i in range(m):
        lo, hi = i * m, (n if i + 1 == m else (i + 1) * m)
        D.extend(sorted(A[lo:hi]))

    def bucket(e):  # the first i with e <= pivots[i] (pivots[m-1] is the greatest pair)
        for i, p in enumerate(piv):
            if e <= p:
                return i

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
        _, _, _, rs = oracle.sort(keys, vals, seed=seed, cutoff=8, root_skew=True, variant="appendix")
        got = list(zip((int(k) for k in rs[0]), (int(v) for v in rs[1])))
        assert got == root_skew_from_the_listing(keys, vals, seed), seed
        m = math.isqrt(n)
        pos = [position(draw(F(seed), 0, r), n) for r in range(m)]
        dup += len(set(pos)) < len(pos)
        checked += 1
    assert checked == 60 and dup >= 10


def one_pair_inputs():
    for dt in ("u32", "u64"):
        top_k, top_v = TOP[dt]
        kdt = np.uint32 if dt == "u32" else np.uint64
        for k, v in [(0, 0), (top_k, top_v), (5, 7)]:
            for n in (4, 40, 3000):
                yield dt, np.full(n, k, dtype=kdt), np.full(n, v, dtype=np.uint32)
    # two pairs only, and the least pair next to a few others
    k = np.array([0, 0, 1] * 700, dtype=np.uint32)
    yield "u32", k, np.zeros(k.size, dtype=np.uint32)
    k = np.array([3, 3, 3, 4] * 500, dtype=np.uint32)
    yield "u32", k, np.array([9, 9, 9, 0] * 500, dtype=np.uint32)


@pytest.mark.parametrize("cutoff", [8, 16, 100])
def test_repeated_pairs_sort(cutoff):
    for dt, keys, vals in one_pair_inputs():
        ok, ov, _, _ = oracle.sort(keys, vals, seed=5, cutoff=cutoff, dtype=dt, variant="appendix")
        ek, ev = lexsorted(keys, vals)
        assert (ok == ek).all() and (ov == ev).all(), (dt, keys[:3], vals[:3], cutoff)
    g = np.random.default_rng(3)
    for n in (500, 20000):
        keys = g.integers(0, 4, size=n).astype(np.uint32)
        vals = g.integers(0, 2, size=n).astype(np.uint32)
        ok, ov, _, _ = oracle.sort(keys, vals, seed=6, cutoff=cutoff, variant="appendix")
        ek, ev = lexsorted(keys, vals)
        assert (ok == ek).all() and (ov == ev).all()


def mono_buckets_at_the_root(A, piv):
    """For each root bucket (pivots as root_pivots_from_the_listing gives
    them): its size and whether its range holds a single pair."""
    out = []
    for b in range(len(piv)):
        lo = piv[b - 1] if b > 0 else None
        size = sum(1 for e in A if (lo is None or lo < e) and e <= piv[b])
        mono = piv[0] == (0, 0) if b == 0 else (piv[b - 1] < piv[b] and pred(piv[b]) == piv[b - 1])
        out.append((size, mono))
    return out


def test_monochromatic_buckets_are_copied():
    """Repeated pairs: at the root, the buckets with more than `cutoff`
    elements recurse (one trace record each, with their size) unless their
    range holds a single pair; the others leave no record."""
    checked_mono = 0
    for seed in range(12):
        g = np.random.default_rng(seed)
        n = 3000 + 500 * seed
        keys = g.integers(0, 6, size=n).astype(np.uint32)
        vals = g.integers(0, 3, size=n).astype(np.uint32)
        if seed % 3 == 0:
            keys[: n // 2], vals[: n // 2] = 0, 0  # many copies of the least pair
        if seed % 3 == 1:  # copies of the greatest pair, about one in the sample
            keys[: n // 40], vals[: n // 40] = TOP["u32"]
        cutoff = 8
        A = list(zip((int(k) for k in keys), (int(v) for v in vals)))
        piv = root_pivots_from_the_listing(A, seed)
        want = {}
        for b, (size, mono) in enumerate(mono_buckets_at_the_root(A, piv)):
            checked_mono += mono and size > cutoff
            if size > cutoff and not mono:
                want[b] = size
        _, _, trace, _ = oracle.sort(keys, vals, seed=seed, cutoff=cutoff, trace_cap=1 << 20, variant="appendix")
        got = {r["index"]: r["n"] for r in trace if r["depth"] == 1 and r["kind"] == 2}
        assert got == want, seed
    assert checked_mono >= 12


MUTANTS = {
    "strict_bounds": ("  if (c->variant) return !elem_less(c->dtype, &pv->p[idx], e); /* appendix: bucket i holds e <= pivot i */",
                      "  if (c->variant) return elem_less(c->dtype, e, &pv->p[idx]);"),
    "ceil_geometry": ("  const uint64_t m = sqo_isqrt_floor(n);", "  const uint64_t m = sqo_isqrt_ceil(n);"),
    "short_last_column": ("    last[i] = (i + 1 < m) ? (i + 1) * m : n;", "    last[i] = (i + 1) * m < n ? (i + 1) * m : n;"),
    "sample_after_sorts": ("  appendix_pivots(c, A, n, m, h, smp);\n", ""),
    "no_separation": ("    if (elem_equal(c->dtype, &smp[r], &smp[r + 1])) smp[r] = elem_pred(smp[r]);", "    ;"),
    "no_mono_copy": ("    if (mono)\n", "    if (0)\n"),
    "no_least_pair_copy": ("      mono = elem_equal(c->dtype, &smp[0], &least);", "      mono = 0; (void)least;"),
    "inf_flag_not_compared": ("  for (uint64_t r = 0; r + 1 < m; r++)\n    if (elem_equal(c->dtype, &smp[r], &smp[r + 1]))",
                              "  for (uint64_t r = 0; r + 2 < m; r++)\n    if (elem_equal(c->dtype, &smp[r], &smp[r + 1]))"),
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
            _, _, _, rs = oracle.sort(keys, vals, seed=seed, cutoff=8, root_skew=True, lib=lib, variant="appendix")
            got = list(zip((int(k) for k in rs[0]), (int(v) for v in rs[1])))
            if got != root_skew_from_the_listing(keys, vals, seed):
                return "root_skew"
        n = 100000
        _, _, trace, _ = oracle.sort(W.uniform_u32(n, 9), W.iota(n), seed=2, cutoff=40, trace_cap=1 << 20, lib=lib,
                                     variant="appendix")
        for r in trace:
            if r["m"] != math.isqrt(r["n"]):
                return "shape"
        for seed in range(6):  # repeated pairs: which root buckets recurse
            g = np.random.default_rng(seed)
            n = 3000
            keys = g.integers(0, 6, size=n).astype(np.uint32)
            vals = g.integers(0, 3, size=n).astype(np.uint32)
            if seed % 2:
                keys[: n // 40], vals[: n // 40] = TOP["u32"]
            A = list(zip((int(k) for k in keys), (int(v) for v in vals)))
            piv = root_pivots_from_the_listing(A, seed)
            want = {b: size for b, (size, mono) in enumerate(mono_buckets_at_the_root(A, piv))
                    if size > 8 and not mono}
            _, _, trace, _ = oracle.sort(keys, vals, seed=seed, cutoff=8, trace_cap=1 << 20, lib=lib,
                                         variant="appendix")
            if {r["index"]: r["n"] for r in trace if r["depth"] == 1 and r["kind"] == 2} != want:
                return "mono"
        ok, ov, _, _ = oracle.sort(np.zeros(300, dtype=np.uint32), np.zeros(300, dtype=np.uint32), seed=1,
                                   cutoff=16, lib=lib, variant="appendix")  # the least pair only
        if ok.any() or ov.any():
            return "least pair"
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

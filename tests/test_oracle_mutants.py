"""Planted mistakes: each plausible slip in the oracle must fail some pin.

Every case copies the oracle's C source, plants one mistake by a textual edit
(on the CPU, in a temporary directory), builds it, and runs a compact battery
of the pins from the other oracle tests against the broken copy.  The pristine
oracle must pass the battery; every mutant must fail at least one check.
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

SRC = os.path.join(os.path.dirname(oracle.__file__), "squaresort_oracle.c")

MUTANTS = {
    # Algorithm 3's comparison taken literally (<=) against the [p_j, p_{j+1}) buckets
    "bucket_bound_le": ("  return elem_less(c->dtype, e, &pv->p[idx]);",
                        "  return !elem_less(c->dtype, &pv->p[idx], e);"),
    # Algorithm 2's call order broken: (C2,B1) before (C1,B1)
    "skew_call_order": (
        "  skew_transpose(c, A, D, l2, col, colEnd, k2, pv, piv0, buc, threshold);\n"
        "  skew_transpose(c, A, D, l - l2, col + l2, colEnd + l2, k2, pv, piv0, buc, threshold);",
        "  skew_transpose(c, A, D, l - l2, col + l2, colEnd + l2, k2, pv, piv0, buc, threshold);\n"
        "  skew_transpose(c, A, D, l2, col, colEnd, k2, pv, piv0, buc, threshold);"),
    # min(D) allowed as a pivot
    "no_min_check": ("    int ok = !elem_equal(c->dtype, &piv[0], mn);", "    int ok = 1;"),
    # repeated pivots allowed
    "no_duplicate_check": ("      if (elem_equal(c->dtype, &piv[r], &piv[r + 1])) ok = 0;", "      ;"),
    # negative floats not reversed
    "f32_sign": ("    if (b & 0x80000000u) return (uint32_t)~b;", "    if (b & 0x80000000u) return b & 0x7fffffffu;"),
    # NaNs placed by payload instead of tied
    "f32_nan_payload": ("return 0xffffffffu; /* NaN: above +inf */", "return b | 0x80000000u;"),
    # ceil(sqrt) off by one on perfect squares
    "isqrt": ("    if (mid * mid >= n) hi = mid;", "    if (mid * mid > n) hi = mid;"),
    # pivots sampled from A (before the column sorts) instead of D
    "sample_from_A": ("  uint32_t attempts = select_pivots(c, D, n, m, col, colEnd, h, piv);",
                      "  uint32_t attempts = select_pivots(c, A, n, m, col, colEnd, h, piv);"),
    # bucket children keyed like column children
    "bucket_hash": ("sqo_child_hash(h, 2, j), depth + 1, 2, (uint32_t)j);",
                    "sqo_child_hash(h, 1, j), depth + 1, 2, (uint32_t)j);"),
    # first pivot-draw attempt re-used for every attempt
    "attempt_stream": ("  uint64_t s = sqo_fmix64(h ^ (0xd1b54a32d192ed03ull * (attempt + 1)));",
                       "  uint64_t s = sqo_fmix64(h ^ 0xd1b54a32d192ed03ull);"),
}


def _build_variant(tmp, name, edit):
    text = open(SRC).read()
    if edit is not None:
        old, new = edit
        assert text.count(old) == 1, f"mutation anchor for {name} not unique"
        text = text.replace(old, new)
    src = os.path.join(tmp, f"{name}.c")
    lib = os.path.join(tmp, f"lib{name}.so")
    open(src, "w").write(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", lib, src], check=True)
    return oracle.load(lib)


def battery(lib):
    """Compact versions of the oracle pins; returns the names that failed."""
    failed = []

    def check(name, fn):
        try:
            if not fn():
                failed.append(name)
        except Exception:  # a crash or a failed status is a failure too
            failed.append(name)

    def sort_ok():
        for dtype, keys in [("u32", W.uniform_u32(3000, 1)), ("u32", W.small_alphabet_u32(2000, 2, 3)),
                            ("f32", W.normal_f32(2000, 3, 0.05, 0.05, 0.05))]:
            vals = np.random.default_rng(2).permutation(keys.size).astype(np.uint32)
            bits = keys.view(np.uint32) if dtype == "f32" else keys
            nan = np.isnan(keys) if dtype == "f32" else np.zeros(keys.size, bool)
            if dtype == "f32":
                value = np.where(nan, np.float32(0), keys).astype(np.float64)
                negz = np.where((keys == 0) & np.signbit(keys) & ~nan, 0, 1)
                ref = np.lexsort((vals, negz, value, nan))
            else:
                ref = np.lexsort((vals, keys))
            for cutoff in (2, 16, 100):
                ko, vo, _, _ = oracle.sort(keys, vals, seed=5, cutoff=cutoff, dtype=dtype, lib=lib)
                kb = ko.view(np.uint32) if dtype == "f32" else ko
                if not ((vo == vals[ref]).all() and (kb == bits[ref]).all()):
                    return False
        return True

    def skew_ok():
        from test_oracle_skew import brute_force, make_case

        seed = 0
        for rows in range(1, 9):
            for cols in range(1, 9):
                for k in (1, 3, 4, 5, 8):
                    seed += 1
                    case = make_case(rows, cols, rows * cols - (seed % rows), k, 3, seed)
                    if case is None:
                        continue
                    keys, vals, pk, pv = case
                    ek, ev, es = brute_force(keys, vals, rows, cols, pk, pv, k)
                    for mode in (0, 1):
                        ko, vo, bs = oracle.skew_transpose(keys, vals, rows, cols, pk, pv, k, mode=mode, lib=lib)
                        if not ((ko == ek).all() and (vo == ev).all() and (bs == es).all()):
                            return False
        return True

    def isqrt_ok():
        return all(oracle.isqrt_ceil(n, lib) == math.isqrt(n - 1) + 1 for n in range(1, 3000))

    def root_skew_ok():
        from test_oracle_sort import root_step_from_definitions

        for n in (50, 257, 1000):
            keys = W.distinct16_u32(n, n)
            vals = np.random.default_rng(n).permutation(n).astype(np.uint32)
            ek, ev, att = root_step_from_definitions(keys, vals, seed=n)
            _, _, tr, (sk, sv) = oracle.sort(keys, vals, seed=n, cutoff=8, trace_cap=10**5, root_skew=True, lib=lib)
            root = [r for r in tr if r["depth"] == 0]
            if not ((sk == ek).all() and (sv == ev).all() and root and root[0]["attempts"] == att):
                return False
        return True

    def invariants_ok():
        for n in (5, 17, 30, 100):
            m = oracle.isqrt_ceil(n, lib)
            rng = np.random.default_rng(n)
            for s in range(300):
                sizes, att = oracle.node_buckets(rng.permutation(n).astype(np.uint64),
                                                 oracle.root_hash(s, lib), lib=lib)
                if att < 1 or sizes.min() < 1 or int(sizes.sum()) != n or sizes.max() > n - m + 1:
                    return False
        return True

    def trace_hash_ok():
        keys = W.uniform_u32(5000, 4)
        _, _, tr, _ = oracle.sort(keys, W.iota(5000), seed=4, cutoff=16, trace_cap=10**5, lib=lib)

        def contains(p, r):
            return p["off"] <= r["off"] and r["off"] + r["n"] <= p["off"] + p["n"]

        for idx, r in enumerate(tr):
            if r["depth"] == 0:
                continue
            if r["kind"] == 1:
                p = next(q for q in tr[idx + 1:] if q["depth"] == r["depth"] - 1 and contains(q, r))
            else:
                p = next(q for q in reversed(tr[:idx]) if q["depth"] == r["depth"] - 1 and contains(q, r))
            if r["hash"] != oracle.child_hash(p["hash"], r["kind"], r["index"]):
                return False
        return True

    def attempts_ok():
        att = [oracle.node_buckets(np.random.default_rng(s).permutation(400).astype(np.uint64),
                                   oracle.root_hash(s, lib), lib=lib)[1] for s in range(400)]
        return 1.1 < np.mean(att) <= math.e ** 2

    check("sort", sort_ok)
    check("skew", skew_ok)
    check("isqrt", isqrt_ok)
    check("root_skew", root_skew_ok)
    check("invariants", invariants_ok)
    check("trace_hash", trace_hash_ok)
    check("attempts", attempts_ok)
    return failed


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="sqo_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_pristine_passes_battery(tmpdir_mod):
    assert battery(_build_variant(tmpdir_mod, "pristine", None)) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_battery(tmpdir_mod, name):
    failed = battery(_build_variant(tmpdir_mod, name, MUTANTS[name]))
    assert failed, f"planted mistake {name} passed every pin"

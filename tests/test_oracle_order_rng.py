"""Pins for the oracle's element order, random source and integer helpers.

Each check compares the oracle with something other than itself: numpy's
float ordering, Python's exact integers, math.isqrt, or the published
SplitMix64 output vector.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _expected_f32_order(x: np.ndarray, vals: np.ndarray) -> np.ndarray:
    """The float order the sort promises, stated with numpy: every NaN after
    +inf (NaNs tied), -0 before +0, otherwise numeric order; ties by val."""
    nan = np.isnan(x)
    value = np.where(nan, np.float32(0), x).astype(np.float64)
    neg_zero_first = np.where((x == 0) & np.signbit(x) & ~nan, 0, 1)
    return np.lexsort((vals, neg_zero_first, value, nan))


def _oracle_order(dtype, keys, vals):
    bits = keys.view(np.uint32) if dtype == "f32" else keys
    ords = np.array([oracle.ordinal(dtype, int(b)) for b in bits], dtype=np.uint64)
    return np.lexsort((vals, ords))


def test_f32_specials_order():
    x = W.special_f32()
    v = np.arange(x.size, dtype=np.uint32)[::-1].copy()
    assert (_oracle_order("f32", x, v) == _expected_f32_order(x, v)).all()


def test_f32_random_order_with_specials():
    x = W.normal_f32(4000, 11, p_inf=0.05, p_negzero=0.05, p_nan=0.05)
    x[::97] = np.float32(0.0)  # +0 too, so -0/+0 ties are exercised
    v = np.random.default_rng(3).permutation(x.size).astype(np.uint32)
    assert (_oracle_order("f32", x, v) == _expected_f32_order(x, v)).all()


def test_f32_nans_tie_by_val_only():
    nans = np.array([0x7FC00000, 0xFFC00000, 0x7F800001, 0xFFFFFFFF], dtype=np.uint32)
    for a in nans:
        for b in nans:
            assert oracle.less("f32", int(a), 1, int(b), 2)
            assert not oracle.less("f32", int(a), 2, int(b), 1)
    assert oracle.less("f32", 0x7F800000, 5, 0xFFC00000, 0)  # +inf < -NaN


def test_integer_ordinals_are_identity():
    for k in [0, 1, 2**31, 2**32 - 1]:
        assert oracle.ordinal("u32", k) == k
    for k in [0, 1, 2**63, 2**64 - 1]:
        assert oracle.ordinal("u64", k) == k
    assert oracle.less("u64", 2**63, 0, 2**63 + 1, 0)
    assert oracle.less("u32", 7, 1, 7, 2) and not oracle.less("u32", 7, 2, 7, 2)


def test_splitmix64_published_vector():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        expected = [int(line) for line in f if line.strip() and not line.startswith("#")]
    gamma, mask, state = 0x9E3779B97F4A7C15, 2**64 - 1, 1234567
    got = []
    for _ in expected:
        state = (state + gamma) & mask
        got.append(oracle.fmix64(state))
    assert got == expected


def test_scale_is_floor_of_product():
    rng = np.random.default_rng(5)
    cases = [(0, 1), (2**64 - 1, 1), (2**64 - 1, 2**32 - 1), (2**63, 3), (1, 2**64 - 1)]
    cases += [(int(rng.integers(0, 2**63)) * 2 + 1, int(rng.integers(1, 2**40))) for _ in range(500)]
    for u, n in cases:
        assert oracle.scale(u, n) == (u * n) >> 64


def test_isqrt_ceil_matches_math_isqrt():
    ns = list(range(1, 5000)) + [2**16, 2**16 + 1, 2**28, 2**28 - 1, 2**28 + 1, 2**32 - 1, 2**40 + 3]
    for n in ns:
        m = oracle.isqrt_ceil(n)
        assert m == math.isqrt(n - 1) + 1, n
        assert m * m >= n and (m - 1) * (m - 1) < n


def test_column_partition_of_17():
    # Algorithm 1 with n = 17: m = 5, columns [0,5) [5,10) [10,15) [15,17) [17,17).
    m = oracle.isqrt_ceil(17)
    sizes = [min((i + 1) * m, 17) - min(i * m, 17) for i in range(m)]
    assert m == 5 and sizes == [5, 5, 5, 2, 0]


def test_pivot_positions_uniform():
    # 64 buckets of positions over many draws: chi-square well inside 5 sigma.
    n, draws = 1024, 64000
    h = oracle.root_hash(99)
    pos = np.array([oracle.scale(oracle.pivot_draw(h, a, r), n) for a in range(64) for r in range(1000)])
    assert pos.min() >= 0 and pos.max() < n
    counts = np.bincount(pos * 64 // n, minlength=64)
    exp = draws / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)


def test_child_hashes_distinct():
    h = oracle.root_hash(1)
    cols = {oracle.child_hash(h, 1, i) for i in range(2000)}
    bucs = {oracle.child_hash(h, 2, i) for i in range(2000)}
    assert len(cols) == 2000 and len(bucs) == 2000 and not (cols & bucs)

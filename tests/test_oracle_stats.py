"""Statistical pins for the oracle's pivot step (Section 3).

* Pivot sampling succeeds with probability >= e^-2 per round, so the mean
  number of rounds is <= e^2 (Section 3.1, pivot paragraph).
* Bucket sizes: every bucket is non-empty and at most n - m + 1 (space
  bound); the sizes sum to n; upper tail P[n_1 >= t sqrt n] <= e^(-0.9t+0.1)
  and lower tail P[n_1 <= s] <= e^2 s / sqrt n for n >= 100 (Propositions
  on the bucket-size distribution); E[sum n_i log n_i] <= n log n / 2 + 4 e n
  (the Lemma that follows them).
"""
import math

import numpy as np
import pytest

import oracle


def _runs(n, count, seed0):
    out = []
    rng = np.random.default_rng(seed0)
    for s in range(count):
        keys = rng.permutation(n).astype(np.uint64)
        sizes, att = oracle.node_buckets(keys, oracle.root_hash(seed0 * 100000 + s))
        assert att >= 1
        out.append((sizes, att))
    return out


@pytest.mark.parametrize("n", [5, 17, 100, 1000, 4096])
def test_bucket_invariants(n):
    m = oracle.isqrt_ceil(n)
    for sizes, att in _runs(n, 300, n):
        assert sizes.size == m and int(sizes.sum()) == n
        assert sizes.min() >= 1 and sizes.max() <= n - m + 1
        assert 1 <= att <= oracle.MAX_ATTEMPTS


def test_mean_attempts_below_e_squared():
    for n in (10, 100, 2000):
        att = np.array([a for _, a in _runs(n, 2000, 7 + n)])
        assert att.mean() <= math.e ** 2
        # with m - 1 ~ sqrt(n) draws the birthday bound puts success near
        # e^(-1/2) for large n: the mean is well above 1 too (redraws happen).
        assert att.mean() > 1.1


def test_upper_tail_of_bucket_sizes():
    n = 400
    sizes = np.array([s[0] for s, _ in _runs(n, 6000, 3)], dtype=np.float64)  # n_1 of each node
    for t in (1, 2, 3, 4, 6):
        freq = (sizes >= t * math.sqrt(n)).mean()
        bound = math.exp(-0.9 * t + 0.1)
        assert freq <= bound + 4 * math.sqrt(bound * (1 - min(bound, 1)) / sizes.size) + 1e-3, (t, freq, bound)


def test_lower_tail_of_first_bucket():
    n = 2500
    first = np.array([s[0] for s, _ in _runs(n, 4000, 4)], dtype=np.float64)
    for s in (2, 5, 10):
        freq = (first <= s).mean()
        bound = math.e ** 2 * s / math.sqrt(n)
        assert freq <= bound


def test_expected_sum_n_log_n():
    n = 3000
    vals = []
    for sizes, _ in _runs(n, 300, 5):
        s = sizes.astype(np.float64)
        vals.append(float((s * np.log2(s)).sum()))
    assert np.mean(vals) <= 0.5 * n * math.log2(n) + 4 * math.e * n

"""Seeded synthetic inputs for SquareSort.

This module only draws inputs; it holds none of the sorting method's
arithmetic (no key ordinals, no pivot draws).  Both the CPU oracle tests and
the CUDA tests / benchmark take their inputs from here, so the two sides see
the same bytes.  Every generator is a pure function of its arguments; numpy's
PCG64 is the source of randomness.

Workloads (the paper sorts synthetic integer arrays, Section 4, so nothing
here stands in for a missing dataset):
  * ``uniform_u32``  -- i.i.d. uniform keys over [0, 2^32);
  * ``sorted_u32`` / ``reverse_u32`` -- that uniform draw ascending / descending;
  * ``distinct16_u32`` -- 16 values drawn uniformly, each key picks one;
  * ``zipf_u64``     -- Zipf(s) ranks over [1, 2^40] by rejection-inversion
    (Hoermann & Derflinger 1996), mapped through a seeded random bijection of
    64-bit words;
  * ``normal_f32``   -- N(0,1) rounded to float32 with 0.1% +-inf, 0.1% -0.0
    and 0.01% NaN of random sign and payload;
  * ``batch_sizes`` / ``serve_requests`` -- log-uniform instance sizes and a
    Poisson request stream.
The payload is always ``iota`` (the original index).
"""
from __future__ import annotations

import math

import numpy as np

M64 = (1 << 64) - 1


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed & M64, stream]))


def iota(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.uint32)


# ---------------------------------------------------------------- uint32 ----

def uniform_u32(n: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(0, 1 << 32, size=n, dtype=np.uint32)


def sorted_u32(n: int, seed: int) -> np.ndarray:
    return np.sort(uniform_u32(n, seed))


def reverse_u32(n: int, seed: int) -> np.ndarray:
    return np.ascontiguousarray(sorted_u32(n, seed)[::-1])


def distinct16_u32(n: int, seed: int) -> np.ndarray:
    g = _rng(seed)
    values = g.integers(0, 1 << 32, size=16, dtype=np.uint32)
    return values[g.integers(0, 16, size=n)]


def small_alphabet_u32(n: int, seed: int, alphabet: int) -> np.ndarray:
    """Keys from {0..alphabet-1}: many ties, resolved by the payload."""
    return _rng(seed).integers(0, alphabet, size=n, dtype=np.uint32)


U32_DISTRIBUTIONS = {
    "uniform": uniform_u32,
    "sorted": sorted_u32,
    "reverse": reverse_u32,
    "distinct16": distinct16_u32,
}


# ---------------------------------------------------------------- uint64 ----

def _zipf_ranks(n: int, s: float, N: int, g: np.random.Generator) -> np.ndarray:
    """Zipf(s) on {1..N} by rejection-inversion (Hoermann & Derflinger, "Rejection-
    inversion to generate variates from monotone discrete distributions", 1996).

    With h(x) = x^-s and H its antiderivative (x^(1-s)-1)/(1-s), a point is
    drawn uniformly from the area under h between 1/2 and N+1/2 by inverting
    H, rounded to the nearest integer k, and accepted when it falls under the
    step function of P(k) (or inside the always-accepted squeeze region).
    """
    one_minus_s = 1.0 - s

    def H(x):
        return np.expm1(one_minus_s * np.log(x)) / one_minus_s

    def H_inv(y):
        return np.exp(np.log1p(y * one_minus_s) / one_minus_s)

    def h(x):
        return np.exp(-s * np.log(x))

    h_x1 = float(H(np.float64(1.5))) - 1.0
    h_n = float(H(np.float64(N + 0.5)))
    squeeze = 2.0 - float(H_inv(H(np.float64(2.5)) - h(np.float64(2.0))))
    out = np.empty(n, dtype=np.uint64)
    todo = np.arange(n)
    while todo.size:
        u = h_n + g.random(todo.size) * (h_x1 - h_n)
        x = H_inv(u)
        k = np.clip(np.floor(x + 0.5), 1, N)
        ok = (k - x <= squeeze) | (u >= H(k + 0.5) - h(k))
        out[todo[ok]] = k[ok].astype(np.uint64)
        todo = todo[~ok]
    return out


def _bijection64(x: np.ndarray, g: np.random.Generator) -> np.ndarray:
    """A seeded bijection of 64-bit words: odd multiply, xor, xor-shift, odd multiply."""
    a = np.uint64(int(g.integers(0, 1 << 63)) * 2 + 1)
    b = np.uint64(int(g.integers(0, 1 << 63)) * 2)
    c = np.uint64(int(g.integers(0, 1 << 63)) * 2 + 1)
    with np.errstate(over="ignore"):
        y = (x * a) ^ b
        y = y ^ (y >> np.uint64(29))
        y = y * c
        y = y ^ (y >> np.uint64(32))
    return y


def zipf_u64(n: int, seed: int, s: float = 1.1, ranks: int = 1 << 40) -> np.ndarray:
    g = _rng(seed)
    return _bijection64(_zipf_ranks(n, s, ranks, g), _rng(seed, 1))


def uniform_u64(n: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(0, 1 << 64, size=n, dtype=np.uint64, endpoint=False)


# --------------------------------------------------------------- float32 ----

def normal_f32(n: int, seed: int, p_inf: float = 1e-3, p_negzero: float = 1e-3,
               p_nan: float = 1e-4) -> np.ndarray:
    g = _rng(seed)
    x = g.standard_normal(n).astype(np.float32)
    bits = x.view(np.uint32)
    kind = g.random(n)
    inf = kind < p_inf
    negz = (kind >= p_inf) & (kind < p_inf + p_negzero)
    nan = (kind >= p_inf + p_negzero) & (kind < p_inf + p_negzero + p_nan)
    sign = g.integers(0, 2, size=n, dtype=np.uint32) << np.uint32(31)
    bits[inf] = np.uint32(0x7F800000) | sign[inf]
    bits[negz] = np.uint32(0x80000000)
    payload = g.integers(1, 1 << 23, size=n, dtype=np.uint32)
    bits[nan] = np.uint32(0x7F800000) | payload[nan] | sign[nan]
    return x


def special_f32() -> np.ndarray:
    """Every float32 class: +-0, +-inf, NaNs of both signs, subnormals, extremes."""
    vals = [0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00000,
            0x7F800001, 0xFFFFFFFF, 0x7FFFFFFF, 0x00000001, 0x80000001, 0x007FFFFF,
            0x807FFFFF, 0x00800000, 0x80800000, 0x7F7FFFFF, 0xFF7FFFFF, 0x3F800000,
            0xBF800000, 0x3F800001, 0xBF800001]
    return np.array(vals, dtype=np.uint32).view(np.float32)


# ------------------------------------------------------ batches & serving ----

def batch_sizes(count: int, seed: int, lo_log2: int = 8, hi_log2: int = 20) -> np.ndarray:
    u = _rng(seed).random(count)
    n = np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
    return np.clip(n, 1 << lo_log2, 1 << hi_log2)


def batch_u32(count: int, seed: int, lo_log2: int = 8, hi_log2: int = 20):
    """Independent instances of log-uniform size with uniform uint32 keys."""
    sizes = batch_sizes(count, seed, lo_log2, hi_log2)
    return [uniform_u32(int(s), (seed << 20) + i + 1) for i, s in enumerate(sizes)]


def keys_for(dtype: str, n: int, seed: int) -> np.ndarray:
    """The per-dtype request generator of the serving workload."""
    if dtype == "u32":
        return uniform_u32(n, seed)
    if dtype == "u64":
        return zipf_u64(n, seed)
    if dtype == "f32":
        return normal_f32(n, seed)
    raise ValueError(dtype)


def serve_requests(count: int, seed: int, rate_per_s: float, lo_log2: int = 10, hi_log2: int = 24):
    """A Poisson request stream: (arrival_s, n, dtype, key_seed) per request."""
    g = _rng(seed)
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps)
    u = g.random(count)
    sizes = np.clip(np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64),
                    1 << lo_log2, 1 << hi_log2)
    dts = np.array(["u32", "u64", "f32"])[g.integers(0, 3, size=count)]
    return [(float(arrivals[i]), int(sizes[i]), str(dts[i]), (seed << 24) + i + 1) for i in range(count)]


def log_uniform_mean(lo_log2: int, hi_log2: int) -> float:
    """E[2^(lo + (hi-lo) U)] for U uniform on [0,1)."""
    span = (hi_log2 - lo_log2) * math.log(2)
    return (2.0 ** lo_log2) * (math.exp(span) - 1) / span

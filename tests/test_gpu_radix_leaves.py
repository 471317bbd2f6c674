"""GPU parity of the radix base case (leaves of 513..64K uint32 / float32
keys, one CTA or a cluster of 2-4 CTAs) against the plain definition of
the result: the input ordered by (ordinal(key), val).

Each case is one instance no larger than the cutoff, so the whole array is
a single leaf of the class under test.  The cases cover the class
boundaries, key ranges that end exactly on a digit boundary, equal keys
whose payloads do not ascend in input order (the radix order is then not
the (key, val) order and the kernel must fall back to its merge sort),
all-equal keys, float32 NaNs below and above the per-leaf NaN list, and
the presorted / reversed / rotated leaves that the kernel moves without
sorting.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = [513, 2048, 2049, 6000, 8192, 8193, 12000, 16384, 16385, 24576, 24577, 32768, 40000, 49152, 49153,
         65535, 65536]


@pytest.fixture(scope="module")
def sq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_14801_gb300 as sq

    sq.lib()
    return sq


def f32_ordinal(bits: np.ndarray) -> np.ndarray:
    b = bits.astype(np.uint64)
    nan = (b & 0x7FFFFFFF) > 0x7F800000
    return np.where(nan, 0xFFFFFFFF, np.where(b & 0x80000000, b ^ 0xFFFFFFFF, b | 0x80000000))


def expected(keys: np.ndarray, vals: np.ndarray, dtype: str):
    bits = keys.view(np.uint32)
    ords = f32_ordinal(bits) if dtype == "f32" else bits
    o = np.lexsort((vals, ords))
    return bits[o], vals[o]


def run_leaf(sq, keys: np.ndarray, vals: np.ndarray, dtype: str):
    view = np.float32 if dtype == "f32" else np.int32
    dk = torch.from_numpy(keys.view(view).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    sq.sort(dk, dv, seed=3, dtype=dtype, cutoff=max(keys.size, 2))
    torch.cuda.synchronize()
    return dk.cpu().numpy().view(np.uint32), dv.cpu().numpy().view(np.uint32)


def case(kind: str, n: int, seed: int):
    g = np.random.default_rng(seed)
    iota = W.iota(n)
    if kind == "uniform":
        return W.uniform_u32(n, seed), iota, "u32"
    if kind == "range_2^20":  # max - min = 2^20 - 1: exactly four 5-bit digits
        k = g.integers(0, 1 << 20, size=n, dtype=np.uint64).astype(np.uint32) + np.uint32(77)
        k[0], k[1] = 77, 77 + (1 << 20) - 1
        return k, iota, "u32"
    if kind == "range_2^20+1":  # one more bit: a fifth pass
        k = g.integers(0, (1 << 20) + 1, size=n, dtype=np.uint64).astype(np.uint32)
        k[5], k[6] = 0, 1 << 20
        return k, iota, "u32"
    if kind == "alphabet_iota":  # many ties, payloads ascending: the radix order holds
        return W.small_alphabet_u32(n, seed, 5), iota, "u32"
    if kind == "alphabet_perm":  # ties with shuffled payloads: the merge fallback
        return W.small_alphabet_u32(n, seed, 5), g.permutation(n).astype(np.uint32), "u32"
    if kind == "one_key_perm":  # every key equal, payloads shuffled
        return np.full(n, 12345, dtype=np.uint32), g.permutation(n).astype(np.uint32), "u32"
    if kind == "extremes":  # 0 and 2^32-1 both present: a 32-bit range
        k = W.uniform_u32(n, seed)
        k[3], k[n - 2] = 0, 0xFFFFFFFF
        return k, iota, "u32"
    if kind == "sorted":
        return np.sort(W.uniform_u32(n, seed)), iota, "u32"
    if kind == "reversed":
        return np.ascontiguousarray(np.sort(W.uniform_u32(n, seed))[::-1]), iota, "u32"
    if kind == "rotated":
        return np.roll(np.sort(W.uniform_u32(n, seed)), n // 3), iota, "u32"
    if kind == "reversed_ties":  # descending with ties, payloads ascending: runs of equal keys reversed
        return np.ascontiguousarray(np.sort(W.small_alphabet_u32(n, seed, n // 4 + 1))[::-1]), iota, "u32"
    if kind == "runs_descending":  # a few ascending runs, each entirely below the one before
        k = np.sort(W.uniform_u32(n, seed))
        cuts = np.sort(g.choice(np.arange(1, n), size=5, replace=False))
        parts = np.split(k, cuts)
        return np.concatenate(parts[::-1]), iota, "u32"
    if kind == "two_runs_ties":  # two ascending runs swapped, with ties across the seam
        k = np.sort(W.small_alphabet_u32(n, seed, 1000))
        r = n // 3
        return np.concatenate([k[r:], k[:r]]), iota, "u32"
    if kind == "f32_few_nans":
        x = W.normal_f32(n, seed, p_inf=0.01, p_negzero=0.01, p_nan=0.0)
        x[g.choice(n, 40, replace=False)] = np.float32("nan")
        x[::997] = np.float32(0.0)
        return x.view(np.uint32), g.permutation(n).astype(np.uint32), "f32"
    if kind == "f32_many_nans":
        x = W.normal_f32(n, seed, p_nan=0.01)
        return x.view(np.uint32), iota, "f32"
    raise ValueError(kind)


KINDS = ["uniform", "range_2^20", "range_2^20+1", "alphabet_iota", "alphabet_perm", "one_key_perm", "extremes",
         "sorted", "reversed", "rotated", "reversed_ties", "runs_descending", "two_runs_ties", "f32_few_nans",
         "f32_many_nans"]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", KINDS)
def test_radix_leaf_matches_definition(sq, kind, n):
    keys, vals, dtype = case(kind, n, seed=n % 1000 + len(kind))
    gk, gv = run_leaf(sq, keys, vals, dtype)
    ek, ev = expected(keys, vals, dtype)
    assert (gk == ek).all() and (gv == ev).all()


def test_radix_leaves_in_a_batch_of_mixed_classes(sq):
    """Many leaves of every radix class in the same launches (host-driven
    and persistent grids alike), each equal to its own definition."""
    g = np.random.default_rng(11)
    sizes = list(g.integers(513, 65537, size=60)) + SIZES
    items, refs = [], []
    for i, n in enumerate(sizes):
        n = int(n)
        kind = KINDS[i % 7]  # the integer kinds
        k, v, dtype = case(kind, n, seed=500 + i)
        refs.append(expected(k, v, dtype))
        items.append((torch.from_numpy(k.view(np.int32).copy()).cuda(),
                      torch.from_numpy(v.view(np.int32).copy()).cuda(), i))
    sq.set_cutoff("u32", 65536)
    try:
        sq.sort_batch(items)
        torch.cuda.synchronize()
    finally:
        sq.set_cutoff("u32", 0)
    for (dk, dv, _), (ek, ev) in zip(items, refs):
        assert (dk.cpu().numpy().view(np.uint32) == ek).all()
        assert (dv.cpu().numpy().view(np.uint32) == ev).all()


@pytest.mark.parametrize("n", [1 << 22, 1 << 24, 1 << 26])
def test_reversed_with_ties_through_the_recursion(sq, n):
    """A reversed uniform draw (ties among 2^32 values) at the default cutoff:
    reversed columns with ties, then buckets made of swapped or descending
    runs, in every leaf class."""
    keys = np.ascontiguousarray(np.sort(W.uniform_u32(n, 4))[::-1])
    dk = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    dv = torch.arange(n, dtype=torch.int32, device="cuda")
    sq.sort(dk, dv, seed=11, dtype="u32")
    torch.cuda.synchronize()
    gk = dk.cpu().numpy().view(np.uint32)
    gv = dv.cpu().numpy().view(np.uint32)
    ek, ev = expected(keys, W.iota(n), "u32")
    bad = np.nonzero((gk != ek) | (gv != ev))[0]
    assert bad.size == 0, (bad.size, bad[:5])

"""The oracle's random source restated in plain Python integers.

The pivot rule of Algorithm 1 (Section 2.1) draws m-1 positions at random and
redraws the whole sample when two drawn elements coincide or when its
smallest element is the minimum of D.  The paper leaves the random source
open; the oracle fixes it as counter-based SplitMix64 (Steele, Lea & Flood
2014) keyed by the node's path:

    F(z)            the SplitMix64 output function
    root            h = F(seed)
    column child i  F(h + gamma*(2i+1))
    bucket child j  F(h + gamma*(2j+2))
    attempt a       s_a = F(h xor C*(a+1)),  C = 0xd1b54a32d192ed03
    draw r          u = F(s_a + gamma*(r+1)),  position floor(u*n / 2^64)

(all arithmetic mod 2^64).  These checks state that definition again in
Python integers -- nothing here calls into the oracle's arithmetic except the
functions under test -- and compare, over thousands of inputs, the oracle's
root_hash, child_hash and pivot_draw with it, then follow the hashes and the
redraw count through the oracle's own recursion trace.  A slip in a
constant, an offset (2i+1, 2j+2, a+1, r+1) or the xor would fail here even
though the distributional pins elsewhere would still pass.
"""
import os

import numpy as np

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
ATTEMPT_MUL = 0xD1B54A32D192ED03


def F(z: int) -> int:
    """SplitMix64's output function (Steele, Lea & Flood 2014; the variant
    Vigna publishes as splitmix64.c): two xor-shift-multiply rounds and a
    final xor-shift."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def root(seed: int) -> int:
    return F(seed)


def column_child(h: int, i: int) -> int:
    return F(h + GAMMA * (2 * i + 1))


def bucket_child(h: int, j: int) -> int:
    return F(h + GAMMA * (2 * j + 2))


def draw(h: int, a: int, r: int) -> int:
    s = F(h ^ ((ATTEMPT_MUL * (a + 1)) & MASK))
    return F(s + GAMMA * (r + 1))


def position(u: int, n: int) -> int:
    return (u * n) >> 64


def _inputs(count: int, seed: int):
    g = np.random.default_rng(seed)
    edge = [0, 1, 2, 3, GAMMA, MASK, MASK - 1, 1 << 63, (1 << 63) - 1, ATTEMPT_MUL]
    rand = [int(x) for x in g.integers(0, 1 << 63, size=count, dtype=np.int64)]
    rand = [x * 2 + (i & 1) for i, x in enumerate(rand)]  # full 64-bit range
    return edge + rand


def test_restated_F_matches_published_vector():
    """The restatement's F reproduces SplitMix64's published outputs for seed
    1234567, so the comparisons below test the oracle against SplitMix64 itself."""
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        expected = [int(line) for line in f if line.strip() and not line.startswith("#")]
    state, got = 1234567, []
    for _ in expected:
        state = (state + GAMMA) & MASK
        got.append(F(state))
    assert got == expected


def test_root_hash_restated():
    for seed in _inputs(3000, 1):
        assert oracle.root_hash(seed) == root(seed), seed


def test_child_hashes_restated():
    g = np.random.default_rng(2)
    for h in _inputs(1500, 3):
        for i in [0, 1, 2, int(g.integers(0, 1 << 14)), int(g.integers(0, 1 << 32)), (1 << 32) - 1]:
            assert oracle.child_hash(h, 1, i) == column_child(h, i), (h, i)
            assert oracle.child_hash(h, 2, i) == bucket_child(h, i), (h, i)


def test_pivot_draws_restated():
    g = np.random.default_rng(4)
    for h in _inputs(1000, 5):
        for a in [0, 1, 2, int(g.integers(3, 256))]:
            for r in [0, 1, int(g.integers(2, 1 << 14)), (1 << 14) - 2]:
                assert oracle.pivot_draw(h, a, r) == draw(h, a, r), (h, a, r)


def test_positions_restated():
    g = np.random.default_rng(6)
    for h in _inputs(300, 7):
        for n in [1, 2, 17, 1000, int(g.integers(2, 1 << 28)), (1 << 40) + 3]:
            u = draw(h, 0, 5)
            assert oracle.scale(u, n) == position(u, n)


def _composite(keys: np.ndarray, vals: np.ndarray) -> np.ndarray:
    return (keys.astype(np.uint64) << np.uint64(32)) | vals.astype(np.uint64)


def _attempts_from_definition(a_keys, a_vals, h):
    """Algorithm 1's pivot step on one node, from the definitions: columns
    [i*m, (i+1)*m) sorted by (key, val), then samples a = 0, 1, ... of m-1
    positions drawn with the restated source; a sample is rejected if two
    drawn elements are equal (with distinct elements: equal positions) or if
    its smallest element equals the smallest column head.  Returns the number
    of samples drawn."""
    n = a_keys.size
    m = 1
    while m * m < n:
        m += 1
    e = _composite(a_keys, a_vals)
    D = np.concatenate([np.sort(e[min(i * m, n):min((i + 1) * m, n)]) for i in range(m)])
    dmin = min(D[min(i * m, n)] for i in range(m) if i * m < n)
    for a in range(256):
        pos = [position(draw(h, a, r), n) for r in range(m - 1)]
        if len(set(pos)) < len(pos):
            continue
        if min(D[p] for p in pos) == dmin:
            continue
        return a + 1
    return 0


def test_trace_hashes_and_attempts_follow_the_definition():
    """In the oracle's recursion trace, the root's hash is F(seed); every
    column or bucket child's hash is the restated formula applied to its
    parent's hash and its index; and the root's sample count is the one the
    restated draws give under the redraw rule.  Small nodes (m - 1 draws out
    of a few dozen positions) make redraws frequent, so the attempt stream
    is exercised, not just attempt 0."""
    redraws = 0
    for seed in range(150):
        n = 20 + (seed * 7) % 60
        keys = W.uniform_u32(n, 900 + seed)
        vals = W.iota(n)
        _, _, trace, _ = oracle.sort(keys, vals, seed=seed, cutoff=4, trace_cap=4096)
        roots = [r for r in trace if r["depth"] == 0]  # (records are written as pivots are chosen)
        assert len(roots) == 1
        rt = roots[0]
        assert rt["hash"] == root(seed)
        want = _attempts_from_definition(keys, vals, rt["hash"])
        assert rt["attempts"] == want, (seed, rt["attempts"], want)
        redraws += want > 1
        by_depth = {}
        for r in trace:
            by_depth.setdefault(r["depth"], []).append(r)
        for r in trace:
            if r["depth"] == 0:
                continue
            # a column node and a bucket node of the same parent share a range,
            # so the range alone does not name the parent: exactly one node one
            # level up must give this record's hash through the restated formula
            cands = [p for p in by_depth[r["depth"] - 1]
                     if p["off"] <= r["off"] and r["off"] + r["n"] <= p["off"] + p["n"]]
            child = column_child if r["kind"] == 1 else bucket_child
            assert r["kind"] in (1, 2)
            parents = [p for p in cands if child(p["hash"], r["index"]) == r["hash"]]
            assert len(parents) == 1, (seed, r)
            if r["kind"] == 1:
                p = parents[0]
                assert r["off"] == p["off"] + r["index"] * p["m"] and r["n"] <= p["m"]
    assert redraws >= 10  # the test reached attempts beyond the first

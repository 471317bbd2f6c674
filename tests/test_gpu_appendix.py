"""GPU parity of the appendix variant (the code the paper prints in its
appendix; Section 2.1 notes it departs slightly from Algorithm 1) against
the oracle's appendix mode, through the C ABI.

Sorted output must be bit-exact, and the recursion trace (every node's
offset, size, m = floor(sqrt n), path hash, one pivot sample) must equal the
oracle's: the trace pins the sample drawn from the node's input before its
columns are sorted, the duplicate separation, the (p_{i-1}, p_i] buckets and
the extended last column.  Small cutoffs make columns recurse, which is the
case where the engine keeps the samples in its sample store.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_14801_gb300 as sq

    sq.lib()
    return sq


VIEW = {"u32": (np.int32, np.uint32), "u64": (np.int64, np.uint64)}


def trace_key(r):
    return (r["off"], r["depth"], r["kind"], r["index"])


def gpu_sort(sq, keys, vals, dtype, seed, cutoff, trace=True):
    dk = torch.from_numpy(keys.view(VIEW[dtype][0]).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda() if vals is not None else None
    tr = sq.sort(dk, dv, seed=seed, dtype=dtype, cutoff=cutoff, trace_cap=(1 << 20) if trace else 0,
                 variant="appendix")
    torch.cuda.synchronize()
    gk = dk.cpu().numpy().view(VIEW[dtype][1])
    gv = dv.cpu().numpy().view(np.uint32) if dv is not None else None
    return gk, gv, tr


def check(sq, keys, vals, dtype, seed, cutoff):
    gk, gv, gtr = gpu_sort(sq, keys, vals, dtype, seed, cutoff)
    ov_in = vals if vals is not None else W.iota(keys.size)
    ok, ov, otr, _ = oracle.sort(keys, ov_in, seed=seed, cutoff=cutoff, dtype=dtype, trace_cap=1 << 20,
                                 variant="appendix")
    assert (gk == ok).all(), "keys differ"
    if vals is not None:
        assert (gv == ov).all(), "payloads differ"
    assert sorted(gtr, key=trace_key) == sorted(otr, key=trace_key), "recursion trace differs"
    return len(otr)


SIZES = [1, 2, 3, 4, 8, 9, 15, 16, 17, 63, 64, 65, 100, 511, 513, 1000, 2048, 2049, 5000, 8192, 8193, 16385,
         32769, 50000, 65536, 65537, 200003, 1000003]


@pytest.mark.parametrize("cutoff", [8, 9, 16, 64, 512, 8192, 65536])
def test_u32_uniform_all_sizes(sq, cutoff):
    nodes = 0
    for n in SIZES:
        if (cutoff <= 9 and n > 50000) or (cutoff <= 64 and n > 200003):
            continue
        perm = np.random.default_rng(n).permutation(n).astype(np.uint32)
        nodes += check(sq, W.uniform_u32(n, 300 + n), perm, "u32", seed=n + cutoff, cutoff=cutoff)
    assert nodes > 0


def distribution(name, n, seed):
    g = np.random.default_rng(seed)
    if name == "alphabet":  # few keys: ties decided by the payload, duplicate samples separated
        return W.small_alphabet_u32(n, seed, 7), g.permutation(n).astype(np.uint32)
    if name == "one_key":
        return np.full(n, 99, dtype=np.uint32), g.permutation(n).astype(np.uint32)
    if name == "sorted":
        return W.sorted_u32(n, seed), W.iota(n)
    if name == "reverse":
        return W.reverse_u32(n, seed), W.iota(n)
    if name == "extremes":  # 0 and 2^32-1 with payloads 0 and 2^32-1: the predecessor at both ends
        k = np.where(g.random(n) < 0.5, 0, 0xFFFFFFFF).astype(np.uint32)
        v = g.permutation(n).astype(np.uint32)
        v[g.choice(n, 2, replace=False)] = [0, 0xFFFFFFFF]
        return k, v
    raise ValueError(name)


@pytest.mark.parametrize("name", ["alphabet", "one_key", "sorted", "reverse", "extremes"])
@pytest.mark.parametrize("cutoff", [8, 16, 700, 65536])
def test_u32_distributions(sq, name, cutoff):
    for n in [1000, 65536, 300001, 2000000]:
        if (cutoff == 8 and n > 65536) or (cutoff == 16 and n > 300001):
            continue
        keys, vals = distribution(name, n, 11 + n)
        check(sq, keys, vals, "u32", seed=5, cutoff=cutoff)


@pytest.mark.parametrize("cutoff", [8, 64, 8192])
def test_u64_keys(sq, cutoff):
    for n in [17, 5000, 100000, 1000003]:
        if cutoff == 8 and n > 100000:
            continue
        check(sq, W.zipf_u64(n, n), W.iota(n), "u64", seed=7, cutoff=cutoff)
        check(sq, W.uniform_u64(n, n + 1), np.random.default_rng(n).permutation(n).astype(np.uint32), "u64",
              seed=8, cutoff=cutoff)


def test_null_payload_uses_the_position(sq):
    keys = W.small_alphabet_u32(100000, 3, 50)
    check(sq, keys, None, "u32", seed=2, cutoff=40)


def test_large_default_cutoff(sq):
    """2^24 uint32 keys at the default cutoff (columns and buckets are leaves
    of the radix classes) and 2^22 uint64 keys at a cutoff whose columns
    recurse."""
    n = 1 << 24
    check(sq, W.uniform_u32(n, 77), W.iota(n), "u32", seed=1, cutoff=65536)
    n = 1 << 22
    check(sq, W.uniform_u64(n, 78), W.iota(n), "u64", seed=2, cutoff=1024)


def test_graph_launch_mode(sq):
    """The same sorts with every round in one graph launch (asynchronous when
    no trace is taken)."""
    sq.set_launch_mode("graph")
    try:
        for n, cutoff in [(300001, 16), (1 << 22, 65536)]:
            keys, vals = W.uniform_u32(n, n), np.random.default_rng(1).permutation(n).astype(np.uint32)
            check(sq, keys, vals, "u32", seed=4, cutoff=cutoff)
            gk, gv, _ = gpu_sort(sq, keys, vals, "u32", 4, cutoff, trace=False)
            sq.sync()
            o = np.lexsort((vals, keys))
            assert (gk == keys[o]).all() and (gv == vals[o]).all()
    finally:
        sq.set_launch_mode("auto")


def test_refusals(sq):
    with pytest.raises(RuntimeError):
        sq.sort(torch.zeros(100, dtype=torch.float32, device="cuda"), None, cutoff=16, variant="appendix")
    with pytest.raises(RuntimeError):
        sq.sort(torch.zeros(100, dtype=torch.int32, device="cuda"), None, dtype="u32", cutoff=7,
                variant="appendix")
    with pytest.raises(ValueError):
        sq.sort(torch.zeros(100, dtype=torch.int32, device="cuda"), None, dtype="u32", variant="listing")


TOP = {"u32": (0xFFFFFFFF, 0xFFFFFFFF), "u64": (2**64 - 1, 0xFFFFFFFF)}


def repeated_pair_inputs(n):
    """Inputs whose (key, val) pairs repeat: buckets that hold one pair are
    copied, at the least pair, the greatest, and in between."""
    g = np.random.default_rng(n)
    for dt in ("u32", "u64"):
        kdt = np.uint32 if dt == "u32" else np.uint64
        for k, v in [(0, 0), TOP[dt], (5, 7)]:
            yield dt, np.full(n, k, dtype=kdt), np.full(n, v, dtype=np.uint32)
    keys = g.integers(0, 6, size=n).astype(np.uint32)
    vals = g.integers(0, 3, size=n).astype(np.uint32)
    yield "u32", keys, vals
    k2, v2 = keys.copy(), vals.copy()
    k2[: n // 40], v2[: n // 40] = TOP["u32"]  # a few copies of the greatest pair
    yield "u32", k2, v2
    k3, v3 = keys.copy(), vals.copy()
    k3[: n // 2], v3[: n // 2] = 0, 0  # half the input the least pair
    yield "u32", k3, v3
    yield "u64", W.zipf_u64(n, n).copy(), np.zeros(n, dtype=np.uint32)


@pytest.mark.parametrize("cutoff", [8, 16, 100, 65536])
def test_repeated_pairs_match_the_oracle(sq, cutoff):
    for n in [9, 1000, 65536, 1 << 20]:
        if cutoff <= 16 and n > 65536:
            continue
        for dt, keys, vals in repeated_pair_inputs(n):
            check(sq, keys, vals, dt, seed=n + cutoff, cutoff=cutoff)


def test_repeated_pairs_from_pinned_host_buffers(sq):
    """Host buffers: the first pass reads them and the last writes them in
    place, so a copied bucket goes to the host buffer too."""
    n = 1 << 20
    for dt, keys, vals in repeated_pair_inputs(n):
        view, back = VIEW[dt]
        hk = torch.from_numpy(keys.view(view).copy()).pin_memory()
        hv = torch.from_numpy(vals.view(np.int32).copy()).pin_memory()
        sq.sort(hk, hv, seed=3, dtype=dt, cutoff=256, variant="appendix")
        o = np.lexsort((vals, keys))
        assert (hk.numpy().view(back) == keys[o]).all() and (hv.numpy().view(np.uint32) == vals[o]).all(), dt


def test_repeated_pairs_in_graph_launch_mode(sq):
    sq.set_launch_mode("graph")
    try:
        for dt, keys, vals in repeated_pair_inputs(300001):
            check(sq, keys, vals, dt, seed=9, cutoff=64)
    finally:
        sq.set_launch_mode("auto")

"""GPU parity: the CUDA SquareSort against the CPU oracle, element by element,
through the C ABI (via the ctypes binding).

Sorted output must be bit-exact (keys, payloads); the recursion trace (every
node's offset, size, m, path hash and pivot-sample count) must equal the
oracle's, which pins the pivot draws, the column partition and the buckets.
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
    from paper_2407_14801_gb300 import build

    build.build()
    import paper_2407_14801_gb300 as sq

    return sq


TORCH_VIEW = {"u32": np.int32, "u64": np.int64, "f32": np.float32}


def to_dev(a, dtype):
    bits = a.view(TORCH_VIEW[dtype]) if dtype != "f32" else a
    return torch.from_numpy(np.ascontiguousarray(bits).copy()).to("cuda")


def from_dev(t, dtype):
    a = t.cpu().numpy()
    return a.view({"u32": np.uint32, "u64": np.uint64, "f32": np.float32}[dtype])


def gpu_sort(sq, keys, vals, dtype, seed, cutoff, trace=True):
    dk = to_dev(keys, dtype)
    dv = to_dev(vals, "u32") if vals is not None else None
    tr = sq.sort(dk, dv, seed=seed, dtype=dtype, cutoff=cutoff, trace_cap=(1 << 20) if trace else 0)
    torch.cuda.synchronize()
    return from_dev(dk, dtype), (from_dev(dv, "u32") if dv is not None else None), tr


def trace_key(r):
    return (r["off"], r["depth"], r["kind"], r["index"])


def check_against_oracle(sq, keys, vals, dtype, seed, cutoff):
    gk, gv, gtr = gpu_sort(sq, keys, vals, dtype, seed, cutoff)
    ok, ov, otr, _ = oracle.sort(keys, vals, seed=seed, cutoff=cutoff, dtype=dtype, trace_cap=1 << 20)
    bits = (lambda a: a.view(np.uint32)) if dtype == "f32" else (lambda a: a)
    assert (bits(gk) == bits(ok)).all(), "keys differ"
    if vals is not None:
        assert (gv == ov).all(), "payloads differ"
    assert sorted(gtr, key=trace_key) == sorted(otr, key=trace_key), "recursion trace differs"
    return len(otr)


SIZES = [1, 2, 3, 4, 16, 17, 63, 64, 65, 100, 511, 512, 513, 1000, 2048, 2049, 5000, 8192, 8193, 16384, 16385,
         24576, 24577, 32768, 32769, 40000, 45000, 50000, 57344, 57345, 65536, 65537, 200003, 1000003]


@pytest.mark.parametrize("cutoff", [2, 3, 16, 64, 512, 2048, 8192, 16384, 32768, 65536])
def test_u32_uniform_all_sizes(sq, cutoff):
    nodes = 0
    for n in SIZES:
        if (cutoff <= 3 and n > 40000) or (cutoff <= 64 and n > 200003):
            continue
        keys = W.uniform_u32(n, 100 + n)
        nodes += check_against_oracle(sq, keys, W.iota(n), "u32", seed=n, cutoff=cutoff)
    assert nodes > 0


@pytest.mark.parametrize("dist", ["sorted", "reverse", "distinct16"])
@pytest.mark.parametrize("cutoff", [16, 700, 16384, 65536])
def test_u32_distributions(sq, dist, cutoff):
    for n in [1000, 65536, 300001, 2000000]:
        if cutoff == 16 and n > 300001:
            continue
        keys = W.U32_DISTRIBUTIONS[dist](n, 7 + n)
        check_against_oracle(sq, keys, W.iota(n), "u32", seed=3, cutoff=cutoff)


@pytest.mark.parametrize("alphabet", [1, 2, 3])
def test_ties_with_permuted_payload(sq, alphabet):
    for n, cutoff in [(5000, 16), (70000, 300), (70000, 16384), (900000, 65536)]:
        keys = W.small_alphabet_u32(n, alphabet, alphabet)
        vals = np.random.default_rng(n).permutation(n).astype(np.uint32)
        check_against_oracle(sq, keys, vals, "u32", seed=alphabet, cutoff=cutoff)


def test_config1_workload(sq):
    """n = 2^16 (a 256 x 256 view), uniform keys from seed 1, index payload."""
    n = 1 << 16
    keys = W.uniform_u32(n, 1)
    for cutoff in (16, 255, 256, 1024, 16384, 65536):
        check_against_oracle(sq, keys, W.iota(n), "u32", seed=1, cutoff=cutoff)


@pytest.mark.parametrize("cutoff", [2, 16, 500, 8192, 16384, 32768, 65536])
def test_u64_zipf(sq, cutoff):
    for n in [3, 100, 4097, 50000, 150000, 1000000]:
        if cutoff <= 16 and n > 150000:
            continue
        if cutoff == 2 and n > 50000:
            continue
        check_against_oracle(sq, W.zipf_u64(n, n), W.iota(n), "u64", seed=5, cutoff=cutoff)
        check_against_oracle(sq, W.uniform_u64(n, n + 1), W.iota(n), "u64", seed=6, cutoff=cutoff)


@pytest.mark.parametrize("cutoff", [2, 16, 500, 8192, 16384, 32768, 65536])
def test_f32_specials(sq, cutoff):
    for n in [5, 700, 30000, 150000, 1000000]:
        if cutoff <= 16 and n > 150000:
            continue
        if cutoff == 2 and n > 30000:
            continue
        keys = W.normal_f32(n, n, p_inf=0.01, p_negzero=0.01, p_nan=0.01)
        keys[::37] = np.float32(0.0)
        check_against_oracle(sq, keys, W.iota(n), "f32", seed=9, cutoff=cutoff)
    check_against_oracle(sq, np.tile(W.special_f32(), 50), W.iota(21 * 50), "f32", seed=1, cutoff=16)


def test_null_payload(sq):
    n = 100000
    keys = W.distinct16_u32(n, 4)
    gk, _, _ = gpu_sort(sq, keys, None, "u32", 2, 1000, trace=False)
    ok, _, _, _ = oracle.sort(keys, None, seed=2, cutoff=1000)
    assert (gk == ok).all()


def test_host_buffers_are_staged(sq):
    """sq_sort on host memory (the end-to-end path): copies inside the call."""
    n = 123457
    keys = W.uniform_u32(n, 8)
    vals = W.iota(n)
    hk, hv = keys.copy(), vals.copy()
    sq.sort(hk, hv, seed=4, dtype="u32", cutoff=2000)
    ok, ov, _, _ = oracle.sort(keys, vals, seed=4, cutoff=2000)
    assert (hk == ok).all() and (hv == ov).all()


def test_repeated_pairs_report_attempts_exhausted(sq):
    """Equal (key, val) pairs make every pivot sample invalid; the bounded
    redraw loop gives up after 256 samples and the call reports it."""
    keys = np.full(100, 7, dtype=np.uint32)
    vals = np.zeros(100, dtype=np.uint32)
    dk, dv = to_dev(keys, "u32"), to_dev(vals, "u32")
    with pytest.raises(sq.SquareSortError) as e:
        sq.sort(dk, dv, seed=1, dtype="u32", cutoff=16)
    assert e.value.status == 7
    with pytest.raises(RuntimeError):
        oracle.sort(keys, vals, seed=1, cutoff=16)
    # the context is still usable
    check_against_oracle(sq, W.uniform_u32(1000, 1), W.iota(1000), "u32", seed=1, cutoff=16)


def test_empty_and_tiny(sq):
    for n in (0, 1, 2):
        keys = W.uniform_u32(n, 3)
        gk, gv, _ = gpu_sort(sq, keys, W.iota(n), "u32", 1, 2, trace=False)
        assert (gk == np.sort(keys)).all()


@pytest.mark.parametrize("n", [60, 500, 2000, 8000, 16000, 20000, 30000, 40000, 45000, 52000, 65536])
def test_f32_leaf_nan_bits_restored(sq, n):
    """Single-leaf float32 sorts with 0, 1, a few, exactly 64, 65 and many NaNs
    of random sign and payload: the leaf kernels hold float keys as one
    compare word and restore NaN bits afterwards (or hand the leaf to the
    exact fix-up sort), so every NaN must come back bit for bit."""
    rng = np.random.default_rng(n)
    for nan_count in (0, 1, 7, 64, 65, 300, n):
        if nan_count > n:
            continue
        keys = W.normal_f32(n, n + nan_count, p_inf=0.01, p_negzero=0.01, p_nan=0.0)
        where = rng.choice(n, size=nan_count, replace=False)
        bits = keys.view(np.uint32)
        payload = rng.integers(1, 1 << 23, size=nan_count, dtype=np.uint32)
        sign = rng.integers(0, 2, size=nan_count, dtype=np.uint32) << np.uint32(31)
        bits[where] = np.uint32(0x7F800000) | payload | sign
        vals = rng.permutation(n).astype(np.uint32)
        check_against_oracle(sq, keys, vals, "f32", seed=nan_count, cutoff=65536)
        if n > 2048:  # also as a recursion whose leaves carry a few NaNs each
            check_against_oracle(sq, keys, vals, "f32", seed=nan_count, cutoff=2048)


def _presorted_cases(n, rng):
    """Leaves the adaptive base case takes without sorting (sorted, strictly
    reversed, two sorted runs swapped) and near misses it must sort."""
    base = np.sort(rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32))
    iota = W.iota(n)
    yield "sorted", base.copy(), iota
    yield "reversed", base[::-1].copy(), iota
    yield "equal keys, payload ascending", np.full(n, 5, np.uint32), iota
    yield "equal keys, payload descending", np.full(n, 5, np.uint32), iota[::-1].copy()
    if n >= 2:
        for p in sorted({1, n // 3, n - 1}):
            yield f"rotated at {p}", np.roll(base, -p).copy(), np.roll(iota, -p).copy()
        # the two runs meet at an equal key: the payloads decide
        k = np.sort(rng.integers(0, 50, size=n, dtype=np.uint32))
        k[0] = k[-1] = 50
        k = np.sort(k)
        yield "rotated, equal key at the seam", np.roll(k, -(n // 2)).copy(), np.roll(iota, -(n // 2)).copy()
    if n >= 3:
        sw = base.copy()
        sw[[n // 2, n // 2 - 1]] = sw[[n // 2 - 1, n // 2]]
        yield "sorted but one swap", sw, iota
        rv = base[::-1].copy()
        rv[n // 2] = rv[n // 2 - 1]  # a tie breaks the strict descent: sorted the usual way
        yield "reversed with one tie", rv, iota
        two = np.concatenate([base[: n // 2][::-1], base[n // 2:]])
        yield "two descents at the seam", np.roll(two, 1).copy(), iota
        # ascending runs in descending order: moved run by run
        ties = np.sort(rng.integers(0, 16 * n, size=n, dtype=np.uint32))[::-1].copy()
        yield "reversed with ties", ties, iota  # about one step in 16 a tie: runs of one or two
        yield "reversed with many ties", np.sort(rng.integers(0, max(2, n // 8), size=n, dtype=np.uint32))[::-1].copy(), iota
        for parts in (3, 5, 33):
            if n >= parts:
                cuts = np.linspace(0, n, parts + 1).astype(int)
                runs = [base[cuts[j]:cuts[j + 1]] for j in range(parts)][::-1]
                yield f"{parts} sorted runs in descending order", np.concatenate(runs), iota
                shuffled = runs[1:] + runs[:1]  # the same runs, one out of order: sorted the usual way
                yield f"{parts} sorted runs out of order", np.concatenate(shuffled), iota
        bad = ties.copy()
        bad[[0, n - 1]] = bad[[n - 1, 0]]  # first and last swapped: the runs no longer descend
        yield "reversed with ties, ends swapped", bad, iota
    if n >= 16384:  # runs meeting exactly at the 8192-element parts of a cluster leaf
        runs = [base[j:j + 8192] for j in range(0, n - n % 8192, 8192)][::-1]
        yield "runs at the part boundaries", np.concatenate(runs + [base[n - n % 8192:]][:0]), W.iota(len(runs) * 8192)


@pytest.mark.parametrize("n", [2, 3, 40, 64, 400, 512, 2000, 2048, 8000, 8192, 16000, 24577, 40000, 57345, 65536])
def test_presorted_leaves(sq, n):
    """The leaf kernels detect sorted, reversed and rotated input and only
    move it; every other input is sorted.  Each case against the oracle, as
    one leaf (the whole input, sorted in place) and, for the larger sizes,
    as a recursion whose columns and buckets are leaves."""
    rng = np.random.default_rng(n)
    for name, keys, vals in _presorted_cases(n, rng):
        check_against_oracle(sq, keys, vals, "u32", seed=n, cutoff=65536)
        if n > 8192:
            check_against_oracle(sq, keys, vals, "u32", seed=n, cutoff=4096)


@pytest.mark.parametrize("n", [100, 3000, 20000, 65536])
def test_presorted_leaves_wide_keys(sq, n):
    """The same for uint64 keys and for float32 keys with NaNs (which sort
    last and keep their bits)."""
    rng = np.random.default_rng(n + 1)
    base = np.sort(rng.integers(0, 1 << 64, size=n, dtype=np.uint64))
    iota = W.iota(n)
    tied = np.sort(rng.integers(0, max(2, n // 4), size=n, dtype=np.uint64))[::-1].copy()
    for keys, vals in ((base, iota), (base[::-1].copy(), iota), (np.roll(base, -(n // 4)), np.roll(iota, -(n // 4))),
                       (tied, iota)):
        check_against_oracle(sq, keys.copy(), vals.copy(), "u64", seed=2, cutoff=65536)
    f = np.sort(W.normal_f32(n, n, p_inf=0.01, p_negzero=0.01, p_nan=0.0))
    bits = f.view(np.uint32)
    nn = max(1, n // 100)
    bits[-nn:] = np.uint32(0x7FC00000) | rng.integers(0, 1 << 22, size=nn, dtype=np.uint32)
    ft = np.sort(np.round(W.normal_f32(n, n + 2, p_inf=0.01, p_negzero=0.01, p_nan=0.0) * 4) / 4).astype(np.float32)
    ft.view(np.uint32)[-nn:] = np.uint32(0xFFC00000) | rng.integers(0, 1 << 22, size=nn, dtype=np.uint32)
    for keys, vals in ((f, iota), (f[::-1].copy(), iota[::-1].copy()), (np.roll(f, -(n // 3)), np.roll(iota, -(n // 3))),
                       (ft[::-1].copy(), iota)):
        check_against_oracle(sq, keys.copy(), vals.copy(), "f32", seed=3, cutoff=65536)
        if n > 8192:
            check_against_oracle(sq, keys.copy(), vals.copy(), "f32", seed=3, cutoff=2048)


@pytest.mark.parametrize("dtype", ["u32", "u64", "f32"])
def test_pinned_host_buffers_are_read_and_written_in_place(sq, dtype):
    """sq_sort on page-locked host buffers: the first pass reads them and the
    last pass writes them through the device mapping (no staging copies).
    A single leaf, one level, and deep recursions whose column nodes read the
    host input at every depth; sorted input (whose buckets are copied, not
    skipped); float32 leaves with more NaNs than a leaf restores (the exact
    fix-up sort then runs in the host buffer); no payload."""
    gen = {"u32": lambda n, s: W.uniform_u32(n, s), "u64": lambda n, s: W.zipf_u64(n, s),
           "f32": lambda n, s: W.normal_f32(n, s, p_inf=0.01, p_negzero=0.01, p_nan=0.02)}[dtype]
    view = {"u32": torch.int32, "u64": torch.int64, "f32": torch.float32}[dtype]
    cases = [(5000, 65536), (300000, 65536), (70000, 16), (5000, 3), (1 << 20, 4096)]
    if dtype == "u32":
        cases.append(("sorted", 65536))
    for n, cutoff in cases:
        if n == "sorted":
            keys = np.sort(W.uniform_u32(1 << 20, 5))
            n = keys.size
        else:
            keys = gen(n, n)
        vals = np.random.default_rng(n).permutation(n).astype(np.uint32)
        hk = torch.from_numpy(keys.view(TORCH_VIEW[dtype]) if dtype != "f32" else keys.copy()).pin_memory()
        hv = torch.from_numpy(vals.view(np.int32)).pin_memory()
        assert hk.dtype == view and hk.is_pinned() and hv.is_pinned()
        sq.sort(hk, hv, seed=n, dtype=dtype, cutoff=cutoff)
        ok, ov, _, _ = oracle.sort(keys, vals, seed=n, cutoff=cutoff, dtype=dtype)
        got = hk.numpy().view({"u32": np.uint32, "u64": np.uint64, "f32": np.uint32}[dtype])
        want = ok.view(np.uint32) if dtype == "f32" else ok
        assert (got == want).all(), (n, cutoff, "keys differ")
        assert (hv.numpy().view(np.uint32) == ov).all(), (n, cutoff, "payloads differ")
    # no payload
    keys = gen(100000, 3)
    hk = torch.from_numpy(keys.view(TORCH_VIEW[dtype]) if dtype != "f32" else keys.copy()).pin_memory()
    sq.sort(hk, None, seed=2, dtype=dtype, cutoff=1000)
    ok, _, _, _ = oracle.sort(keys, None, seed=2, cutoff=1000, dtype=dtype)
    got = hk.numpy().view({"u32": np.uint32, "u64": np.uint64, "f32": np.uint32}[dtype])
    assert (got == (ok.view(np.uint32) if dtype == "f32" else ok)).all()


@pytest.mark.parametrize("dtype", ["u64", "f32"])
def test_sorted_and_reversed_wide_keys_through_the_skew(sq, dtype):
    """Sorted and reversed uint64 / float32 input large enough that the
    SkewTranspose's diagonal tiles copy runs of one tag straight to their
    bucket (16-byte elements in the copy path), against the oracle."""
    n = 1 << 21
    if dtype == "u64":
        base = np.sort(W.zipf_u64(n, 9))
    else:
        base = np.sort(W.normal_f32(n, 9, p_inf=0.001, p_negzero=0.001, p_nan=0.0))
    for keys in (base, base[::-1].copy()):
        check_against_oracle(sq, keys.copy(), W.iota(n), dtype, seed=4, cutoff=16384)

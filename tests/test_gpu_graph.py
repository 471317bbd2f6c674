"""GPU parity of the CUDA-graph launch mode: all recursion rounds of a sort
run as one graph launch (a device-side loop) instead of one host round trip
per round.  Results, recursion traces and the number of rounds and nodes must
equal the host-driven mode's and the oracle's."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VIEW = {"u32": np.int32, "u64": np.int64, "f32": np.float32}
BACK = {"u32": np.uint32, "u64": np.uint64, "f32": np.float32}


@pytest.fixture(scope="module")
def sq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_14801_gb300 as sq

    sq.lib()
    yield sq
    sq.set_launch_mode("auto")


def run(sq, mode, keys, vals, dtype, seed, cutoff):
    sq.set_launch_mode(mode)
    dk = torch.from_numpy(np.ascontiguousarray(keys).view(VIEW[dtype]).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    before = sq.stats()
    tr = sq.sort(dk, dv, seed=seed, dtype=dtype, cutoff=cutoff, trace_cap=1 << 20)
    after = sq.stats()
    torch.cuda.synchronize()
    work = (after["rounds"] - before["rounds"], after["nodes"] - before["nodes"])
    return dk.cpu().numpy().view(BACK[dtype]), dv.cpu().numpy().view(np.uint32), tr, work


def key(r):
    return (r["off"], r["depth"], r["kind"], r["index"])


CASES = [
    ("u32", 1000003, 65536), ("u32", 1000003, 2048), ("u32", 200003, 64), ("u32", 40000, 2), ("u32", 40000, 3),
    ("u32", 65537, 16384), ("u32", 16385, 512), ("u32", 5000, 16), ("u32", 3, 2), ("u32", 1, 2),
    ("u64", 1000000, 8192), ("u64", 150000, 16), ("u64", 4097, 2),
    ("f32", 1000000, 32768), ("f32", 150000, 500), ("f32", 30000, 2),
]


@pytest.mark.parametrize("dtype,n,cutoff", CASES)
def test_graph_equals_host_and_oracle(sq, dtype, n, cutoff):
    if dtype == "u32":
        keys = W.uniform_u32(n, n + cutoff)
    elif dtype == "u64":
        keys = W.zipf_u64(n, n)
    else:
        keys = W.normal_f32(n, n, p_inf=0.01, p_negzero=0.01, p_nan=0.01)
    vals = W.iota(n)
    gk, gv, gtr, gwork = run(sq, "graph", keys, vals, dtype, 5, cutoff)
    hk, hv, htr, hwork = run(sq, "host", keys, vals, dtype, 5, cutoff)
    ok, ov, otr, _ = oracle.sort(keys, vals, seed=5, cutoff=cutoff, dtype=dtype, trace_cap=1 << 20)
    bits = (lambda a: a.view(np.uint32)) if dtype == "f32" else (lambda a: a)
    assert (bits(gk) == bits(ok)).all() and (gv == ov).all()
    assert (bits(hk) == bits(ok)).all() and (hv == ov).all()
    assert sorted(gtr, key=key) == sorted(otr, key=key) == sorted(htr, key=key)
    assert gwork == hwork  # the same rounds and nodes, whoever drives them
    assert gwork[1] == len(otr)


def test_graph_distributions_and_ties(sq):
    for dist in ("sorted", "reverse", "distinct16"):
        keys = W.U32_DISTRIBUTIONS[dist](300001, 9)
        gk, gv, gtr, _ = run(sq, "graph", keys, W.iota(keys.size), "u32", 3, 700)
        ok, ov, otr, _ = oracle.sort(keys, W.iota(keys.size), seed=3, cutoff=700, trace_cap=1 << 20)
        assert (gk == ok).all() and (gv == ov).all()
        assert sorted(gtr, key=key) == sorted(otr, key=key)
    keys = W.small_alphabet_u32(70000, 2, 2)
    vals = np.random.default_rng(1).permutation(70000).astype(np.uint32)
    gk, gv, _, _ = run(sq, "graph", keys, vals, "u32", 2, 300)
    ok, ov, _, _ = oracle.sort(keys, vals, seed=2, cutoff=300)
    assert (gk == ok).all() and (gv == ov).all()


def test_graph_reports_attempts_exhausted_and_recovers(sq):
    sq.set_launch_mode("graph")
    keys = torch.full((100,), 7, dtype=torch.int32, device="cuda")
    vals = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(sq.SquareSortError) as e:  # from the call, or from sq_sync (asynchronous sort)
        sq.sort(keys, vals, seed=1, dtype="u32", cutoff=16)
        sq.sync()
    assert e.value.status == 7
    k = W.uniform_u32(5000, 4)
    gk, gv, _, _ = run(sq, "graph", k, W.iota(5000), "u32", 1, 16)
    ok, ov, _, _ = oracle.sort(k, W.iota(5000), seed=1, cutoff=16)
    assert (gk == ok).all() and (gv == ov).all()


def test_graph_batch_equals_oracle(sq):
    sq.set_launch_mode("graph")
    sizes = W.batch_sizes(300, 11, 4, 18)
    srcs = [W.uniform_u32(int(n), 50 + i) for i, n in enumerate(sizes)]
    batch = [(torch.from_numpy(s.view(np.int32).copy()).cuda(), torch.arange(s.size, dtype=torch.int32).cuda(), i)
             for i, s in enumerate(srcs)]
    sq.set_cutoff("u32", 128)
    try:
        sq.sort_batch(batch)
    finally:
        sq.set_cutoff("u32", 0)
    for (bk, bv, i), s in zip(batch, srcs):
        ok, ov, _, _ = oracle.sort(s, W.iota(s.size), seed=i, cutoff=128)
        assert (bk.cpu().numpy().view(np.uint32) == ok).all()
        assert (bv.cpu().numpy().view(np.uint32) == ov).all()


def test_launch_mode_setting(sq):
    for m in ("host", "graph", "auto"):
        sq.set_launch_mode(m)
        assert sq.get_launch_mode() == m
    with pytest.raises(sq.SquareSortError):
        sq._check(sq.lib().sq_set_launch_mode(7))

"""GPU parity of the batched form (sq_sort_batch) and the served form
(sq_serve_*): every instance's result equals the oracle's, whether it runs
alone or mixed with others of other sizes and key types."""
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
    for dt in ("u32", "u64", "f32"):
        sq.set_cutoff(dt, 0)


def instance(i, dt, n):
    keys = W.keys_for(dt, n, 1000 + i)
    vals = np.random.default_rng(i).permutation(n).astype(np.uint32) if i % 3 == 0 else W.iota(n)
    return keys, vals


def expected(keys, vals, dt, seed, cutoff):
    ok, ov, _, _ = oracle.sort(keys, vals, seed=seed, cutoff=cutoff, dtype=dt)
    return ok, ov


def same(a, b, dt):
    if dt == "f32":
        return (a.view(np.uint32) == b.view(np.uint32)).all()
    return (a == b).all()


@pytest.mark.parametrize("cutoff", [64, 2048, 0])
def test_batch_matches_oracle_per_instance(sq, cutoff):
    rng = np.random.default_rng(cutoff)
    specs = []
    for i in range(120):
        dt = ["u32", "u64", "f32"][i % 3]
        n = int(2 ** rng.uniform(0, 17))
        specs.append((i, dt, n))
    specs.append((500, "u32", 0))
    specs.append((501, "u32", 1))
    for dt in ("u32", "u64", "f32"):
        sq.set_cutoff(dt, cutoff)
    items, host = [], []
    for i, dt, n in specs:
        k, v = instance(i, dt, n)
        dk = torch.from_numpy(k.view(VIEW[dt]).copy()).cuda()
        dv = torch.from_numpy(v.view(np.int32).copy()).cuda() if i % 5 else None
        items.append((dk, dv, i))
        host.append((k, v if i % 5 else None, dt))
    sq.sort_batch(items)
    torch.cuda.synchronize()
    for (dk, dv, seed), (k, v, dt) in zip(items, host):
        c = cutoff or sq.get_cutoff(dt)
        ek, ev = expected(k, v, dt, seed, c)
        assert same(dk.cpu().numpy().view(BACK[dt]), ek, dt)
        if dv is not None:
            assert (dv.cpu().numpy().view(np.uint32) == ev).all()


def test_batch_equals_single_sorts(sq):
    sq.set_cutoff("u32", 256)
    sizes = W.batch_sizes(64, 7, 8, 16)
    srcs = [W.uniform_u32(int(n), i + 1) for i, n in enumerate(sizes)]
    batch = [(torch.from_numpy(s.view(np.int32).copy()).cuda(), torch.arange(s.size, dtype=torch.int32).cuda(), i)
             for i, s in enumerate(srcs)]
    sq.sort_batch(batch)
    for (bk, bv, i), s in zip(batch, srcs):
        k = torch.from_numpy(s.view(np.int32).copy()).cuda()
        v = torch.arange(s.size, dtype=torch.int32).cuda()
        tr = sq.sort(k, v, seed=i, dtype="u32", trace_cap=1 << 16)
        assert torch.equal(k, bk) and torch.equal(v, bv)
        _, _, otr, _ = oracle.sort(s, W.iota(s.size), seed=i, cutoff=256, trace_cap=1 << 16)
        key = lambda r: (r["off"], r["depth"], r["kind"], r["index"])
        assert sorted(tr, key=key) == sorted(otr, key=key)


def serve_all(sq, reqs, budget=512 << 20, cutoff=300):
    srv = sq.Server(budget, cutoff=cutoff)
    try:
        tickets = [srv.submit(k, v, seed=s, dtype=dt) for (k, v, dt, s) in reqs]
        results = {}
        import time

        t0 = time.time()
        while len(results) < len(tickets):
            for t in tickets:
                if t not in results:
                    r = srv.poll(t)
                    if r is not None:
                        results[t] = r
            assert time.time() - t0 < 120, "server did not finish"
        return [results[t] for t in tickets]
    finally:
        srv.close()


def test_serve_mixed_requests_match_oracle(sq):
    rng = np.random.default_rng(3)
    reqs, refs = [], []
    for i in range(48):
        dt = ["u32", "u64", "f32"][i % 3]
        n = int(2 ** rng.uniform(4, 18))
        k, v = instance(i, dt, n)
        refs.append(expected(k, v, dt, i, 300) + (dt,))
        reqs.append((k.copy(), v.copy(), dt, i))
    res = serve_all(sq, reqs)
    for (st, lat), (k, v, dt, _), (ek, ev, _) in zip(res, reqs, refs):
        assert st == 0 and lat > 0
        assert same(k, ek, dt) and (v == ev).all()


def test_serve_alone_equals_in_mix(sq):
    k0, v0 = instance(7, "u64", 90001)
    alone = [(k0.copy(), v0.copy(), "u64", 5)]
    serve_all(sq, alone)
    mix = [(k0.copy(), v0.copy(), "u64", 5)]
    for i in range(20):
        dt = ["u32", "f32"][i % 2]
        k, v = instance(100 + i, dt, 5000 + 997 * i)
        mix.append((k, v, dt, i))
    serve_all(sq, mix)
    assert (alone[0][0] == mix[0][0]).all() and (alone[0][1] == mix[0][1]).all()
    ek, ev = expected(k0, v0, "u64", 5, 300)
    assert (alone[0][0] == ek).all() and (alone[0][1] == ev).all()


def test_serve_budget_and_errors(sq):
    srv = sq.Server(64 << 20)
    try:
        big = np.zeros(1 << 23, dtype=np.uint64)
        with pytest.raises(sq.SquareSortError) as e:
            srv.submit(big, np.zeros(big.size, dtype=np.uint32), dtype="u64")
        assert e.value.status == 3  # SQ_ERR_BUDGET
        with pytest.raises(sq.SquareSortError):
            srv.poll(12345)
    finally:
        srv.close()


def test_cutoff_table_applies_per_instance(sq):
    """A cutoff table picks each instance's cutoff by its size, in single
    sorts and inside one batch: the recursion (trace, node count) is the
    oracle's at that cutoff."""
    table = {9: 64, 11: 512, 13: 2048, 15: 16384}
    try:
        sq.set_cutoff("u32", 0)
        sq.set_cutoff_table("u32", table)
        sizes = [600, 1000, 3000, 4095, 9000, 12000, 40000, 65000, 520, 2100]
        srcs = [W.uniform_u32(n, 70 + i) for i, n in enumerate(sizes)]
        want_nodes = 0
        for i, s in enumerate(srcs):
            c = table[max(k for k in table if (1 << k) <= s.size)]
            assert sq.cutoff_for("u32", s.size) == c
            ok, ov, otr, _ = oracle.sort(s, W.iota(s.size), seed=i, cutoff=c, trace_cap=1 << 16)
            want_nodes += len(otr)
            k = torch.from_numpy(s.view(np.int32).copy()).cuda()
            v = torch.arange(s.size, dtype=torch.int32).cuda()
            tr = sq.sort(k, v, seed=i, dtype="u32", trace_cap=1 << 16)
            key = lambda r: (r["off"], r["depth"], r["kind"], r["index"])
            assert sorted(tr, key=key) == sorted(otr, key=key)
        batch = [(torch.from_numpy(s.view(np.int32).copy()).cuda(), torch.arange(s.size, dtype=torch.int32).cuda(), i)
                 for i, s in enumerate(srcs)]
        before = sq.stats()["nodes"]
        sq.sort_batch(batch)
        assert sq.stats()["nodes"] - before == want_nodes
        for (bk, bv, i), s in zip(batch, srcs):
            ok, ov, _, _ = oracle.sort(s, W.iota(s.size), seed=i, cutoff=64)
            assert same(bk.cpu().numpy().view(np.uint32), ok, "u32")
            assert (bv.cpu().numpy().view(np.uint32) == ov).all()
    finally:
        sq.set_cutoff_table("u32", [])
        sq.load_tuning()


def test_serve_admits_while_others_run(sq):
    """Continuous batching: a small request submitted while a large one of
    the same key type is being sorted joins the running engine at a round
    boundary and comes back before the large one; both results are exact."""
    big_k = W.uniform_u32(1 << 26, 41)
    small_k = W.uniform_u32(1 << 10, 42)
    reqs = [(big_k.copy(), W.iota(big_k.size), "u32", 1), (small_k.copy(), W.iota(small_k.size), "u32", 2)]
    srv = sq.Server(4 << 30)
    try:
        import time

        t_big = srv.submit(reqs[0][0], reqs[0][1], seed=1, dtype="u32")
        t_small = srv.submit(reqs[1][0], reqs[1][1], seed=2, dtype="u32")
        got, t0 = {}, time.time()
        while len(got) < 2:
            for t in (t_big, t_small):
                if t not in got:
                    r = srv.poll(t)
                    if r is not None:
                        got[t] = r
            assert time.time() - t0 < 120, "server did not finish"
    finally:
        srv.close()
    assert got[t_big][0] == 0 and got[t_small][0] == 0
    # submitted later, finished earlier: it did not wait for the large sort
    assert got[t_small][1] < got[t_big][1]
    assert (reqs[1][0] == np.sort(small_k)).all()
    assert (reqs[0][0] == np.sort(big_k)).all()
    assert (reqs[0][0] == big_k[reqs[0][1].view(np.uint32)]).all()

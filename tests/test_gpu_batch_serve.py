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


# ------------------------------------------------- the stated workload sizes --

def _segmented_unique_result(src, keys, vals, offs, dtype):
    """check_unique_result over many instances laid end to end: within every
    instance the output is non-decreasing by (ordinal(key), val), its payloads
    are a permutation of 0..n_i-1, and each key is the original key of its
    payload -- which together pin the unique sorted result of each."""
    from test_gpu_fullsize import ordinal64

    total = keys.numel()
    dev = keys.device
    sizes = offs[1:] - offs[:-1]
    inst = torch.repeat_interleave(torch.arange(sizes.numel(), device=dev), sizes)
    v = vals.to(torch.int64) & 0xFFFFFFFF
    o = ordinal64(keys, dtype)
    start = torch.zeros(total, dtype=torch.bool, device=dev)
    start[offs[:-1][sizes > 0]] = True
    ok = (o[1:] > o[:-1]) | ((o[1:] == o[:-1]) & (v[1:] > v[:-1])) | start[1:]
    assert bool(ok.all()), "an instance is not sorted by (key, val)"
    del ok, o
    assert bool((v < sizes[inst]).all()), "a payload is out of its instance's range"
    g = offs[:-1][inst] + v
    seen = torch.zeros(total, dtype=torch.bool, device=dev)
    seen[g] = True
    assert bool(seen.all()), "payloads are not a permutation within each instance"
    assert bool((src[g] == keys).all()), "a key left its payload"


def test_batch_config_4096_instances_2e8_to_2e20(sq):
    """The batched workload at its stated size: 4096 uint32 instances of
    sizes log-uniform in [2^8, 2^20] (size seed 7), uniform keys, index
    payload, all in one sq_sort_batch at the default cutoffs.  Every
    instance is checked on the device by the unique-result properties, and
    64 of them -- the largest among them -- element by element against the
    oracle."""
    count = 4096
    sizes = W.batch_sizes(count, 7)
    offs_np = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(offs_np[-1])
    flat = np.empty(total, dtype=np.uint32)
    for i in range(count):
        flat[offs_np[i]:offs_np[i + 1]] = W.uniform_u32(int(sizes[i]), (7 << 20) + i + 1)
    src = torch.from_numpy(flat.view(np.int32)).cuda()
    keys = src.clone()
    offs = torch.from_numpy(offs_np).cuda()
    inst = torch.repeat_interleave(torch.arange(count, device="cuda"), offs[1:] - offs[:-1])
    vals = (torch.arange(total, device="cuda") - offs[:-1][inst]).to(torch.int32)
    del inst
    seeds = [7 + i for i in range(count)]
    sq.sort_batch([(keys[offs_np[i]:offs_np[i + 1]], vals[offs_np[i]:offs_np[i + 1]], seeds[i])
                   for i in range(count)])
    torch.cuda.synchronize()
    _segmented_unique_result(src, keys, vals, offs, "u32")
    big = int(np.argmax(sizes))
    pick = [big] + [i for i in range(0, count, 64) if i != big][:63]
    assert len(pick) == 64
    gk = keys.cpu().numpy().view(np.uint32)
    gv = vals.cpu().numpy().view(np.uint32)
    for i in pick:
        a, b = offs_np[i], offs_np[i + 1]
        ek, ev, _, _ = oracle.sort(flat[a:b], W.iota(b - a), seed=seeds[i], cutoff=sq.cutoff_for("u32", b - a))
        assert (gk[a:b] == ek).all() and (gv[a:b] == ev).all(), i


def test_serve_config_sizes_2e10_to_2e24_all_key_types(sq):
    """The served workload's request mix: sizes log-uniform in [2^10, 2^24]
    and key types uniform over uint32 / uint64 / float32 with their
    workload generators (uniform, Zipf(1.1), N(0,1) with specials), drawn as
    the request stream draws them, plus one 2^24 request and one 2^10
    request of each key type, all in flight together under the 16 GB budget.
    Requests up to 2^18 keys are compared with the oracle element by
    element; larger ones by the unique-result properties on the device."""
    stream = W.serve_requests(36, 5, rate_per_s=1.0)
    specs = [(n, dt, s) for (_, n, dt, s) in stream]
    specs += [(1 << 24, dt, 900 + i) for i, dt in enumerate(("u64", "f32", "u32"))]
    specs += [(1 << 10, dt, 910 + i) for i, dt in enumerate(("u64", "f32", "u32"))]
    reqs = []
    for n, dt, s in specs:
        k = W.keys_for(dt, n, s)
        reqs.append((k, W.iota(n), dt, s))
    srcs = [r[0].copy() for r in reqs]
    res = serve_all(sq, reqs, budget=16 << 30, cutoff=0)
    n_oracle = n_props = 0
    for (st, lat), (k, v, dt, s), src in zip(res, reqs, srcs):
        assert st == 0 and lat > 0
        if k.size <= (1 << 18):
            ek, ev = expected(src, W.iota(k.size), dt, s, sq.cutoff_for(dt, k.size))
            assert same(k, ek, dt) and (v == ev).all(), (k.size, dt, s)
            n_oracle += 1
        else:
            from test_gpu_fullsize import check_unique_result

            tv = VIEW[dt]
            sb = torch.from_numpy(src.view(tv)).cuda()
            ob = torch.from_numpy(k.view(tv)).cuda()
            ov = torch.from_numpy(v.view(np.int32)).cuda()
            if dt == "f32":
                sb, ob = sb.view(torch.int32), ob.view(torch.int32)
            check_unique_result(sb, ob, ov, dt)
            n_props += 1
    assert n_oracle >= 10 and n_props >= 6
    assert {dt for (n, dt, _) in specs if n == 1 << 24} == {"u32", "u64", "f32"}

"""The asynchronous boundary: in the CUDA-graph launch mode, sq_sort on
device buffers (no trace) and sq_sort_batch enqueue the whole recursion and
return; errors found on the device are latched and returned by sq_sync or
by the next call on the same stream.  Results stay bit-exact."""
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
    sq.set_launch_mode("graph")
    yield sq
    sq.set_launch_mode("auto")


def unique_result(src, keys, vals):
    from test_gpu_fullsize import check_unique_result

    check_unique_result(src, keys, vals, "u32")


def test_sort_returns_before_the_gpu_finishes(sq):
    """A 2^26-key sort: the call comes back while its work is still queued or
    running on the stream (the stream reports unfinished work), and after
    sq_sync the result is the unique sorted one."""
    n = 1 << 26
    src = torch.from_numpy(W.uniform_u32(n, 61).view(np.int32)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    keys = src.clone()
    sq.sort(keys, vals, seed=1, dtype="u32")  # warm: the graph is built on first use
    sq.sync()
    keys.copy_(src)
    vals.copy_(torch.arange(n, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sq.sort(keys, vals, seed=2, dtype="u32")
    pending = not stream.query()
    sq.sync()
    assert pending, "the call waited for its work"
    unique_result(src, keys, vals)


def test_async_results_equal_the_oracle_and_host_rounds(sq):
    """Back-to-back asynchronous sorts on one stream, then on a second
    stream, against the oracle element by element."""
    cases = [(W.uniform_u32(1 << 20, 62), 3), (W.distinct16_u32(300001, 63), 4), (W.uniform_u32(70001, 64), 5)]
    outs = []
    side = torch.cuda.Stream()
    for j, (k, seed) in enumerate(cases):
        dk = torch.from_numpy(k.view(np.int32).copy()).cuda()
        dv = torch.arange(k.size, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        st = side if j == 2 else torch.cuda.current_stream()
        sq.sort(dk, dv, seed=seed, dtype="u32", stream=st)
        outs.append((dk, dv, st))
    for dk, dv, st in outs:
        sq.sync(st)
    for (k, seed), (dk, dv, _) in zip(cases, outs):
        ok, ov, _, _ = oracle.sort(k, W.iota(k.size), seed=seed, cutoff=sq.cutoff_for("u32", k.size))
        assert (dk.cpu().numpy().view(np.uint32) == ok).all() and (dv.cpu().numpy().view(np.uint32) == ov).all()


def test_latched_error_returned_by_sync_then_cleared(sq):
    """Repeated (key, val) pairs exhaust the pivot redraws on the device: the
    asynchronous call itself succeeds, sq_sync returns SQ_ERR_ATTEMPTS once,
    and the stream works again afterwards."""
    keys = torch.full((50000,), 7, dtype=torch.int32, device="cuda")
    vals = torch.zeros(50000, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    sq.sort(keys, vals, seed=1, dtype="u32", cutoff=16)
    with pytest.raises(sq.SquareSortError) as e:
        sq.sync()
    assert e.value.status == 7
    sq.sync()  # reported once
    k = W.uniform_u32(5000, 66)
    dk = torch.from_numpy(k.view(np.int32).copy()).cuda()
    dv = torch.arange(5000, dtype=torch.int32, device="cuda")
    sq.sort(dk, dv, seed=1, dtype="u32", cutoff=16)
    sq.sync()
    ok, ov, _, _ = oracle.sort(k, W.iota(5000), seed=1, cutoff=16)
    assert (dk.cpu().numpy().view(np.uint32) == ok).all() and (dv.cpu().numpy().view(np.uint32) == ov).all()


def test_latched_error_returned_by_the_next_call(sq):
    keys = torch.full((50000,), 9, dtype=torch.int32, device="cuda")
    vals = torch.zeros(50000, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    sq.sort(keys, vals, seed=1, dtype="u32", cutoff=16)
    torch.cuda.synchronize()  # the bad sort has finished; its error waits in the latch
    good = torch.from_numpy(W.uniform_u32(4000, 67).view(np.int32)).cuda()
    gv = torch.arange(4000, dtype=torch.int32, device="cuda")
    with pytest.raises(sq.SquareSortError) as e:
        sq.sort(good, gv, seed=2, dtype="u32")
    assert e.value.status == 7
    sq.sort(good, gv, seed=2, dtype="u32")
    sq.sync()
    assert bool((good.to(torch.int64) & 0xFFFFFFFF).diff().ge(0).all())


def test_batch_is_asynchronous_and_exact(sq):
    sizes = W.batch_sizes(200, 13, 8, 18)
    srcs = [W.uniform_u32(int(n), 80 + i) for i, n in enumerate(sizes)]
    batch = [(torch.from_numpy(s.view(np.int32).copy()).cuda(), torch.arange(s.size, dtype=torch.int32).cuda(), i)
             for i, s in enumerate(srcs)]
    before = sq.stats()["sorts"]
    torch.cuda.synchronize()
    sq.sort_batch(batch)
    sq.sync()
    assert sq.stats()["sorts"] - before == len(batch)
    for (bk, bv, i), s in zip(batch, srcs):
        ok, ov, _, _ = oracle.sort(s, W.iota(s.size), seed=i, cutoff=sq.cutoff_for("u32", s.size))
        assert (bk.cpu().numpy().view(np.uint32) == ok).all() and (bv.cpu().numpy().view(np.uint32) == ov).all()

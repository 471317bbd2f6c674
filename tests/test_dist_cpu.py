"""Multi-rank host logic on CPU with the gloo backend (world size 2): the
instance sharding used by the benchmark and the max-over-ranks timing."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2407_14801_gb300 import dist as D

    d = D.init(backend="gloo")
    r, w, lr = D.rank_world()
    share = list(D.shard(4097, r, w))
    t = D.max_over_ranks(1.5 + r, d)
    D.barrier(d)
    q.put((r, share[0], share[-1], len(share), t))
    d.destroy_process_group()


def test_shard_and_max_over_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, b0, n0, t0), (r1, a1, b1, n1, t1) = res
    assert (a0, b0, n0) == (0, 2048, 2049) and (a1, b1, n1) == (2049, 4096, 2048)
    assert t0 == t1 == 2.5


def test_shard_covers_everything():
    from paper_2407_14801_gb300 import dist as D

    for count in (0, 1, 7, 4096):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in D.shard(count, r, world)]
            assert got == list(range(count))

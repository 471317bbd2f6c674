"""Process-group helpers for multi-GPU runs (one process per GPU).

SquareSort instances are independent, so ranks never exchange data: each
rank sorts its own share of the instances (replicas of the single-instance
workload, or a slice of a batch) and the only collectives are a barrier and
the max-reduction of the timed duration.
"""
from __future__ import annotations

import os


def rank_world() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init(backend: str | None = None):
    """Initialise torch.distributed when WORLD_SIZE > 1; returns the module or None."""
    rank, world, _ = rank_world()
    if world <= 1:
        return None
    import torch.distributed as dist

    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend or "nccl", rank=rank, world_size=world)
    return dist


def shard(count: int, rank: int, world: int) -> range:
    """Contiguous share of `count` independent instances for `rank`."""
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank scalar (the timed duration) over all ranks."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist=None):
    if dist is not None:
        dist.barrier()

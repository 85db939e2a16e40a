"""Multi-GPU plumbing of the batch workloads: voxels are independent, so every rank solves
its own batch (weak scaling) and no collective touches the data path.  The only
collectives are the timing barrier and the max-over-ranks of the step time."""
from __future__ import annotations

import os


def rank_world() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (1 process = 1 GPU)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank r's synthetic batch: distinct independent batches per rank."""
    return base_seed + 1000 * rank


def shard(nitems: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of nitems for a rank (sizes differ by at most 1),
    for splitting one fixed batch across ranks (strong scaling)."""
    q, r = divmod(nitems, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (the step time the whole job waits for)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Multi-GPU host logic: independent meshes per rank (the method needs no
exchange between subdomains, §2.1, so ranks share nothing on the data path).

Each rank runs its own mesh generations: its own Philox key (`rank_seed`) or
its own slice of a request list (`shard`).  The only collective is the
max-over-ranks of the timed region for reporting (`max_over_ranks`), on
whatever process group is initialised (NCCL on GPUs, gloo in CPU tests).
"""
from __future__ import annotations

RANK_SEED_STRIDE = 1000003


def rank_seed(base_seed: int, rank: int) -> int:
    """Philox key of rank `rank`'s copy of a workload: distinct streams."""
    return int(base_seed) + RANK_SEED_STRIDE * int(rank)


def shard(items, rank: int, world: int):
    """Round-robin slice of a request list for one rank (disjoint, covering)."""
    return list(items)[rank::world]


def max_over_ranks(value: float, device=None) -> float:
    """MAX of a per-rank float over the default process group (identity when
    no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / t_max

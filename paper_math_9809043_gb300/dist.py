"""Host-side helpers for running independent solves on several GPUs.

The recursive multi-scale PCG of one problem does not shard (its coarse
levels are a sequential chain), so several GPUs only share a stream of
independent problems: each rank takes its own slice and no data-path
collective is needed.  The only collectives are the timing barrier and the
max-over-ranks reduction of the benchmark.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env_rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def shard(items, rank: int, world: int):
    """Contiguous, balanced slice of `items` for `rank` (sizes differ by <= 1)."""
    n = len(items)
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return items[lo:hi]


def shard_by_work(works, rank: int, world: int):
    """Greedy longest-first assignment of weighted items to ranks; returns
    the indices owned by `rank` (deterministic on every rank)."""
    order = sorted(range(len(works)), key=lambda i: (-works[i], i))
    load = [0.0] * world
    owner = [0] * len(works)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += works[i]
    return [i for i in range(len(works)) if owner[i] == rank]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over all ranks (the identity with one process)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None and torch.device(device).type == "cuda":
            dist.barrier(device_ids=[torch.device(device).index or 0])
        else:
            dist.barrier()

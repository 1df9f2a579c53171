"""Replicas across GPUs: one process per GPU, each simplifying its own scenes.

The simplification of one scene does not shard: the kNN search needs every
point of the scene and the greedy pair selection a global order, so a scene
split over GPUs would need a halo exchange per pass and a boundary exchange
per matching round.  Several GPUs therefore run independent replicas.  Each
rank processes its own scenes (the whole scene per rank for the headline
workload, a share of the scenes for the batched one), and the ranks meet only
to agree on timing: a barrier around the timed region and the maximum of the
ranks' times.  These host-side collectives run on gloo; there is no
data-path collective.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return ws, rank, local


def init():
    """Join the process group (gloo) when there is more than one rank."""
    ws, rank, _ = env()
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo")
    return ws, rank


def finish():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _reduce(x: float, op: str) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float) -> float:
    return _reduce(x, "max")


def sum_over_ranks(x: float) -> float:
    return _reduce(x, "sum")


def shard(items, rank: int, world_size: int):
    """This rank's share of a list of independent work items (round robin)."""
    return list(items)[rank::world_size]


def whole_job_rate(units_this_rank: float, seconds_this_rank: float) -> float:
    """Units of all ranks divided by the slowest rank's time."""
    units = sum_over_ranks(units_this_rank)
    secs = max_over_ranks(seconds_this_rank)
    return units / secs if secs > 0 else 0.0

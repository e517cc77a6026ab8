"""Running the stream on several GPUs: one process per GPU, no data-path
collective.

Histograms of disjoint pixel ranges add, and a stream's switch and pattern
depend only on its own previous chunks, so each rank runs its own stream over
its own share of the data.  The process group is used for three things only:
the barrier around a timed region, the slowest rank's time (a max over
ranks), and -- when a caller wants one histogram of everything -- a single
sum of the ranks' uint64 totals (2 KiB) at the end.

Rank variables follow torchrun: RANK, LOCAL_RANK, WORLD_SIZE.
"""
from __future__ import annotations

import os

import torch


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(count: int, world: int, rank: int) -> range:
    """The contiguous block of `count` units (chunks, images, requests) that
    `rank` owns: units are split as evenly as possible, lower ranks taking the
    extra one."""
    if world < 1 or not 0 <= rank < world or count < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def merge_totals(totals: torch.Tensor, group=None) -> torch.Tensor:
    """Sum the ranks' stream totals (uint64[256] held in an int64 tensor) in
    place: the histogram of every rank's data.  Counts stay exact below 2^63."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(totals, op=dist.ReduceOp.SUM, group=group)
    return totals


def slowest(seconds: float, device=None, group=None) -> float:
    """The largest of the ranks' times: a job is as fast as its slowest rank."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1):
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

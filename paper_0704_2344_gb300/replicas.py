"""Replicas on several GPUs.

The problems of the hot path are independent of one another: right-hand
sides of one system, or requests of a serving stream.  On N GPUs every rank
therefore solves its own share with no data exchange ("weak" scaling), and a
run is timed by its slowest rank.  These helpers hold that logic; they work
with any torch.distributed backend (NCCL on GPUs, gloo on the CPU in tests)
and degrade to no-ops in a single process.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def _multi() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def shard(items, rank: int, world: int):
    """This rank's share of independent work items: every world-th item."""
    return items[rank::world]


def barrier() -> None:
    if _multi():
        dist.barrier()


def max_over_ranks(values, device="cpu") -> list[float]:
    """Element-wise maximum over ranks (the slowest rank's times)."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if _multi():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def sum_over_ranks(values, device="cpu") -> list[float]:
    """Element-wise sum over ranks (work done by the whole job)."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if _multi():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.cpu()]

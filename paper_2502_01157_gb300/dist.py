"""Multi-process (one process per GPU) helpers.

Rays and cameras are independent, so a multi-GPU render partitions cameras
across ranks with no data-path communication; a training step sums the
per-rank site gradients (density, SH, positions) with one all-reduce, the
only exchange the method has.  Everything here is backend-agnostic
(``nccl`` on GPUs, ``gloo`` in the CPU tests).
"""
from __future__ import annotations

import os
from typing import Dict, List, Sequence

import torch
import torch.distributed as dist


def env_rank():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items: Sequence, rank: int, world: int) -> List:
    """Contiguous, balanced block of ``items`` owned by ``rank``."""
    n = len(items)
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return list(items[lo:hi])


def allreduce_grads(grads: Dict[str, torch.Tensor], group=None) -> Dict[str, torch.Tensor]:
    """Sum every gradient tensor over the ranks, in place."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        for k in sorted(grads):
            dist.all_reduce(grads[k], op=dist.ReduceOp.SUM, group=group)
    return grads


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar (the slowest rank's time)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

"""Replicas across GPUs: the PiT solves of a batch are independent problems,
so N GPUs run N replicas (one process per GPU) on disjoint seeded inputs
with no collective on the data path.  The only exchange is the timing
reduction: the whole job takes as long as its slowest rank.

Host logic only (no CUDA): the benchmark and the multi-process tests use it
with NCCL or gloo process groups alike.
"""
from __future__ import annotations

import os
from typing import Optional, Tuple

# seeds of rank r, step s: base + RANK_STRIDE r + STEP_STRIDE s (distinct
# for any r < STEP_STRIDE / RANK_STRIDE ranks and any step count used here)
RANK_STRIDE = 7919
STEP_STRIDE = 104729


def dist_env() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(base: int, rank: int, step: int = 0) -> int:
    """Seed of the inputs one rank solves at one step."""
    return base + RANK_STRIDE * rank + STEP_STRIDE * step


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity
    without an initialised process group)."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu().tolist()]


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Weak scaling: every rank processes the same number of units, and the
    job's time is the slowest rank's."""
    if seconds_max <= 0:
        raise ValueError("non-positive time")
    return units_per_rank * world / seconds_max


def barrier(device_index: Optional[int] = None) -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend() == "nccl" and device_index is not None:
            dist.barrier(device_ids=[device_index])
        else:
            dist.barrier()

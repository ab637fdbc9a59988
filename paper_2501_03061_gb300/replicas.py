"""Replica runs on several GPUs of one node (one process per GPU, launched by torchrun).

The hot path does not shard across GPUs here: every rank propagates its own system, with no
collective on the data path.  The only exchange between ranks is the job's timing: the job time
is the slowest rank's, and the job's throughput counts every rank's steps (weak scaling).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def slowest(seconds: float, device=None) -> float:
    """The largest of the ranks' times (this rank's time when there is no process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(seconds: float, steps: int, device=None) -> tuple[float, float]:
    """(job time = slowest rank, job throughput = all ranks' steps / job time)."""
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = slowest(seconds, device)
    return t, world * steps / t

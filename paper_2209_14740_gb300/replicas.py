"""Replica bookkeeping for multi-GPU runs of independent solves.

The SG solves do not shard: a run on N GPUs is N replicas, one process per
GPU, each solving its own systems.  There is no data-path collective; the
only communication is the barrier around the timed region and the maximum
of the per-rank times, from which the whole-job rate is formed.
"""
from __future__ import annotations

import os


def init(backend: str | None = None):
    """(world, rank, local_rank) from the torchrun environment; joins the
    process group when world > 1 (NCCL on GPUs unless `backend` says)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if backend is None:
            backend = "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int, device="cuda") -> float:
    """Largest value over the ranks (the slowest replica sets the job time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, max_seconds: float, world: int) -> float:
    """Units all ranks completed per second of the slowest rank."""
    return world * units_per_rank / max_seconds

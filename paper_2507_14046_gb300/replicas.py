"""Replica parallelism for independent sequences (one process per GPU).

Frames of one sequence are chained by TPP, so a sequence never spans GPUs; every rank fits
its own sequences and the ranks only meet to agree on the timed interval (a barrier and a
max over ranks).  There is no collective on the data path.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None) -> None:
    import torch
    import torch.distributed as dist
    _, size, _ = world()
    if size > 1 and not dist.is_initialized():
        dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds_max: float, size: int) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return size * units_per_rank / seconds_max

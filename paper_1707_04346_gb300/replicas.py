"""Replica bookkeeping for multi-GPU runs (one process per GPU).

The sigma build needs no exchange between GPUs here: each rank runs an
independent replica of the same workload ("replicas only": a row-sharded
sigma would need an all-gather of c per step, which a one-GPU run cannot
exercise).  Whole-job throughput is the units of all ranks divided by the
slowest rank's time.  NCCL when CUDA is available, else gloo (CPU tests).
"""
from __future__ import annotations

import os


def setup():
    """(rank, world_size, local_rank) from the torchrun environment; joins the
    process group when world_size > 1."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def _device():
    import torch
    import torch.distributed as dist

    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Weak scaling: every rank processes units_per_rank in its own replica."""
    return world * units_per_rank / seconds_max

"""Replica runs on several GPUs of one node: one independent run per rank (the
runs shard trivially -- there is no data exchange between them), so the only
collectives are a barrier and the max of the per-rank timings.  Works with
the NCCL backend (CUDA tensors) and with gloo (CPU tensors)."""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None) -> None:
    import torch
    import torch.distributed as dist

    if device is not None and torch.device(device).type == "cuda":
        torch.cuda.synchronize(device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_throughput(world: int, units_per_rank: float, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank does the same work)."""
    return world * units_per_rank / t_max


def replica_seed(base: int, rank: int) -> int:
    """Distinct seed per replica, so replicas are different runs."""
    return base + 1000003 * rank

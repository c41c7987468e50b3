"""Multi-process runs: one independent CDBM problem per rank ("replicas", weak
scaling).  The time step exchanges nothing between ranks; only the timing is
reduced: the job's time is the slowest rank's, and the job's throughput counts the
cells of every rank."""
from __future__ import annotations


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over the ranks of the default process group (the value
    itself without one).  device: where the reduction tensor lives (CUDA for NCCL)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / seconds_max

"""Multi-rank bookkeeping of the benchmark: every rank runs an independent replica (the method does not
exchange data between GPUs here), the job's rate is all ranks' work over the slowest rank's time."""
from __future__ import annotations


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, slowest_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    return units_per_rank * world / slowest_seconds

"""Host logic of multi-GPU runs: the method needs no communication (every processor holds
all tables, Sec. I of the paper), so N GPUs run N independent replicas over disjoint
slices of the quadruple stream (weak scaling).  The only collective is the timing
reduction: the job's time is the slowest rank's.  Works with any torch.distributed
backend (NCCL on GPUs, gloo on CPU for tests)."""
from __future__ import annotations


def quad_slice(rank: int, n_per_rank: int):
    """(first quadruple number, count) of `rank`'s slice of the seeded quadruple stream."""
    if rank < 0 or n_per_rank < 0:
        raise ValueError("rank and slice size must be non-negative")
    return rank * n_per_rank, n_per_rank


def max_over_ranks(ms: float, device=None) -> float:
    """Largest value of `ms` over all ranks (the job time); identity without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    v = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def job_throughput(units_per_rank: float, world: int, job_ms: float) -> float:
    """Whole-job rate: every rank processed units_per_rank in at most job_ms."""
    return world * units_per_rank / (job_ms * 1e-3)

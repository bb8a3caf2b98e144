"""Host-side logic of runs on several GPUs of one node (one process per GPU).

A single run does not shard (every mode-plane solve needs all of z at each node for the nonlinear
terms, so splitting it would take an all-to-all transpose per transform); a job on N GPUs is N
independent replicas, or an ensemble of independent runs split across ranks.  Nothing crosses
ranks on the data path: the only collectives are the timing barrier, the maximum of the ranks'
times and a gather of per-rank counts, all over torch.distributed (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import List, Sequence


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of rank `rank` among `world` ranks of n_units independent units
    (runs of an ensemble): sizes differ by at most one, shares are disjoint and cover all units."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("need 0 <= rank < world and n_units >= 0")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """The largest of the ranks' values (a job's time is its slowest rank's); the value itself
    when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_counts(count: int, device=None) -> List[int]:
    """Every rank's count (units processed), in rank order; [count] without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [int(count)]
    t = torch.tensor([int(count)], dtype=torch.int64, device=device)
    out = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [int(o.item()) for o in out]


def job_rate(units_per_rank: Sequence[int], max_seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    if not max_seconds > 0:
        raise ValueError("time must be positive")
    return float(sum(units_per_rank)) / max_seconds

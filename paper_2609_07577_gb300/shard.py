"""Job sharding for runs on several GPUs (one process per GPU). A single
hypergraph does not shard (every level needs global histograms, matching and
contraction), so independent jobs are dealt round-robin to ranks and run
with no collective on the data path; ranks only agree on timings."""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_jobs(n_jobs: int, rank: int, world: int) -> list[int]:
    """Jobs of `rank`: j with j % world == rank (disjoint, together all)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    return [j for j in range(n_jobs) if j % world == rank]


def _reduce(x: float, op, device) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value over ranks (the job's time is its slowest rank's)."""
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device="cpu") -> float:
    return _reduce(x, dist.ReduceOp.SUM, device)

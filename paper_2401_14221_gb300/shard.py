"""Sharding of independent tracks over ranks, and whole-job timing.

Tracks never interact (paper section 2: every track is propagated and
updated on its own), so a multi-GPU run gives each rank its own events and
needs no collective on the data path.  The only communication is for timing:
a barrier on both sides of the timed region and the maximum elapsed time
over ranks, from which the whole-job throughput is computed.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_seed(base_seed: int, rank: int) -> int:
    """Distinct, reproducible workload seed per rank."""
    return int(base_seed) + int(rank)


def shard_range(n: int, rank: int, world: int):
    """Contiguous [lo, hi) share of n items for `rank` (sizes differ by <= 1)."""
    q, r = divmod(int(n), int(world))
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def barrier(world: int):
    if world > 1:
        dist.barrier()


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank: int, steps: int, world: int, elapsed_max_s: float):
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank * steps / elapsed_max_s

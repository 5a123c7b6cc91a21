"""Sharding of cells over ranks (one process per GPU).

Cells are independent (the paper's thermochemistry step couples no two cells), so the
only multi-GPU structure is a partition of the cells: no data-path collective, only
the max-over-ranks of the timed interval and, for reporting, sums of counters.

Two partitions:
  weak scaling    every rank integrates its own full batch of the workload, drawn with
                  a rank-dependent seed (the benchmark: per-GPU work fixed as ranks grow);
  strong scaling  one batch split into contiguous cell ranges (a simulation's domain
                  decomposition); the union of the ranks' results is the single-process
                  result cell for cell.
"""
from __future__ import annotations

from typing import Tuple

from . import inputs as I

RANK_SEED_STRIDE = 1000


def rank_seed(workload_id: int, rank: int) -> int:
    """Seed of a rank's own batch under weak scaling (rank 0 draws the default batch)."""
    return I.SEED_BASE + workload_id + RANK_SEED_STRIDE * rank


def contiguous_range(ncells: int, rank: int, world: int) -> Tuple[int, int]:
    """[lo, hi) of rank's cells when ncells are split into world contiguous ranges whose
    sizes differ by at most one (the first ncells % world ranges get the extra cell)."""
    if world < 1 or not 0 <= rank < world or ncells < 0:
        raise ValueError(f"bad partition: ncells={ncells} rank={rank} world={world}")
    base, extra = divmod(ncells, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(seconds: float, device=None) -> float:
    """The slowest rank's time (all_reduce MAX); the local value without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank counter over ranks (the local value without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def weak_throughput(ncells_per_rank: int, world: int, steps: int, max_seconds: float) -> float:
    """Whole-job cell-integrations/s: every rank's cells over the slowest rank's time."""
    return world * ncells_per_rank * steps / max_seconds

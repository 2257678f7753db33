"""Walker sharding across ranks (one process per GPU).

Walkers are independent Markov chains (the paper runs one walker per core), so
rank k of a world of size P owns walkers [k W, (k + 1) W) and draws its random
numbers with those global walker indices: the union of the shards is bitwise
the single-process run of all P W walkers, with no data-path collective.  Only
the timing (and, if wanted, the energy accumulators) is reduced.
"""
from __future__ import annotations


def walker_offset(walkers_per_rank: int, rank: int) -> int:
    """Global index of this rank's first walker (the Philox walker counter base)."""
    if walkers_per_rank <= 0 or rank < 0:
        raise ValueError("walkers_per_rank must be positive and rank non-negative")
    return walkers_per_rank * rank


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a per-rank number (e.g. a timed region) over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(values, device=None):
    """Element-wise sum of per-rank accumulators (FP64)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(values, dtype=torch.float64, device=device).clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t

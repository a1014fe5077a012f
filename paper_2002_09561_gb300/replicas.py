"""Replica bookkeeping for one process per GPU.

Received vectors are independent, so N ranks each detect their own shard of
the workload stream with no collective on the data path.  The only exchanges
are at the end of a measurement: one max-reduction of the elapsed time (the
job takes as long as its slowest rank) and one sum-reduction of the int64
counters (bit and symbol errors, symbols, bits, visited nodes, radius
doublings) so that rank 0 reports the whole job's error rates.
"""

from __future__ import annotations


def shard(rank: int, world: int, per_rank: int):
    """(start, count): rank r detects vectors r*per_rank .. (r+1)*per_rank-1 of
    the seeded stream (weak scaling: per-rank work fixed)."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank / world / per_rank")
    return rank * per_rank, per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself without a group)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_counters(counts: dict, dist=None, device=None) -> dict:
    """Element-wise sum of integer counters over all ranks (same keys on every
    rank, in any order)."""
    keys = sorted(counts)
    if dist is None:
        return {k: int(counts[k]) for k in keys}
    import torch

    t = torch.tensor([int(counts[k]) for k in keys], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return {k: int(v) for k, v in zip(keys, t.tolist())}

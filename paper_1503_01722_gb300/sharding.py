"""Sharding of histories over GPUs and the one exchange step of the method.

Histories are independent (Sec. 2.2.1: one work-item per particle), and every
particle's random stream is keyed by its global history id, so a run of N
histories split into disjoint ranges over ranks gives, after an integer sum of
the int64 tallies, exactly the tally of the single run. The sum is the only
collective: one all-reduce of B x nvox int64 per step.
"""
from __future__ import annotations


def shard(rank: int, world: int, n_per_rank: int):
    """Weak scaling: rank r transports histories [r n, (r+1) n) of a run of world*n."""
    return rank * n_per_rank, n_per_rank, world * n_per_rank


def split(n_total: int, rank: int, world: int):
    """Strong scaling: contiguous, disjoint ranges covering [0, n_total)."""
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0), n_total


def allreduce_tally(engine, tally, dist, group=None):
    """Sum the int64 tallies of all ranks into `tally` (a device tensor of the engine's
    B x nz x ny x nx shape). Integer addition makes the result independent of the order."""
    engine.raw_tally(out=tally)
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally

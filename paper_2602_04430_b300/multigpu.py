"""One process per GPU for the operator path (host logic only).

Tuples are independent: an operator produces one output per item from that
item's own cache (Sec. 5), so ranks process disjoint tuple shards and nothing
on the data path crosses ranks.  The only collective is on the timing: the
job's time is the slowest rank's, and throughput is all ranks' units over it.

Two sharding modes:
  * ``weak``   -- every rank gets its own table of the same size (per-GPU work
                  fixed as ranks are added); seeds differ per rank.
  * ``strong`` -- one table split into contiguous shards whose sizes differ by
                  at most one tuple.
"""
from __future__ import annotations

from typing import List, Tuple


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank ``rank``'s synthetic table in weak scaling."""
    return base + 17 * rank


def shard_range(n_total: int, world: int, rank: int) -> Tuple[int, int]:
    """[begin, end) of rank ``rank``'s contiguous tuple shard (strong scaling)."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def reduce_max(value: float, dist=None, device=None) -> float:
    """Maximum of ``value`` over all ranks (the value itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: List[int], ms_max: float) -> float:
    """Whole-job throughput: units of all ranks per second of the slowest rank."""
    if ms_max <= 0:
        raise ValueError("non-positive time")
    return sum(units_per_rank) / (ms_max / 1000.0)

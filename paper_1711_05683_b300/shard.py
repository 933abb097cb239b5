"""Event-range sharding across ranks (one process per GPU).

Events are independent and counter-keyed, so N ranks each process their own disjoint
counter-event range with no collective on the data path; only the benchmark's timing uses a
barrier and a max over ranks.  These helpers are plain host logic, exercised with the gloo
backend on CPU by the tests.
"""
from __future__ import annotations


def rank_event_offset(rank: int, per_rank_events: int) -> int:
    """First counter-event index of `rank` when every rank processes per_rank_events events."""
    if rank < 0 or per_rank_events < 0:
        raise ValueError("rank and per_rank_events must be >= 0")
    return rank * per_rank_events


def rank_slice(rank: int, world: int, total: int, quantum: int = 1) -> tuple[int, int]:
    """[first, last) of a total split into world contiguous parts on multiples of `quantum`
    (e.g. 2^21 events so integral shards hold whole segments)."""
    units = (total + quantum - 1) // quantum
    lo = units * rank // world * quantum
    hi = min(total, units * (rank + 1) // world * quantum)
    return lo, hi


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over the ranks of the default process group (value if not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

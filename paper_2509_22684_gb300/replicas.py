"""Replicas across GPUs: independent transforms are split over ranks with no
data-path collective (each rank runs its share on its own GPU).  Collectives
are used only for barriers and for combining timings/counters.

A transform of 2^L elements costs about L * 2^L butterfly operations, so the
split is greedy largest-first onto the least-loaded rank (deterministic: every
rank computes the same assignment from the same list).
"""
from __future__ import annotations


def unit_cost(log_n: int) -> float:
    return float(log_n) * float(1 << log_n)


def shard_units(log_ns, world: int) -> list[list[int]]:
    """Indices of the units each rank runs; every index appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(log_ns)), key=lambda i: (-unit_cost(log_ns[i]), i))
    loads = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += unit_cost(log_ns[i])
    for p in parts:
        p.sort()
    return parts


def my_units(log_ns, rank: int, world: int) -> list[int]:
    return shard_units(log_ns, world)[rank]


def max_over_ranks(value: float, group=None, device=None) -> float:
    """Max of a host float over the process group (returns the value itself
    when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(value: float, group=None, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())

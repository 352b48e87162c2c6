"""Replica routing across GPUs: one process per GPU, no collective on the data path.

Data blocks and tracking streams are independent units of work (the paper
reaches real time by splitting the processing over the GPUs of two K80 boards,
Sec. 1.3), so N GPUs run N independent replicas. Each unit is routed to one
rank by a greedy longest-processing-time rule on its cost (for a DE fit,
N x pop x (gens + 1) sample-evaluations); each rank solves its own units and
only the small per-unit results and each rank's elapsed time travel, over
torch.distributed on the host (NCCL on GPU machines, gloo on CPU).

A fit needs no data from another rank, so the only collectives are the final
gather of results and the max-over-ranks of the timed region.
"""
from __future__ import annotations

import heapq
from typing import Any, List, Sequence


def assign(costs: Sequence[float], world: int) -> List[List[int]]:
    """Units per rank: longest-processing-time first onto the least-loaded rank.

    Deterministic: ties in cost keep the unit order, ties in load go to the
    lowest rank. Every unit lands on exactly one rank; within a rank, units
    keep their original order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    for c in costs:
        if not c >= 0.0:
            raise ValueError("costs must be non-negative numbers")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    for units in out:
        units.sort()
    return out


def my_units(costs: Sequence[float], world: int, rank: int) -> List[int]:
    """The units `rank` solves under assign()."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return assign(costs, world)[rank]


def gather(obj: Any) -> List[Any]:
    """Every rank's `obj`, in rank order (the caller's process group)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return [obj]
    out: List[Any] = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def max_over_ranks(x: float, device: str = "cpu") -> float:
    """The largest `x` over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

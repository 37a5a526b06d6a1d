"""Sharding an ensemble across processes (one GPU each).

Instances are independent -- each has its own grid, time step and CFL
control -- so an ensemble splits across ranks with no data-path
communication: every rank advances its own instances and only the final
states (or any per-instance diagnostics) are gathered.  The split balances
the total cells per rank (longest-processing-time-first greedy).
"""
from __future__ import annotations

from typing import List, Sequence


def partition_instances(cells: Sequence[int], world: int) -> List[List[int]]:
    """Instance indices for each of `world` ranks, balancing total cells."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(cells[i])
    return [sorted(p) for p in parts]


def gather_by_instance(local: dict, world: int, group=None) -> dict:
    """All-gather {instance index: value} dicts from every rank (any
    picklable values) into one dict on every rank."""
    import torch.distributed as dist
    if world == 1:
        return dict(local)
    out = [None] * world
    dist.all_gather_object(out, local, group=group)
    merged = {}
    for d in out:
        for k, v in d.items():
            if k in merged:
                raise RuntimeError(f"instance {k} produced by two ranks")
            merged[k] = v
    return merged

"""Host-side logic of the multi-GPU forms: one process per GPU, independent units per rank.

The streaming update of one stream is a chain of dependent steps and stays on one GPU (several
ranks run replicas). The batched form's streams are independent units: ranks take disjoint sets
of streams, balanced by their per-step cost, with no collective on the data path. A collective
only reduces the timing (max over ranks) and the unit count at the end of a run.
"""

from __future__ import annotations


def stream_cost(spatial) -> int:
    """Per-step cost proxy of a stream: elements of one slice (the update streams each slice once
    and its other passes scale with the slice size at fixed ranks)."""
    c = 1
    for n in spatial:
        c *= int(n)
    return c


def assign_streams(costs, world_size: int) -> list[list[int]]:
    """Partition stream indices among ranks: longest-processing-time-first greedy (each stream,
    largest cost first, goes to the rank with the least total cost so far; ties to the lower
    rank). Deterministic, so every rank computes the same partition without communicating."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world_size
    parts: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda j: (load[j], j))
        parts[r].append(i)
        load[r] += costs[i]
    for p in parts:
        p.sort()
    return parts


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

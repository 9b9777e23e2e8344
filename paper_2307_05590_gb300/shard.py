"""Sharding of the batched sweep over GPUs (one process per GPU).

The sweep has no data-path exchange: objects are independent, so a batch is split by object
and every rank sweeps its own part; the only collectives are for reporting (the slowest rank's
step time).  Two modes: weak scaling (every rank its own batch of the same size) and strong
scaling (one batch split by ``balanced_split``).
"""
from __future__ import annotations

import numpy as np


def sweep_cost(r, n_w: int) -> np.ndarray:
    """Relative cost of sweeping objects of basis size r over n_w frequencies on the pencil
    route, in float64 flops: the O(r^3) preparation once plus O(r) per frequency (the
    pole-split forms)."""
    r = np.asarray(r, dtype=np.float64)
    return 60.0 * r ** 3 + 130.0 * n_w * r


def balanced_split(costs, n_parts: int) -> list:
    """Greedy longest-processing-time split of objects into n_parts lists of indices (each
    sorted) with nearly equal total cost; every object appears exactly once."""
    costs = np.asarray(costs, dtype=np.float64)
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    load = np.zeros(n_parts)
    parts = [[] for _ in range(n_parts)]
    for k in np.argsort(-costs, kind="stable"):
        p = int(np.argmin(load))
        parts[p].append(int(k))
        load[p] += costs[k]
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over the ranks of the default process group (the value itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """The sum of value over the ranks of the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

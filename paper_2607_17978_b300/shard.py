"""Host-side helpers for running batches of independent structures on several GPUs.

The structures of a batch are independent QEq problems, so a multi-GPU run splits
them across ranks and every rank solves its share with no collective on the data
path (the paper's structure-level parallelism, Sec. 3, done with one process per
GPU).  The split is the greedy largest-first rule: structures in order of
decreasing cost, each onto the rank with the least cost so far.  The only
collective is the timing reduction (the slowest rank sets the step time).
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world size, local rank) from the torch.distributed launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def structure_cost(struct) -> float:
    """Work estimate of one structure: its atom count (per PCG iteration the mesh
    and pair work grow with the cell volume, i.e. with the atoms at fixed density)."""
    return float(struct.n)


def partition(costs, n_parts: int) -> list:
    """Split indices 0..len(costs)-1 into n_parts lists by the greedy largest-first rule.

    Deterministic: equal costs keep their index order, equal loads go to the lowest
    part.  Every part's indices are returned in increasing order.  The largest part's
    load is at most the mean load plus the largest single cost.
    """
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    loads = [0.0] * n_parts
    parts = [[] for _ in range(n_parts)]
    for i in order:
        p = min(range(n_parts), key=lambda k: (loads[k], k))
        parts[p].append(i)
        loads[p] += float(costs[i])
    return [sorted(p) for p in parts]


def rank_share(costs, rank: int, world: int) -> list:
    """Indices of the structures that rank `rank` of `world` solves."""
    return partition(costs, world)[rank]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

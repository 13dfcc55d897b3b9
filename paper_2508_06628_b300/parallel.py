"""Multi-process sharding of independent systems (one process per GPU).

Systems never interact, so the batch shards across ranks with no data-path
collective: each rank evolves its own systems and only the timing (a max over
ranks) and optional totals cross ranks.  The partition balances atoms with a
longest-processing-time greedy packing (the 1-D bin-packing idea of the
paper's BinningAutobatcher, Sec. 3, applied across devices).
"""
from __future__ import annotations

import numpy as np


def shard_systems(atoms_per_system, world):
    """Partition system indices over ``world`` ranks, balancing atom counts.
    Returns a list of sorted index arrays (one per rank); deterministic."""
    n = np.asarray(atoms_per_system, dtype=np.int64)
    order = np.lexsort((np.arange(len(n)), -n))     # largest first, ties by index
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(len(n), dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += n[i]
    return [np.sort(np.nonzero(owner == r)[0]) for r in range(world)]


def max_over_ranks(value, device=None):
    """Max of a float across ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t)
    return float(t.item())

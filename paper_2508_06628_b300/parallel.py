"""Multi-process sharding of independent systems (one process per GPU).

Systems never interact, so a batch shards across ranks with no data-path
collective: each rank evolves its own systems on its own GPU, and only the
results (gathered once at the end), the timing (a max over ranks) and the
sums a global observable needs cross ranks.  The partition balances atom
counts with a longest-processing-time greedy packing (the 1-D bin-packing
idea of the paper's BinningAutobatcher, Sec. 3, applied across devices).

The helpers take an optional torch.distributed process group; without an
initialised process group they behave as a single rank.
"""
from __future__ import annotations

import numpy as np


def rank_world(group=None):
    """(rank, world size) of this process, (0, 1) without torch.distributed."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


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


def my_shard(hb, group=None):
    """This rank's system indices of the host batch ``hb`` (workloads.Batch)."""
    rank, world = rank_world(group)
    return shard_systems(np.diff(hb.offsets), world)[rank]


def run_sharded(hb, fn, group=None):
    """Run ``fn(sub_batch)`` on this rank's shard of ``hb`` and gather the
    results on every rank.  ``fn`` returns a dict keyed by the system's index
    in ``sub_batch`` (0 .. n-1); the result is keyed by the index in ``hb``.
    One all-gather of the (host) result objects, after all the work."""
    import torch.distributed as dist
    ids = my_shard(hb, group)
    local = fn(hb.subset(ids)) if len(ids) else {}
    mine = {int(ids[k]): v for k, v in local.items()}
    rank, world = rank_world(group)
    if world == 1:
        return mine
    parts = [None] * world
    dist.all_gather_object(parts, mine, group=group)
    out = {}
    for p in parts:
        out.update(p)
    return out


def allreduce_sum(x, group=None):
    """Sum of a small float64 array over ranks (identity on one rank).  The
    array is reduced on the host: the sums here are a few numbers per call."""
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(x, dtype=np.float64)
    rank, world = rank_world(group)
    if world == 1:
        return a.copy()
    t = torch.from_numpy(a.copy())
    if dist.get_backend(group) == "nccl":   # NCCL reduces device tensors
        t = t.to(torch.device("cuda", torch.cuda.current_device()))
    dist.all_reduce(t, group=group)
    return t.cpu().numpy()


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

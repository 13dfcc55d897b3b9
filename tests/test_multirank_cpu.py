"""Multi-rank host logic on CPU (gloo, world size 2): the system partition is
complete, disjoint and balanced, ranks agree on it, and the timing/totals
reductions the benchmark uses behave as max / sum over ranks."""
import os

import numpy as np
import pytest

from paper_2508_06628_b300 import parallel, workloads as W


def test_shard_is_partition_and_balanced():
    hb = W.ragged_mix(seed=1, n_systems=512)
    n = np.diff(hb.offsets)
    for world in (1, 2, 3, 8):
        parts = parallel.shard_systems(n, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(n)))
        loads = np.array([n[p].sum() for p in parts])
        assert loads.max() - loads.min() <= n.max()


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hb = W.ragged_mix(seed=1, n_systems=64)
    parts = parallel.shard_systems(np.diff(hb.offsets), world)
    mine = parts[rank]
    tmax = parallel.max_over_ranks(1.0 + rank)
    atoms = parallel.sum_over_ranks(float(np.diff(hb.offsets)[mine].sum()))
    out.put((rank, mine.tolist(), tmax, atoms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted([q.get(timeout=120) for _ in ps])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    hb = W.ragged_mix(seed=1, n_systems=64)
    a, b = set(res[0][1]), set(res[1][1])
    assert not (a & b) and a | b == set(range(64))
    assert res[0][2] == res[1][2] == 2.0
    assert res[0][3] == res[1][3] == float(hb.n_atoms)

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


def _system_result(hb_sub, orc_forces):
    """Per-system results of a shard, computed system by system (stands in for
    a GPU relaxation or binned run: systems are independent)."""
    out = {}
    for k in range(hb_sub.n_systems):
        one = hb_sub.subset([k])
        E, F, S = orc_forces(one.offsets, one.pos, one.cell, one.pbc, one.pot_idx, one.pots)
        out[k] = dict(E=float(E[0]), fsum=float(np.abs(F).sum()), n=int(one.n_atoms))
    return out


def _rdf_terms(ids, K=16, P=2):
    """Deterministic per-system RDF rows and parameter Jacobians keyed by the
    system's global index (stand-ins for the GPU's RDF and adjoint)."""
    rows, jac = [], []
    for i in ids:
        r = np.random.default_rng(1000 + int(i))
        rows.append(r.uniform(0, 2, K))
        jac.append(r.normal(size=(K, P)))
    return np.array(rows).reshape(len(ids), K), np.array(jac).reshape(len(ids), K, P)


def _sharded_worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle import oracle
    from paper_2508_06628_b300 import grad
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hb = W.ragged_mix(seed=7, n_systems=20, lo=32, hi=128)
    res = parallel.run_sharded(hb, lambda sub: _system_result(sub, oracle.forces))
    # the sharded RDF-loss gradient's reductions: K bin sums forward, the
    # parameter gradient backward (rank-local systems only, global result)
    ids = parallel.my_shard(hb)
    rows, jac = _rdf_terms(ids)
    n_total = int(parallel.allreduce_sum([len(ids)])[0])
    g = parallel.allreduce_sum(rows.sum(0) / n_total)
    target = np.linspace(0.5, 1.5, rows.shape[1])
    loss, up = grad.rdf_mse_upstream(g, target, n_total, 1)
    gth = parallel.allreduce_sum(np.einsum("k,ikp->p", up, jac))
    out.put((rank, res, loss, gth.tolist(), len(ids)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sharded_results_and_gradient(orc):
    """A batch sharded over two ranks gives every system's result exactly as
    one rank does (gathered on both ranks, keyed by the global index), and the
    sharded RDF loss and parameter gradient (two all-reduces) equal the
    single-rank ones."""
    mp = pytest.importorskip("torch.multiprocessing")
    from paper_2508_06628_b300 import grad
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    ps = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted([q.get(timeout=300) for _ in ps], key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    hb = W.ragged_mix(seed=7, n_systems=20, lo=32, hi=128)
    single = _system_result(hb, orc.forces)
    for rank, res, loss, gth, n_local in got:
        assert sorted(res) == list(range(20))
        assert all(res[i] == single[i] for i in range(20))      # bit for bit: systems are independent
        assert 0 < n_local < 20
    rows, jac = _rdf_terms(np.arange(20))
    g = rows.sum(0) / 20
    loss1, up1 = grad.rdf_mse_upstream(g, np.linspace(0.5, 1.5, rows.shape[1]), 20, 1)
    gth1 = np.einsum("k,ikp->p", up1, jac)
    for _, _, loss, gth, _ in got:
        assert loss == pytest.approx(loss1, rel=1e-13)
        assert np.allclose(gth, gth1, rtol=1e-12, atol=1e-15)

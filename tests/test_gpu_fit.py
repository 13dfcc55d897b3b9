"""Differentiable fitting (Sec. 2, ref. [19]): Adam on the LJ sigma through the
checkpointed trajectory adjoint recovers the sigma of a target RDF computed
by the oracle with sigma = 1.05 (start 1.0)."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [1, 0])
def test_fit_sigma_to_target_rdf(orc, precision):
    torch_cuda()
    from paper_2508_06628_b300 import grad, ts
    hb = W.lj_liquid(seed=3, n_systems=2, reps=(3, 3, 3), rattle=0.08, kT=0.5)
    pot = dict(W.LJ_REDUCED)
    K, rmax, T, every, dt = 50, 2.5, 100, 20, 0.005
    _, target, _ = orc.traj_rdf_loss(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc,
                                     dict(pot, p=(1.05, 1.0, 0.0)), dt, T, every, rmax, K, np.zeros(K), grad=False)
    b = ts.Batch([dict(pot, skin=0.4)], hb.n_atoms, hb.n_systems, precision=precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    params, hist = grad.fit_rdf(b, s, target, dt, T, every, rmax, K, iters=15, lr=0.01, fit=((0, 0),), checkpoint=50)
    b.poll()
    losses = [h[0] for h in hist]
    assert abs(params[0, 0] - 1.05) < 5e-3
    assert min(losses) < 1e-2 * losses[0]
    assert params[0, 1] == 1.0                       # epsilon not fitted
    b.close()

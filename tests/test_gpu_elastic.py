"""Batched elastic constants on the GPU (12 strained copies of every system
in one pair-force call) against the oracle's stress differences, and the
Cauchy relation C12 = C44 of central forces for perfect FCC crystals at zero
pressure."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import torch_cuda
from tests.test_oracle_elastic import LJ, MORSE, _zero_pressure_a

pytestmark = pytest.mark.gpu


def test_elastic_constants_vs_oracle(orc):
    torch = torch_cuda()
    from paper_2508_06628_b300 import grad, ts
    rng = np.random.default_rng(4)
    systems = []
    for pot_i, pot, a0, reps in [(0, LJ, 1.5496, (4, 4, 4)), (1, MORSE, 3.6616, (4, 4, 4)), (1, MORSE, 3.6616, (3, 4, 5))]:
        a = _zero_pressure_a(pot, a0)
        pos, cell = W.lattice("fcc", reps, a)
        if reps == (3, 4, 5):   # a rattled, sheared copy: a general configuration
            cell = cell @ (np.eye(3) + np.array([[0, 0.03, 0], [0.03, 0, 0.01], [0, 0.01, 0]]))
            pos = pos @ (np.eye(3) + np.array([[0, 0.03, 0], [0.03, 0, 0.01], [0, 0.01, 0]])) + rng.normal(0, 0.02, pos.shape)
        systems.append(dict(pos=pos, vel=np.zeros_like(pos), mass=np.ones(len(pos)), cell=cell, pot=pot_i))
    hb = W.concat(systems, [LJ, MORSE])
    pots = [dict(p, skin=0.3) for p in hb.pots]
    s = ts.DeviceState.from_host(hb)
    C = grad.elastic_constants(pots, s, delta=1e-5).cpu().numpy()
    Cr = orc.elastic_constants(hb.offsets, hb.pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots, delta=1e-5)
    for k in range(3):
        scale = np.abs(Cr[k]).max()
        assert np.abs(C[k] - Cr[k]).max() <= 1e-6 * scale, k
    for k in (0, 1):   # perfect crystals at zero pressure
        assert C[k, 3, 3] == pytest.approx(C[k, 0, 1], rel=1e-6)
        assert C[k, 0, 0] > C[k, 0, 1] > 0

"""In-flight batched relaxation (Sec. 3, Fig. 3) on the GPU: a stream of 12
systems under a 760-atom budget; every system converges exactly once, the
active atom count never exceeds the budget, and each system ends where it
ends when relaxed alone (systems are independent and the layout is
batch-invariant)."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_inflight_fig3_stream_fp64():
    torch_cuda()
    from paper_2508_06628_b300 import runtime, ts
    hb = W.fire_stream(seed=21, n_systems=12, lo=32, hi=256, rattle=0.05)
    pots = [dict(W.MORSE_CU, skin=0.5)]
    rounds = []
    res, log = runtime.relax_inflight(hb, pots, max_scaler=760, max_active=16, n_inner=20, precision=ts.TS_FP64,
                                      on_round=rounds.append)
    assert sorted(res) == list(range(12))
    assert all(r["atoms"] <= 760 for r in log)
    assert any(r["admitted"] > 0 for r in log[1:])      # refilled after retirements
    for i in [0, 5, 11]:
        alone, _ = runtime.relax_inflight(hb.subset([i]), pots, max_scaler=760, max_active=1, n_inner=20,
                                          precision=ts.TS_FP64)
        a = alone[0]
        assert res[i]["E"] == pytest.approx(a["E"], rel=1e-9, abs=1e-12)
        assert np.allclose(res[i]["cell"], a["cell"], atol=1e-9)
        assert res[i]["fmax"] <= 1e-3 and res[i]["smax"] <= 1e-4


def test_inflight_byte_budget_density_scaler_fp64():
    """Admission by a device-memory budget with the n_atoms x density memory
    scaler (Sec. 3): the Fig. 2 probe turns the budget into a scaler limit,
    no round exceeds it or the atom capacity the budget leaves, the budget
    (not the 16-system cap) limits admission, every system relaxes exactly
    once and ends where it ends when relaxed alone."""
    torch_cuda()
    from paper_2508_06628_b300 import runtime, ts
    hb = W.fire_stream(seed=22, n_systems=20, lo=32, hi=256, rattle=0.05)
    pots = [dict(W.MORSE_CU, skin=0.5)]
    per_atom, per_sys = runtime.memory_model(pots, ts.TS_FP64)
    max_active = 16
    budget = int(per_sys * max_active + per_atom * 700)      # about 700 atoms beside 16 systems' overhead
    res, log = runtime.relax_inflight(hb, pots, max_active=max_active, n_inner=20, precision=ts.TS_FP64,
                                      memory_budget_bytes=budget, memory_scales_with="n_atoms_x_density")
    assert sorted(res) == list(range(20))
    n_of = np.diff(hb.offsets)
    dens = runtime.memory_sizes(hb, "n_atoms_x_density")
    probes = sorted({int(np.argmax(n_of)), int(np.argmax(dens))})
    limit, _ = runtime.max_scaler_from_budget(n_of[probes], dens[probes], per_atom, per_sys, budget)
    atoms_cap = int((budget - per_sys * max_active) / per_atom) - 32
    assert all(r["scaler"] <= limit * (1 + 1e-12) and r["atoms"] <= atoms_cap for r in log)
    assert log[0]["active"] < max_active            # the budget binds, not the system cap
    for i in [0, 7, 19]:
        alone, _ = runtime.relax_inflight(hb.subset([i]), pots, max_scaler=760, max_active=1, n_inner=20,
                                          precision=ts.TS_FP64)
        assert res[i]["E"] == pytest.approx(alone[0]["E"], rel=1e-9, abs=1e-12)
        assert np.allclose(res[i]["cell"], alone[0]["cell"], atol=1e-9)

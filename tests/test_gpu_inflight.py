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

"""Failure detection without a GPU fault: invalid input that the kernels' own
guards turn into the batch's sticky error word, read by ts_batch_poll.

* Neighbour-list overflow: every list append is guarded by the capacity, so a
  tiny max_neighbors only truncates the lists and raises the error; a batch
  created with the default capacity then runs clean.
* A non-finite position: the import leaves that atom's slot at its last
  finite value and raises the error; the next call with finite positions runs
  clean.
No kernel waits on a flag, so there is no device wait to time out."""
import numpy as np
import pytest

from tests.gpu_util import force_tolerance_ok, kinds_of, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def _forces(torch, ts, b, s, hb):
    F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    b.pair_forces(s, F, E)
    return F, E


def test_neighbor_overflow_is_reported_then_default_capacity_runs_clean(orc):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(71, n_systems=6, lo=32, hi=400)
    b = make_batch(hb, ts.TS_MIXED, max_neighbors=8)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    with pytest.raises(ts.TSError) as ei:
        b.poll()
    assert ei.value.status == ts.TS_ERR_NEIGHBOR_OVERFLOW
    b.poll()   # the error word was cleared by the first poll
    b.close()
    b = make_batch(hb, ts.TS_MIXED)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    F, E = _forces(torch, ts, b, s, hb)
    b.poll()
    pos = s.pos.cpu().numpy()
    Er, Fr, _ = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F.cpu().numpy(), Fr, hb.offsets, False, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_position_is_reported(orc, precision):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(72, n_systems=5, lo=32, hi=300)
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    F0, E0 = _forces(torch, ts, b, s, hb)
    b.poll()
    good = s.pos.clone()
    s.pos[7, 1] = float("nan")
    s.pos[hb.offsets[3] + 2, 0] = float("inf")
    _forces(torch, ts, b, s, hb)
    with pytest.raises(ts.TSError) as ei:
        b.poll()
    assert ei.value.status == ts.TS_ERR_NONFINITE
    # the slots kept their finite values: the returned positions are finite
    assert torch.isfinite(s.pos).all()
    s.pos.copy_(good)
    F1, E1 = _forces(torch, ts, b, s, hb)
    b.poll()
    Er, Fr, _ = orc.forces(hb.offsets, good.cpu().numpy(), hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F1.cpu().numpy(), Fr, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    assert np.all(np.abs(E1.cpu().numpy() - Er) <= (1e-6 if precision == 0 else 1e-9) * np.abs(Er) + 1e-9)
    b.close()

"""State exchange with the caller between calls.

* A host round trip of the exported state (positions and velocities copied
  out and back in, as a caller that keeps the state on the host does) leaves
  the trajectory bit-identical to calls that never touch it: the import sees
  the same values and neither re-splits positions nor marks forces stale.
* A caller that changes a system's periodicity or cell between calls gets
  forces for the new geometry (the per-system geometry and image tables are
  rebuilt only when something changed, and then they must be)."""
import numpy as np
import pytest

from tests.gpu_util import force_tolerance_ok, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def run(hb, round_trip, calls=4, n=10):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, 0)
    s = ts.DeviceState.from_host(hb)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        for c in range(calls):
            b.md_step(s, n, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=2, step0=n * c,
                      stream=stream)
            if round_trip:
                stream.synchronize()
                x, v = s.pos.cpu(), s.vel.cpu()
                s.pos.copy_(x.to("cuda"))
                s.vel.copy_(v.to("cuda"))
        b.poll(stream)
    stream.synchronize()
    out = s.pos.cpu().numpy(), s.vel.cpu().numpy(), b.counters()[1]
    b.close()
    return out


def test_host_round_trip_keeps_trajectory():
    hb = small_mix(131, n_systems=10, lo=32, hi=500)
    xa, va, ra = run(hb, False)
    xb, vb, rb = run(hb, True)
    assert ra == rb
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_periodicity_and_cell_changes_between_calls(orc):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(132, n_systems=4, lo=64, hi=300)
    b = make_batch(hb, 1)
    s = ts.DeviceState.from_host(hb)
    F = torch.zeros_like(s.pos)

    def check(pbc, cell):
        b.pair_forces(s, F, None, None)
        b.poll()
        _, Fr, _ = orc.forces(hb.offsets, s.pos.cpu().numpy(), cell, pbc, hb.pot_idx, hb.pots)
        ok, worst, _ = force_tolerance_ok(F.cpu().numpy(), Fr, hb.offsets, True)
        assert ok, worst

    pbc = hb.pbc.copy()
    check(pbc, hb.cell)
    pbc[1] = [1, 0, 1]                                  # system 1 opens an axis
    s.pbc.copy_(torch.as_tensor(pbc, device="cuda"))
    check(pbc, hb.cell)
    pbc[1] = [1, 1, 1]                                  # and closes it again
    s.pbc.copy_(torch.as_tensor(pbc, device="cuda"))
    check(pbc, hb.cell)
    cell = hb.cell.copy()
    cell[2] = cell[2] @ (np.eye(3) + np.diag([0.03, 0.0, -0.02]))   # system 2 strained
    s.cell.copy_(torch.as_tensor(cell, device="cuda"))
    check(pbc, cell)
    s.cell.copy_(torch.as_tensor(hb.cell, device="cuda"))           # back to the first cell
    check(pbc, hb.cell)
    b.close()

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

from tests.gpu_util import force_tolerance_ok, kinds_of, make_batch, small_mix, torch_cuda

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


@pytest.mark.parametrize("precision", [0, 1])
def test_positions_shifted_by_lattice_vectors_cost_no_relisting(orc, precision):
    """Positions handed back displaced by whole lattice vectors along the
    periodic axes (unwrapped coordinates) are the same configuration: the
    import takes the image nearest each atom's listing reference, so nothing
    re-lists and the forces are those of the original positions."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(131, n_systems=6, lo=32, hi=300)
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    F0 = torch.zeros_like(s.pos)
    b.pair_forces(s, F0, None, None)
    b.poll()
    _, r0 = b.counters()
    x = s.pos.cpu().numpy()
    rng = np.random.default_rng(7)
    off = hb.offsets
    xs = x.copy()
    for k in range(hb.n_systems):
        n = rng.integers(-2, 3, size=(off[k + 1] - off[k], 3)) * hb.pbc[k].astype(int)
        xs[off[k]:off[k + 1]] += n @ hb.cell[k]
    assert np.abs(xs - x).max() > 1.0
    s.pos.copy_(torch.as_tensor(xs, device="cuda"))
    F1 = torch.zeros_like(s.pos)
    b.pair_forces(s, F1, None, None)
    b.poll()
    _, r1 = b.counters()
    assert r1 == r0
    F0, F1 = F0.cpu().numpy(), F1.cpu().numpy()
    Er, Fr, _ = orc.forces(hb.offsets, xs, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F1, Fr, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    assert np.abs(F1 - F0).max() <= (1e-12 if precision == 1 else 1e-5) * np.abs(F0).max()
    b.close()

"""Dynamic pruning of the Verlet list in MD steps.

Forces in MD steps come from an inner list: the Verlet-list entries within
rc plus a fraction of the skin, re-filtered for a system once one of its
atoms moved half that fraction.  Every pair inside rc between two filterings
is in the inner list and pairs beyond rc contribute exactly zero, so the
trajectory is bit-identical to one computed from the full Verlet list
(TS_INNER=1: the inner list is the Verlet list).  Checked with Langevin
steps in both precisions, with positions moved by the caller and by FIRE
between MD calls (both must trigger a re-filtering), and with a cell changed
by the caller (which must trigger a re-listing)."""
import numpy as np
import pytest

from tests.gpu_util import make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def run(hb, precision, steps=150, jolt=False, fire=False):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(5)
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        for c in range(steps // 10):
            if jolt and c == 5:      # the caller moves every atom by 0.1 A: more than half the inner skin
                d = rng.normal(size=(hb.n_atoms, 3))
                d *= 0.1 / np.linalg.norm(d, axis=1, keepdims=True)
                s.pos.add_(torch.as_tensor(d, device="cuda"))
            if fire and c == 8:      # a few fixed-cell FIRE steps move the atoms outside MD
                P = ts.FireParams(0.1, 1.0, 1.1, 0.5, 0.1, 0.99, 0.2, 1e-3, 1e-4, 0.0, 5, 0)
                fs = torch.zeros(hb.n_systems * ts.FIRE_STATE_BYTES, dtype=torch.uint8, device="cuda")
                fv = torch.zeros((hb.n_atoms + 3 * hb.n_systems, 3), dtype=torch.float64, device="cuda")
                b.fire_init(s, P, fs, fv, stream=stream)
                b.fire_step(s, fs, fv, P, 5, stream=stream)
            b.md_step(s, 10, hb.meta["dt"], kind=1, gamma=hb.meta["gamma"], seed=4, step0=10 * c, stream=stream)
        b.poll(stream)
    stream.synchronize()
    out = s.pos.cpu().numpy(), s.vel.cpu().numpy(), b.counters()[1], b.prunes()
    b.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_pruned_md_bit_identical(monkeypatch, precision):
    hb = small_mix(111, n_systems=10, lo=32, hi=600)
    xa, va, ra, pa = run(hb, precision)
    monkeypatch.setenv("TS_INNER", "1")
    xb, vb, rb, _ = run(hb, precision)
    assert pa > 0                        # filterings happened
    assert ra == rb
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


@pytest.mark.parametrize("precision", [0, 1])
def test_pruned_md_after_caller_and_fire_moves(monkeypatch, precision):
    hb = small_mix(112, n_systems=8, lo=32, hi=400)
    xa, va, _, _ = run(hb, precision, jolt=True, fire=True)
    monkeypatch.setenv("TS_INNER", "1")
    xb, vb, _, _ = run(hb, precision, jolt=True, fire=True)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_cell_change_by_caller_relists(orc):
    """A caller that strains the cell (positions unchanged) gets forces for the
    new cell: the lists built for the old cell are re-listed."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(113, n_systems=4, lo=64, hi=300)
    b = make_batch(hb, 1)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    f = torch.zeros_like(s.pos)
    b.pair_forces(s, f, None, None)
    b.poll()
    _, r0 = b.counters()
    strain = np.eye(3) + np.diag([0.04, -0.03, 0.02])
    cell = hb.cell @ strain
    s.cell.copy_(torch.as_tensor(cell, device="cuda"))
    b.pair_forces(s, f, None, None)
    b.poll()
    _, r1 = b.counters()
    assert r1 - r0 == hb.n_systems
    F = f.cpu().numpy()
    _, Fr, _ = orc.forces(hb.offsets, s.pos.cpu().numpy(), cell, hb.pbc, hb.pot_idx, hb.pots)
    assert np.abs(F - Fr).max() <= 1e-9 * np.abs(Fr).max()
    b.close()


def test_pruned_md_large_system_mixed(monkeypatch):
    """A system above the shared-memory pair kernel's size (the gather kernel's
    inner-list path, mixed precision) beside small ones: bit-identical to MD
    from the full lists."""
    from paper_2508_06628_b300 import workloads as W
    rng = np.random.default_rng(7)
    small = small_mix(114, n_systems=4, lo=32, hi=200)
    pos, cell = W.lattice("fcc", (9, 9, 8), 5.26)                 # 2,592 argon atoms
    pos = pos + rng.normal(0.0, 0.05, pos.shape)
    mass = np.full(len(pos), 39.948)
    big = dict(pos=pos, vel=W.maxwell_boltzmann(rng, mass, W.KB_EV * 300.0), mass=mass, cell=cell, pot=0,
               kT=W.KB_EV * 300.0, uid=99)
    systems = [big] + [dict(pos=small.pos[a:e], vel=small.vel[a:e], mass=small.mass[a:e], cell=small.cell[k],
                            pot=int(small.pot_idx[k]), kT=W.KB_EV * 300.0, uid=k)
                       for k, (a, e) in enumerate(zip(small.offsets[:-1], small.offsets[1:]))]
    hb = W.concat(systems, small.pots)
    hb.meta = dict(small.meta)
    assert np.diff(hb.offsets).max() > 2048
    xa, va, ra, pa = run(hb, 0, steps=100)
    monkeypatch.setenv("TS_INNER", "1")
    xb, vb, rb, _ = run(hb, 0, steps=100)
    assert pa > 0 and ra == rb
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def _thin_cells_batch():
    """Thin cells whose lists reach images beyond |n_a| = 2 (a BCC argon and a
    BCC copper slab one cubic cell thick: widths below r_list / 2) beside
    ordinary cells, so that every inner-list format of the shared-memory pair
    kernel is exercised in one batch."""
    from paper_2508_06628_b300 import workloads as W
    rng = np.random.default_rng(17)
    systems = []
    for kind, reps, a, pot, sp in [("bcc", (1, 4, 4), 4.175, 0, "Ar"), ("bcc", (1, 3, 5), 2.865, 1, "Cu"),
                                   ("fcc", (3, 3, 3), 5.26, 0, "Ar"), ("fcc", (2, 3, 4), 3.61, 1, "Cu"),
                                   ("fcc", (4, 4, 2), 1.27, 2, "SS")]:
        pos, cell = W.lattice(kind, reps, a)
        pos = pos + rng.normal(0.0, 0.04, pos.shape)
        mass = np.full(len(pos), W.MASS[sp])
        systems.append(dict(pos=pos, vel=W.maxwell_boltzmann(rng, mass, W.KB_EV * 300.0), mass=mass, cell=cell,
                            pot=pot, kT=W.KB_EV * 300.0, uid=len(systems)))
    hb = W.concat(systems, [W.LJ_AR, W.MORSE_CU, W.SOFT_SPHERE])
    hb.meta = dict(dt=1.0 / W.T0_FS, gamma=0.01 * W.T0_FS)
    return hb


def test_pruned_md_all_inner_formats(monkeypatch, orc):
    """Systems whose inner lists hold staged-table entries and systems whose
    lists reach images beyond the staged table (global image shifts): MD is
    bit-identical with pruning on and off, and the forces after the run match
    the oracle."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    from tests.gpu_util import force_tolerance_ok, kinds_of
    hb = _thin_cells_batch()
    xa, va, ra, pa = run(hb, 0, steps=100)
    monkeypatch.setenv("TS_INNER", "1")
    xb, vb, rb, _ = run(hb, 0, steps=100)
    assert pa > 0 and ra == rb
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    monkeypatch.delenv("TS_INNER")
    b = make_batch(hb, 0)
    s = ts.DeviceState.from_host(hb)
    s.pos.copy_(torch.as_tensor(xa, device="cuda"))
    s.vel.copy_(torch.as_tensor(va, device="cuda"))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        b.md_step(s, 10, hb.meta["dt"], kind=1, gamma=hb.meta["gamma"], seed=4, step0=100, stream=stream)
        b.profile_pair(s, reps=1, stream=stream)   # a forces-only launch from the inner lists
        b.poll(stream)
    F = torch.zeros_like(s.pos)
    b.pair_forces(s, F)
    b.poll()
    Er, Fr, _ = orc.forces(hb.offsets, s.pos.cpu().numpy(), hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F.cpu().numpy(), Fr, hb.offsets, False, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    b.close()

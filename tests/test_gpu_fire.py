"""GPU parity of batched variable-cell FIRE against the FP64 oracle."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import frac_diff, make_batch, torch_cuda

pytestmark = pytest.mark.gpu

FIRE = dict(dt0=0.1, dt_max=1.0, finc=1.1, fdec=0.5, alpha0=0.1, falpha=0.99, maxstep=0.2, fmax=1e-3, smax=1e-4,
            p_ext=0.0, nmin=5, variable_cell=1)


def gpu_fire(hb, precision, n_steps, calls=1, **kw):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    prm = dict(FIRE); prm.update(kw)
    P = ts.FireParams(*[prm[k] for k in ["dt0", "dt_max", "finc", "fdec", "alpha0", "falpha", "maxstep", "fmax",
                                          "smax", "p_ext"]], prm["nmin"], prm["variable_cell"])
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    fs = torch.zeros(hb.n_systems * ts.FIRE_STATE_BYTES, dtype=torch.uint8, device="cuda")
    fvel = torch.zeros((hb.n_atoms + 3 * hb.n_systems, 3), dtype=torch.float64, device="cuda")
    conv = torch.zeros(hb.n_systems, dtype=torch.uint8, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    fm = torch.zeros_like(E)
    sm = torch.zeros_like(E)
    b.neighbor_build(s, force=True)
    b.fire_init(s, P, fs, fvel)
    for _ in range(calls):
        b.fire_step(s, fs, fvel, P, n_steps, conv, E, fm, sm)
    b.poll()
    return (s.pos.cpu().numpy(), s.cell.cpu().numpy(), conv.cpu().numpy().astype(bool), E.cpu().numpy(),
            fm.cpu().numpy(), sm.cpu().numpy(), fvel.cpu().numpy())


def test_fire_fp64_trajectory_matches_oracle(orc):
    """40 variable-cell FIRE steps on a ragged Morse Cu batch, FP64 mode: the
    positions, cells and energies follow the oracle step for step."""
    hb = W.fire_stream(seed=9, n_systems=4, lo=32, hi=256)
    x, h, conv, E, fm, sm, fv = gpu_fire(hb, 1, 20, calls=2)
    fr = orc.FireRun(hb.offsets, hb.pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    Er, fmr, smr = fr.step(40)
    assert np.abs(h - fr.cells).max() < 1e-9
    assert np.abs(frac_diff(x, fr.x, h, hb.offsets)).max() < 1e-8
    assert np.allclose(E, Er, rtol=1e-9) and np.allclose(fm, fmr, rtol=1e-6, atol=1e-9)
    assert np.array_equal(conv, fr.converged())


@pytest.mark.parametrize("precision", [0, 1])
def test_fire_relaxes_to_lattice_constant(orc, precision):
    """Mixed and FP64 FIRE relax a rattled, 3%-compressed Cu FCC supercell to
    the lattice constant that minimises the FCC lattice-vector sum."""
    from tests.test_oracle_dynamics import _fcc_energy_per_atom_numpy, _golden_section
    pot = W.MORSE_CU
    astar = _golden_section(lambda a: _fcc_energy_per_atom_numpy(pot, a), 3.3, 4.0)
    rng = np.random.default_rng(4)
    pos, cell = W.lattice("fcc", (2, 2, 2), 3.61 * 0.97)
    pos = pos + rng.normal(0, 0.05, pos.shape)
    hb = W.concat([dict(pos=pos, vel=np.zeros_like(pos), mass=np.full(32, 63.546), cell=cell, pot=0)], [pot])
    x, h, conv, E, fm, sm, fv = gpu_fire(hb, precision, 400, calls=3, fmax=1e-5, smax=1e-6)
    assert conv[0]
    a_fit = np.cbrt(abs(np.linalg.det(h[0])) / 8)
    assert a_fit == pytest.approx(astar, abs=1e-4)
    assert E[0] / 32 == pytest.approx(_fcc_energy_per_atom_numpy(pot, astar), abs=1e-6)


def test_fire_stream_batch_converges_like_oracle(orc):
    """A ragged batch relaxed to fmax 1e-3 eV/A and |sigma| 1e-4 eV/A^3 on both
    sides: every system converges, converged energies per atom agree."""
    hb = W.fire_stream(seed=13, n_systems=6, lo=64, hi=256)
    x, h, conv, E, fm, sm, fv = gpu_fire(hb, 0, 300, calls=4)
    fr = orc.FireRun(hb.offsets, hb.pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    for _ in range(6):
        Er, fmr, smr = fr.step(300)
        if fr.converged().all():
            break
    assert conv.all() and fr.converged().all()
    n = np.diff(hb.offsets)
    assert np.allclose(E / n, Er / n, atol=1e-5)
    assert np.all(fm <= 1e-3) and np.all(sm <= 1e-4)


def tiny_cells():
    """Cells narrower than the list radius along some axes, so that lists hold
    images up to |n| = 2..4 and the image bound moves as the cells relax: a
    compressed 1-atom primitive FCC cell, a rattled 4-atom cubic cell and a
    stretched 2x1x1 supercell (one wide and two narrow axes)."""
    rng = np.random.default_rng(21)
    a1 = 3.61 * 0.95
    prim = 0.5 * a1 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    systems = [dict(pos=np.zeros((1, 3)), vel=np.zeros((1, 3)), mass=np.full(1, 63.546), cell=prim, pot=0)]
    p4, c4 = W.lattice("fcc", (1, 1, 1), 3.61 * 0.97)
    p4 = p4 + rng.normal(0, 0.05, p4.shape)
    systems.append(dict(pos=p4, vel=np.zeros_like(p4), mass=np.full(4, 63.546), cell=c4, pot=0))
    p8, c8 = W.lattice("fcc", (2, 1, 1), 3.61 * 1.03)
    p8 = p8 + rng.normal(0, 0.05, p8.shape)
    systems.append(dict(pos=p8, vel=np.zeros_like(p8), mass=np.full(8, 63.546), cell=c8, pot=0))
    return W.concat(systems, [W.MORSE_CU])


@pytest.mark.parametrize("precision", [0, 1])
def test_fire_tiny_cells_match_oracle(orc, precision):
    """Variable-cell FIRE on cells whose lists reach 2-4 images out: the image
    tables, rebuilt every step only for the codes the lists and the wrap can
    read, give the oracle's trajectory."""
    hb = tiny_cells()
    x, h, conv, E, fm, sm, fv = gpu_fire(hb, precision, 15, calls=2)
    fr = orc.FireRun(hb.offsets, hb.pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    Er, fmr, smr = fr.step(30)
    moved = np.abs(fr.cells - hb.cell).max(axis=(1, 2))
    assert np.all(moved > 1e-3)                       # every cell took part in the relaxation
    if precision == 1:
        assert np.abs(h - fr.cells).max() < 1e-9
        assert np.abs(frac_diff(x, fr.x, h, hb.offsets)).max() < 1e-8
        assert np.allclose(E, Er, rtol=1e-9)
    else:
        assert np.abs(h - fr.cells).max() < 1e-5 * np.abs(fr.cells).max()
        assert np.abs(frac_diff(x, fr.x, h, hb.offsets)).max() < 1e-5
        assert np.allclose(E, Er, rtol=1e-5, atol=1e-5)

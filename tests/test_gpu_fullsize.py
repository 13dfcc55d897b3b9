"""Parity at full workload sizes, in the launch configuration bench.py times:
sampled systems against the oracle one by one, and size-independent
properties (Newton's third law, finite energies) for every system."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import force_tolerance_ok, frac_diff, kinds_of, torch_cuda

pytestmark = pytest.mark.gpu


def test_ragged_mix_512_sampled(orc):
    """The 512-system benchmark batch: forces on 8 sampled systems and ten
    BAOAB steps (one CUDA-graph call, as timed) on 4 sampled systems."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = W.ragged_mix(seed=1, n_systems=512)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots))]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems)
    s = ts.DeviceState.from_host(hb)
    F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    b.neighbor_build(s, force=True)
    b.pair_forces(s, F, E)
    b.poll()
    F, E, pos = F.cpu().numpy(), E.cpu().numpy(), s.pos.cpu().numpy()
    off = hb.offsets
    for k in range(hb.n_systems):   # Newton's third law for every system
        fk = F[off[k]:off[k + 1]]
        assert np.abs(fk.sum(0)).max() <= 1e-5 * max(np.abs(fk).max(), 1e-3) * np.sqrt(len(fk)) + 1e-9
    assert np.all(np.isfinite(E))
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(hb.n_systems, 8, replace=False))
    sub = hb.subset(pick)
    sub.pos = np.concatenate([pos[off[k]:off[k + 1]] for k in pick])
    Er, Fr, _ = orc.forces(sub.offsets, sub.pos, sub.cell, sub.pbc, sub.pot_idx, sub.pots, use_cells=True)
    Fs = np.concatenate([F[off[k]:off[k + 1]] for k in pick])
    ok, worst, frac = force_tolerance_ok(Fs, Fr, sub.offsets, False, kinds=kinds_of(sub))
    assert ok, (worst, frac)
    assert np.all(np.abs(E[pick] - Er) <= 1e-6 * np.abs(Er) + 1e-9)
    # ten BAOAB steps as the bench runs them
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.md_step(s, 10, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=5, step0=0, stream=stream)
        b.poll(stream)
    x1 = s.pos.cpu().numpy()
    pick4 = pick[:4]
    sub4 = hb.subset(pick4)
    sub4.pos = np.concatenate([pos[off[k]:off[k + 1]] for k in pick4])
    xr, vr, _, _ = orc.md(sub4.offsets, sub4.pos, sub4.vel, sub4.mass, sub4.cell, sub4.pbc, sub4.pot_idx, sub4.pots,
                          hb.meta["dt"], 10, kind=1, kT=sub4.kT, gamma=hb.meta["gamma"], seed=5, uid=sub4.uid,
                          use_cells=True)
    xg = np.concatenate([x1[off[k]:off[k + 1]] for k in pick4])
    assert np.abs(frac_diff(xg, xr, sub4.cell, sub4.offsets)).max() < 1e-6


def test_large_scale_8x2048000_lj(orc):
    """Eight 2.048 M-atom reduced-LJ FCC boxes (rho* = 0.85), rattled: the
    multi-kernel re-listing path and the L1-gather pair kernel at full size.
    One whole box (box 5) is compared atom by atom with the oracle in
    cell-list mode at the mixed-precision tolerance; Newton's third law and the
    perfect-lattice energy per atom bound every box; then 20 NVE steps."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = W.lj_liquid(seed=4, n_systems=8, reps=(80, 80, 80), rho=0.85, kT=1.2, rattle=0.02)
    pots = [dict(hb.pots[0], skin=0.3)]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems)
    s = ts.DeviceState.from_host(hb)
    F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    S = torch.zeros((hb.n_systems, 3, 3), dtype=torch.float64, device="cuda")
    b.neighbor_build(s, force=True)
    b.pair_forces(s, F, E, S)
    b.poll()
    Fh = F.view(8, -1, 3)
    assert torch.all(Fh.sum(1).abs().max(1).values <= 1e-5 * Fh.abs().amax((1, 2)) * 2048.0)
    n = 2048000
    e_atom = E.cpu().numpy() / n
    # a 0.02 sigma rattle raises the energy above the perfect FCC lattice sum
    # (-6.38315 per atom at rho* 0.85, rc 2.5, shifted) by the harmonic
    # 3/2 K <u^2> ~ 0.04; the eight boxes agree to their sampling noise
    assert np.all(e_atom > -6.38315) and np.all(e_atom < -6.30)
    assert e_atom.max() - e_atom.min() < 1e-3
    # one whole box against the oracle, element by element
    k = 5
    a, e = hb.offsets[k], hb.offsets[k + 1]
    sub = hb.subset([k])
    pos = s.pos[a:e].cpu().numpy()
    Er, Fr, Sr = orc.forces(sub.offsets, pos, sub.cell, sub.pbc, sub.pot_idx, sub.pots, use_cells=True)
    Fg = F[a:e].cpu().numpy()
    ok, worst, frac = force_tolerance_ok(Fg, Fr, sub.offsets, False, kinds=[0])
    assert ok, (worst, frac)
    assert abs(E[k].item() - Er[0]) <= 1e-6 * abs(Er[0])
    Sg = S[k].cpu().numpy()
    assert np.abs(Sg - Sr[0]).max() <= 1e-6 * np.abs(Sr[0]).max() + 1e-9
    # MD through the large path stays consistent
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.md_step(s, 20, 0.005, kind=ts.TS_NVE, stream=stream)
        b.poll(stream)
    assert torch.isfinite(s.pos).all()

"""Non-periodic axes on the GPU path: no images and no wrapping along them.

A batch of an argon slab (open in z, a few atoms above the cell), a copper
wire (periodic in x only), a copper cluster (open in every axis, partly
outside its box) and a sheared soft-sphere film (open in z).  Pair sets,
forces, energies and stresses match the oracle, an FP64 NVE trajectory
follows it, and variable-cell FIRE refuses such systems.
"""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import force_tolerance_ok, kinds_of, frac_diff, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu

KB = 8.617333262e-5   # eV/K


def open_mix():
    rng = np.random.default_rng(91)
    pots = small_mix(1, n_systems=3).pots   # LJ argon, Morse copper, soft sphere
    systems, pbcs = [], []

    def add(p, c, pot, mass, pbc):
        v = W.maxwell_boltzmann(rng, np.full(len(p), mass), KB * 50.0)
        systems.append(dict(pos=p, vel=v, mass=np.full(len(p), mass), cell=c, pot=pot))
        pbcs.append(pbc)

    p, c = W.lattice("fcc", (3, 3, 3), 5.26)             # argon slab with 12 A of vacuum
    c = c.copy(); c[2, 2] += 12.0
    p = p + rng.normal(0, 0.05, p.shape)
    p[:4, 2] += c[2, 2] + 0.5                            # beyond the cell along the open axis
    add(p, c, 0, 39.948, (1, 1, 0))
    p, c = W.lattice("fcc", (4, 2, 2), 3.61)             # copper wire along x
    c = c.copy(); c[1, 1] += 8.0; c[2, 2] += 8.0
    add(p + rng.normal(0, 0.05, p.shape), c, 1, 63.546, (1, 0, 0))
    p, c = W.lattice("fcc", (3, 3, 3), 3.61)             # copper cluster, partly below the box origin
    add(p - 2.0 + rng.normal(0, 0.05, p.shape), np.eye(3) * 30.0, 1, 63.546, (0, 0, 0))
    p, c = W.lattice("fcc", (3, 3, 2), 1.27)             # sheared soft-sphere film
    c = c.copy(); c[2, 2] += 3.0; c[1, 0] += 0.4
    add(p + rng.normal(0, 0.02, p.shape), c, 2, 1.0, (1, 1, 0))
    hb = W.concat(systems, pots)
    hb.pbc[:] = np.array(pbcs, np.uint8)
    return hb


def run_forces(hb, precision):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    S = torch.zeros((hb.n_systems, 3, 3), dtype=torch.float64, device="cuda")
    b.neighbor_build(s, force=True)
    b.pair_forces(s, F, E, S)
    j, img, cnt = b.neighbor_export(s)
    b.poll()
    out = (F.cpu().numpy(), E.cpu().numpy(), S.cpu().numpy(), s.pos.cpu().numpy(), j.cpu().numpy(),
           img.cpu().numpy(), cnt.cpu().numpy())
    b.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_open_axes_pair_sets(orc, precision):
    from paper_2508_06628_b300 import ts
    hb = open_mix()
    _, _, _, pos, j, img, cnt = run_forces(hb, precision)
    off = hb.offsets
    for k in range(hb.n_systems):
        a, e = off[k], off[k + 1]
        pot = hb.pots[hb.pot_idx[k]]
        rl = pot["rc"] + ts.default_skins([pot])[0]
        h = hb.cell[k]
        ref = orc.neighbors(pos[a:e], h, list(hb.pbc[k]), rl)

        def near_cut(i, jj, n):
            d = pos[a + jj] - pos[a + i] + np.asarray(n) @ h
            return abs(np.linalg.norm(d) - rl) < 1e-6

        R = {(int(q[0]), int(q[1]), *map(int, q[2:])) for q in ref if not near_cut(q[0], q[1], q[2:])}
        G = {(i - a, int(j[i, q]) - a, *map(int, img[i, q])) for i in range(a, e) for q in range(cnt[i])}
        G = {t for t in G if not near_cut(t[0], t[1], t[2:])}
        assert G == R, f"system {k}: {len(G ^ R)} pairs differ"
        # no image along an open axis
        assert all(t[2 + ax] == 0 for t in G for ax in range(3) if not hb.pbc[k][ax])


@pytest.mark.parametrize("precision", [0, 1])
def test_open_axes_forces(orc, precision):
    hb = open_mix()
    F, E, S, pos, *_ = run_forces(hb, precision)
    # positions are not wrapped along open axes
    off = hb.offsets
    for k in range(hb.n_systems):
        g = (pos[off[k]:off[k + 1]] - hb.pos[off[k]:off[k + 1]]) @ np.linalg.inv(hb.cell[k])
        for ax in range(3):
            if not hb.pbc[k][ax]:
                assert np.abs(g[:, ax]).max() < 1e-12
    Er, Fr, Sr = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F, Fr, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    if precision == 1:
        assert np.allclose(E, Er, rtol=1e-9, atol=1e-12)
        assert np.allclose(S, Sr, rtol=1e-9, atol=1e-14)
    else:
        assert np.all(np.abs(E - Er) <= 1e-6 * np.abs(Er) + 1e-9)
        for k in range(hb.n_systems):
            assert np.abs(S[k] - Sr[k]).max() <= 1e-5 * np.abs(Sr[k]).max() + 1e-9


def test_open_axes_nve_fp64(orc):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = open_mix()
    dt = 2.0 / W.T0_FS
    b = make_batch(hb, 1)
    s = ts.DeviceState.from_host(hb)
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    KE = torch.zeros_like(E)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for c in range(3):
            b.md_step(s, 20, dt, kind=0, E=E, KE=KE, stream=stream)
        b.poll(stream)
    stream.synchronize()
    x, v = s.pos.cpu().numpy(), s.vel.cpu().numpy()
    xr, vr, Er, KEr = orc.md(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots, dt, 60,
                             use_cells=True)
    assert np.abs(frac_diff(x, xr, hb.cell, hb.offsets)).max() < 1e-9
    assert np.abs(v - vr).max() < 1e-10
    assert np.allclose(E.cpu().numpy(), Er, rtol=1e-9, atol=1e-12)
    assert np.allclose(KE.cpu().numpy(), KEr, rtol=1e-9)
    b.close()


def test_variable_cell_fire_refuses_open_axes():
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = open_mix()
    P = ts.FireParams(0.1, 1.0, 1.1, 0.5, 0.1, 0.99, 0.2, 1e-3, 1e-4, 0.0, 5, 1)
    b = make_batch(hb, 0)
    s = ts.DeviceState.from_host(hb)
    fs = torch.zeros(hb.n_systems * ts.FIRE_STATE_BYTES, dtype=torch.uint8, device="cuda")
    fvel = torch.zeros((hb.n_atoms + 3 * hb.n_systems, 3), dtype=torch.float64, device="cuda")
    b.neighbor_build(s, force=True)
    b.fire_init(s, P, fs, fvel)
    with pytest.raises(ts.TSError) as ei:
        b.fire_step(s, fs, fvel, P, 2)
        b.poll()
    assert ei.value.status == ts.TS_ERR_UNSUPPORTED

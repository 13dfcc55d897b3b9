"""NPT on the GPU (isotropic barostat of Martyna, Tobias and Klein with
Langevin friction and noise on atoms and piston) against the oracle: the FP64
trajectory, cell and piston state over two calls (the state carries over), a
short mixed-precision run, the conserved enthalpy of a frictionless run, and
the refusal of open axes."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import frac_diff, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu

GPA = 1.0 / 160.21766208        # eV/A^3 per GPa


def gpu_npt(hb, precision, calls, n, dt, gamma, tau, p_ext, kT, seed=7):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    kTd = torch.as_tensor(kT, dtype=torch.float64, device="cuda")
    ve = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    KE = torch.zeros_like(E)
    out = []
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for c in range(calls):
            b.md_step(s, n, dt, kind=ts.TS_NPT_LANGEVIN, gamma=gamma, kT=kTd, seed=seed, step0=n * c, tau=tau,
                      p_ext=p_ext, baro=ve, E=E, KE=KE, stream=stream)
            b.poll(stream)
            stream.synchronize()
            out.append((E.cpu().numpy().copy(), KE.cpu().numpy().copy(), ve.cpu().numpy().copy(),
                        s.cell.cpu().numpy().copy()))
    res = s.pos.cpu().numpy(), s.vel.cpu().numpy(), out
    b.close()
    return res


def test_npt_fp64_matches_oracle(orc):
    hb = small_mix(121, n_systems=6, lo=32, hi=300)
    dt, gamma, tau = hb.meta["dt"], hb.meta["gamma"], 100.0 / W.T0_FS
    kT = W.KB_EV * np.linspace(250.0, 450.0, hb.n_systems)
    p_ext = 1.0 * GPA
    x, v, out = gpu_npt(hb, 1, 2, 15, dt, gamma, tau, p_ext, kT)
    xr, vr, hr, ver, Er, Kr, _, _ = orc.md_npt(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx,
                                               hb.pots, dt, 30, kT, gamma, tau, p_ext, seed=7, use_cells=True)
    E, K, ve, h = out[-1]
    assert np.abs(h / hb.cell - 1).max() > 1e-5                      # the cells moved
    assert np.abs(h - hr).max() <= 1e-10 * np.abs(hr).max()
    assert np.abs(ve - ver).max() <= 1e-9 * max(np.abs(ver).max(), 1e-12)
    assert np.abs(frac_diff(x, xr, hr, hb.offsets)).max() < 1e-9
    assert np.abs(v - vr).max() < 1e-10
    assert np.allclose(E, Er, rtol=1e-9, atol=1e-12) and np.allclose(K, Kr, rtol=1e-9)


def test_npt_mixed_short_run(orc):
    hb = small_mix(122, n_systems=6, lo=32, hi=300)
    dt, gamma, tau = hb.meta["dt"], hb.meta["gamma"], 100.0 / W.T0_FS
    kT = np.full(hb.n_systems, W.KB_EV * 300.0)
    x, v, out = gpu_npt(hb, 0, 1, 5, dt, gamma, tau, 0.0, kT)
    xr, vr, hr, ver, Er, Kr, _, _ = orc.md_npt(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx,
                                               hb.pots, dt, 5, kT, gamma, tau, 0.0, seed=7, use_cells=True)
    E, K, ve, h = out[-1]
    assert np.abs(h - hr).max() <= 1e-7 * np.abs(hr).max()
    assert np.abs(ve - ver).max() <= 1e-4 * np.abs(ver).max()
    assert np.abs(frac_diff(x, xr, hr, hb.offsets)).max() < 1e-6
    assert np.abs(v - vr).max() < 1e-5 * np.abs(vr).max()
    assert np.all(np.abs(E - Er) <= 1e-6 * np.abs(Er) + 1e-6)
    assert np.allclose(K, Kr, rtol=1e-5)


def test_npt_mixed_enthalpy_conserved():
    """Without friction the mixed-precision run keeps K + U + W v_e^2/2 +
    p_ext V while the piston moves real energy (and the systems re-list as
    their cells change)."""
    hb = small_mix(123, n_systems=4, lo=64, hi=400)
    dt, tau = hb.meta["dt"], 50.0 / W.T0_FS
    kT = np.full(hb.n_systems, W.KB_EV * 300.0)
    p_ext = 2.0 * GPA
    _, _, out = gpu_npt(hb, 0, 20, 50, dt, 0.0, tau, p_ext, kT)
    n = np.diff(hb.offsets)
    Wp = (3.0 * n + 3.0) * kT * tau * tau
    H = np.array([E + K + 0.5 * Wp * ve ** 2 + p_ext * np.abs(np.linalg.det(h)) for E, K, ve, h in out])
    KU = np.array([E + K for E, K, _, _ in out])
    V = np.array([np.abs(np.linalg.det(h)) for _, _, _, h in out])
    assert np.all(KU.max(0) - KU.min(0) > 0.02)
    assert np.all((V.max(0) - V.min(0)) / V.min(0) > 1e-3)
    assert np.all(np.abs(H - H[0]).max(0) < 0.05 * (KU.max(0) - KU.min(0)))


def test_npt_refuses_open_axes():
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(124, n_systems=3, lo=32, hi=100)
    hb.pbc[1] = [1, 1, 0]
    b = make_batch(hb, 0)
    s = ts.DeviceState.from_host(hb)
    ve = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    kT = torch.full((hb.n_systems,), W.KB_EV * 300.0, dtype=torch.float64, device="cuda")
    with pytest.raises(ts.TSError) as ei:
        b.md_step(s, 2, hb.meta["dt"], kind=ts.TS_NPT_LANGEVIN, gamma=0.01, kT=kT, tau=10.0, baro=ve)
        b.poll()
    assert ei.value.status == ts.TS_ERR_UNSUPPORTED
    b.close()


def test_npt_mixed_large_system(orc):
    """A system above 2048 atoms (the gather pair kernel and the multi-kernel
    re-listing) under the barostat beside small ones, mixed precision, against
    the oracle over a short run."""
    rng = np.random.default_rng(8)
    small = small_mix(125, n_systems=3, lo=32, hi=200)
    pos, cell = W.lattice("fcc", (9, 9, 8), 5.26)
    pos = pos + rng.normal(0.0, 0.05, pos.shape)
    mass = np.full(len(pos), 39.948)
    big = dict(pos=pos, vel=W.maxwell_boltzmann(rng, mass, W.KB_EV * 300.0), mass=mass, cell=cell, pot=0,
               kT=W.KB_EV * 300.0, uid=9)
    systems = [big] + [dict(pos=small.pos[a:e], vel=small.vel[a:e], mass=small.mass[a:e], cell=small.cell[k],
                            pot=int(small.pot_idx[k]), kT=W.KB_EV * 300.0, uid=k)
                       for k, (a, e) in enumerate(zip(small.offsets[:-1], small.offsets[1:]))]
    hb = W.concat(systems, small.pots)
    hb.meta = dict(small.meta)
    dt, gamma, tau = hb.meta["dt"], hb.meta["gamma"], 50.0 / W.T0_FS
    kT = np.full(hb.n_systems, W.KB_EV * 300.0)
    p_ext = 0.5 * GPA
    x, v, out = gpu_npt(hb, 0, 1, 5, dt, gamma, tau, p_ext, kT)
    xr, vr, hr, ver, Er, Kr, _, _ = orc.md_npt(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx,
                                               hb.pots, dt, 5, kT, gamma, tau, p_ext, seed=7, uid=hb.uid,
                                               use_cells=True)
    E, K, ve, h = out[-1]
    assert np.abs(h - hr).max() <= 1e-7 * np.abs(hr).max()
    assert np.abs(frac_diff(x, xr, hr, hb.offsets)).max() < 1e-6
    assert np.abs(v - vr).max() < 1e-5 * np.abs(vr).max()
    assert np.all(np.abs(E - Er) <= 1e-6 * np.abs(Er) + 1e-6)

"""NVT Nose-Hoover chain on the GPU against the oracle: FP64 trajectory and
chain state over two calls (the state carries over), a short mixed-precision
run, and the conserved extended energy of a longer mixed-precision run."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import frac_diff, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def gpu_nhc(hb, precision, calls, n, dt, tau, kT):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    kTd = torch.as_tensor(kT, dtype=torch.float64, device="cuda")
    st = torch.zeros((hb.n_systems, 6), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    KE = torch.zeros_like(E)
    out = []
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for c in range(calls):
            b.md_step(s, n, dt, kind=ts.TS_NVT_NHC, kT=kTd, tau=tau, nhc=st, E=E, KE=KE, stream=stream)
            b.poll(stream)
            stream.synchronize()
            out.append((E.cpu().numpy().copy(), KE.cpu().numpy().copy(), st.cpu().numpy().copy()))
    res = s.pos.cpu().numpy(), s.vel.cpu().numpy(), out
    b.close()
    return res


def extended_energy(E, K, st, kT, tau, n_atoms):
    nf = np.maximum(3.0 * n_atoms - 3.0, 1.0)
    q1, qk = nf * kT * tau * tau, kT * tau * tau
    return (K + E + 0.5 * q1 * st[:, 3] ** 2 + nf * kT * st[:, 0]
            + 0.5 * qk * (st[:, 4] ** 2 + st[:, 5] ** 2) + kT * (st[:, 1] + st[:, 2]))


def test_nhc_fp64_matches_oracle(orc):
    hb = small_mix(101, n_systems=6, lo=32, hi=300)
    dt, tau = hb.meta["dt"], 100.0 / W.T0_FS
    kT = W.KB_EV * np.linspace(200.0, 400.0, hb.n_systems)     # each system its own temperature
    x, v, out = gpu_nhc(hb, 1, 2, 20, dt, tau, kT)
    xr, vr, Er, Kr, str_, _ = orc.md_nhc(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots,
                                        dt, 40, kT, tau, use_cells=True)
    assert np.abs(frac_diff(x, xr, hb.cell, hb.offsets)).max() < 1e-9
    assert np.abs(v - vr).max() < 1e-10
    E, K, st = out[-1]
    assert np.allclose(E, Er, rtol=1e-9, atol=1e-12) and np.allclose(K, Kr, rtol=1e-9)
    assert np.abs(st - str_).max() <= 1e-9 * max(np.abs(str_).max(), 1e-12)


def test_nhc_mixed_short_run(orc):
    hb = small_mix(102, n_systems=6, lo=32, hi=300)
    dt, tau = hb.meta["dt"], 100.0 / W.T0_FS
    kT = np.full(hb.n_systems, W.KB_EV * 300.0)
    x, v, out = gpu_nhc(hb, 0, 1, 5, dt, tau, kT)
    xr, vr, Er, Kr, str_, _ = orc.md_nhc(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots,
                                        dt, 5, kT, tau, use_cells=True)
    assert np.abs(frac_diff(x, xr, hb.cell, hb.offsets)).max() < 1e-6
    assert np.abs(v - vr).max() < 1e-5 * np.abs(vr).max()
    E, K, st = out[-1]
    assert np.all(np.abs(E - Er) <= 1e-6 * np.abs(Er) + 1e-6)
    assert np.allclose(K, Kr, rtol=1e-5)
    assert np.abs(st[:, 3:] - str_[:, 3:]).max() <= 1e-4 * np.abs(str_[:, 3:]).max()


def test_nhc_mixed_extended_energy_conserved():
    hb = small_mix(103, n_systems=4, lo=64, hi=400)
    dt, tau = hb.meta["dt"], 50.0 / W.T0_FS
    kT = np.full(hb.n_systems, W.KB_EV * 600.0)                # heat from 300 K: the chain moves energy
    _, _, out = gpu_nhc(hb, 0, 20, 50, dt, tau, kT)
    n = np.diff(hb.offsets)
    H = np.array([extended_energy(E, K, st, kT, tau, n) for E, K, st in out])
    KU = np.array([E + K for E, K, _ in out])
    span = KU.max(0) - KU.min(0)
    assert np.all(span > 0.05)
    assert np.all(np.abs(H - H[0]).max(0) < 0.02 * span)

"""GPU parity of the MD integrators (velocity Verlet, BAOAB Langevin) against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import frac_diff, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def gpu_md(hb, precision, n_steps, kind, dt, gamma=0.0, seed=0, step0=0, calls=1):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    KE = torch.zeros_like(E)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for c in range(calls):
            b.md_step(s, n_steps, dt, kind=kind, gamma=gamma, seed=seed, step0=step0 + c * n_steps, E=E, KE=KE,
                      stream=stream)
        b.poll(stream)
    stream.synchronize()
    return s.pos.cpu().numpy(), s.vel.cpu().numpy(), E.cpu().numpy(), KE.cpu().numpy(), b


def test_nve_fp64_single_argon(orc):
    """The 256-atom LJ argon box, velocity Verlet at 2 fs in FP64, 100 steps."""
    hb = W.single_lj_argon(seed=0)
    dt = hb.meta["dt"]
    x, v, E, KE, _ = gpu_md(hb, 1, 50, 0, dt, calls=2)
    xr, vr, Er, KEr = orc.md(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots, dt, 100,
                             use_cells=True)
    assert np.abs(frac_diff(x, xr, hb.cell, hb.offsets)).max() < 1e-9
    assert np.abs(v - vr).max() < 1e-10
    assert E[0] == pytest.approx(Er[0], rel=1e-9)
    assert KE[0] == pytest.approx(KEr[0], rel=1e-9)


@pytest.mark.parametrize("precision", [1, 0])
def test_langevin_batched(orc, precision):
    """BAOAB on a ragged batch; FP64 mode reproduces the oracle's noise and
    trajectory; mixed mode one call of 3 steps from the same state."""
    hb = small_mix(51, n_systems=8, lo=32, hi=300)
    dt = hb.meta["dt"]
    gamma = hb.meta["gamma"]
    n = 20 if precision == 1 else 3
    x, v, E, KE, _ = gpu_md(hb, precision, n, 1, dt, gamma=gamma, seed=7, step0=100)
    xr, vr, Er, KEr = orc.md(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots, dt, n,
                             kind=1, kT=hb.kT, gamma=gamma, seed=7, uid=hb.uid, step0=100)
    dx = np.abs(frac_diff(x, xr, hb.cell, hb.offsets)).max()
    dv = np.abs(v - vr).max()
    if precision == 1:
        assert dx < 1e-9 and dv < 1e-9
        assert np.allclose(E, Er, rtol=1e-9, atol=1e-12) and np.allclose(KE, KEr, rtol=1e-9)
    else:
        vs = np.abs(vr).max()
        assert dx < 1e-6 and dv < 1e-5 * vs
        assert np.all(np.abs(E - Er) <= 1e-6 * np.abs(Er) + 1e-6)
        assert np.allclose(KE, KEr, rtol=1e-5)


def test_nve_mixed_energy_conservation():
    """Mixed precision keeps the NVE energy of the LJ argon box: drift over
    1000 steps within twice the oracle's FP64 drift plus the FP32 force noise."""
    hb = W.single_lj_argon(seed=0)
    dt = hb.meta["dt"]
    x, v, E0, K0, b = gpu_md(hb, 0, 1, 0, dt)
    hb2 = W.single_lj_argon(seed=0)
    x1, v1, E1, K1, _ = gpu_md(hb2, 0, 1000, 0, dt)
    drift = abs((E1[0] + K1[0]) - (E0[0] + K0[0])) / hb.n_atoms
    assert drift < 5e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_step_calls_compose(precision):
    """K steps in one call (merged half kicks, graph replay) equal K calls of
    one step (separate half kicks) up to the rounding of the kick products:
    FP32 in mixed mode, FP64 otherwise."""
    hb = small_mix(61, n_systems=4, lo=32, hi=200)
    dt = hb.meta["dt"]
    xa, va, *_ = gpu_md(hb, precision, 6, 1, dt, gamma=hb.meta["gamma"], seed=3, step0=0)
    xb, vb, *_ = gpu_md(hb, precision, 1, 1, dt, gamma=hb.meta["gamma"], seed=3, step0=0, calls=6)
    tol = 1e-12 if precision == 1 else 1e-7
    assert np.abs(frac_diff(xa, xb, hb.cell, hb.offsets)).max() < tol
    assert np.abs(va - vb).max() < tol * 10

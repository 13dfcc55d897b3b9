"""Second-order work from the pair-force adjoint: Hessian-vector products,
per-system Hessian blocks and Gamma-point phonons.

Pins: the product equals minus the oracle's adjoint with gF = v; central
differences of the GPU forces along v; symmetry <u, Hv> = <v, Hu>; a rigid
translation is a zero mode (periodic systems); the Hessian of a perfect FCC
lattice has exactly three zero (acoustic) Gamma modes and no negative ones."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def setup(hb, precision):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    b.poll()
    return torch, b, s


@pytest.mark.parametrize("precision", [0, 1])
def test_hvp_matches_oracle_adjoint(orc, precision):
    from paper_2508_06628_b300 import grad
    hb = small_mix(91, n_systems=5, lo=32, hi=300)
    torch, b, s = setup(hb, precision)
    rng = np.random.default_rng(2)
    v = rng.normal(size=(hb.n_atoms, 3))
    hv = grad.hessian_vector_product(b, s, torch.as_tensor(v, device="cuda")).cpu().numpy()
    b.poll()
    pos = s.pos.cpu().numpy()
    gx, _ = orc.forces_backward(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots, v)
    ref = -gx
    tol = 1e-9 if precision == 1 else 2e-4
    for k in range(hb.n_systems):
        a, e = hb.offsets[k], hb.offsets[k + 1]
        assert np.abs(hv[a:e] - ref[a:e]).max() <= tol * np.abs(ref[a:e]).max()
    b.close()


def test_hvp_central_differences_fp64():
    """Soft spheres only: their force goes to zero continuously at the cutoff,
    while the energy-shifted LJ and Morse forces jump there, which a pair
    within eps of rc would turn into a spurious difference quotient."""
    from paper_2508_06628_b300 import grad
    mix = small_mix(92, n_systems=12, lo=32, hi=200)
    hb = mix.subset([k for k in range(mix.n_systems) if mix.pots[mix.pot_idx[k]]["kind"] == 2])
    assert hb.n_systems >= 2
    torch, b, s = setup(hb, 1)
    rng = np.random.default_rng(3)
    v = torch.as_tensor(rng.normal(size=(hb.n_atoms, 3)), device="cuda")
    hv = grad.hessian_vector_product(b, s, v).cpu().numpy()
    x0 = s.pos.clone()
    F = {}
    eps = 1e-5
    for sign in (1, -1):
        s.pos.copy_(x0 + sign * eps * v)
        f = torch.zeros_like(s.pos)
        b.pair_forces(s, f, None, None)
        b.poll()
        F[sign] = f.cpu().numpy()
    fd = -(F[1] - F[-1]) / (2 * eps)                 # -dF/dx v = H v
    assert np.abs(fd - hv).max() <= 1e-5 * np.abs(hv).max()
    b.close()


def test_hvp_symmetry_and_translation_fp64():
    from paper_2508_06628_b300 import grad
    hb = small_mix(93, n_systems=4, lo=32, hi=200)
    torch, b, s = setup(hb, 1)
    rng = np.random.default_rng(4)
    u = torch.as_tensor(rng.normal(size=(hb.n_atoms, 3)), device="cuda")
    v = torch.as_tensor(rng.normal(size=(hb.n_atoms, 3)), device="cuda")
    hu = grad.hessian_vector_product(b, s, u)
    hv = grad.hessian_vector_product(b, s, v)
    off = hb.offsets
    for k in range(hb.n_systems):
        a, e = off[k], off[k + 1]
        uhv = float((u[a:e] * hv[a:e]).sum())
        vhu = float((v[a:e] * hu[a:e]).sum())
        assert abs(uhv - vhu) <= 1e-10 * max(abs(uhv), 1.0)
    t = torch.zeros_like(s.pos)
    t[:, 0] = 1.0                                    # rigid translation of every system along x
    ht = grad.hessian_vector_product(b, s, t).cpu().numpy()
    assert np.abs(ht).max() <= 1e-9 * np.abs(hv.cpu().numpy()).max()
    b.close()


def test_gamma_phonons_perfect_fcc():
    from paper_2508_06628_b300 import grad
    p, c = W.lattice("fcc", (2, 2, 2), 5.26)         # argon, 32 atoms, no rattle: every atom at a centre of symmetry
    ref = small_mix(1, n_systems=3)
    sysd = dict(pos=p, vel=np.zeros_like(p), mass=np.full(len(p), 39.948), cell=c, pot=0)
    hb = W.concat([sysd], ref.pots)
    torch, b, s = setup(hb, 1)
    blocks = grad.hessian_blocks(b, s)
    assert len(blocks) == 1 and blocks[0].shape == (96, 96)
    H = blocks[0]
    assert np.abs(H - H.T).max() <= 1e-10 * np.abs(H).max()
    w = grad.gamma_frequencies(H, hb.mass)
    lam = np.sort(np.sign(w) * w * w)
    scale = lam[-1]
    assert np.all(np.abs(lam[:3]) <= 1e-9 * scale)    # the three acoustic modes
    assert lam[3] > 1e-3 * scale                     # every other Gamma mode is stable
    b.close()

"""Pins of the FP64 oracle's potentials, neighbour sets, forces and stress.

Each check is independent of the oracle's own code path: closed forms of the
dimers, textbook FCC lattice sums, brute-force enumerations written here in
numpy, central finite differences, PyTorch FP64 autograd of an energy written
here, and symmetry invariants.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")

LJ = dict(kind=0, p=(3.405, 0.0104, 0.0), rc=8.5125, shift=0)
MO = dict(kind=1, p=(0.3429, 1.3588, 2.866), rc=6.0, shift=0)
SS = dict(kind=2, p=(1.0, 1.0, 2.0), rc=1.0, shift=0)


def dimer(orc, pot, r, L=60.0):
    x = np.array([[0.0, 0, 0], [r, 0, 0]])
    cell = np.eye(3)[None] * L
    E, F, S = orc.forces([0, 2], x, cell, [[1, 1, 1]], [0], [pot])
    return E[0], F


def test_lj_dimer_minimum(orc):
    rm = 2 ** (1 / 6) * 3.405
    E, F = dimer(orc, LJ, rm)
    assert E == pytest.approx(-0.0104, rel=1e-13)
    assert np.abs(F).max() < 1e-15
    # shifted: the same minimum lowered by -phi(rc)
    s = 3.405 / 8.5125
    phic = 4 * 0.0104 * (s ** 12 - s ** 6)
    Es, _ = dimer(orc, dict(LJ, shift=1), rm)
    assert Es == pytest.approx(-0.0104 - phic, rel=1e-13)
    # zero of the potential at r = sigma and the repulsive side pushes apart
    E0, F0 = dimer(orc, LJ, 3.405)
    assert abs(E0) < 1e-16 and F0[0, 0] < 0 < F0[1, 0]


def test_morse_dimer_minimum(orc):
    E, F = dimer(orc, MO, 2.866)
    assert E == pytest.approx(-0.3429, rel=1e-13)
    assert np.abs(F).max() < 1e-15
    # equals D (1 - exp(-a(r-r0)))^2 - D at another distance
    r = 3.3
    E2, _ = dimer(orc, MO, r)
    assert E2 == pytest.approx(0.3429 * (1 - np.exp(-1.3588 * (r - 2.866))) ** 2 - 0.3429, rel=1e-13)


def test_soft_sphere_values(orc):
    E, F = dimer(orc, SS, 1.0, L=10.0)
    assert E == 0.0 and np.abs(F).max() == 0.0
    E, F = dimer(orc, SS, 1.2, L=10.0)
    assert E == 0.0
    E, F = dimer(orc, SS, 1e-9, L=10.0)
    assert E == pytest.approx(0.5, rel=1e-8)          # eps/alpha at contact
    E, F = dimer(orc, SS, 0.5, L=10.0)
    assert E == pytest.approx(0.5 * 0.25, rel=1e-13)  # (eps/alpha)(1-r/sigma)^2
    assert F[1, 0] == pytest.approx(0.5, rel=1e-13)   # -(d/dr) = (eps/sigma)(1 - r/sigma)


def _fcc_vectors(a, rmax):
    """All FCC lattice vectors R != 0 with |R| < rmax (numpy enumeration)."""
    m = int(np.ceil(rmax / a)) + 1
    g = np.array(list(itertools.product(range(-m, m + 1), repeat=3)), float)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    R = (g[:, None, :] + basis[None]).reshape(-1, 3) * a
    r = np.linalg.norm(R, axis=1)
    return r[(r > 1e-12) & (r < rmax)]


def test_lj_fcc_textbook_lattice_sum(orc):
    """Infinite-range E/atom = 2 eps [A12 s^12 - A6 s^6] with textbook A12, A6;
    a large cutoff plus the continuum tail of the r^-6 term reproduces it."""
    consts = {}
    for line in open(os.path.join(GOLD, "lj_fcc_lattice_sums.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            consts[k] = float(v)
    sig, eps = 1.0, 1.0
    a = 1.5417
    rc = 9.0 * sig
    pos, cell = W.lattice("fcc", (1, 1, 1), a)
    E, F, S = orc.forces([0, 4], pos, cell[None], [[1, 1, 1]], [0], [dict(kind=0, p=(sig, eps, 0), rc=rc, shift=0)])
    rho = 4 / a ** 3
    tail = -8 * np.pi * rho * eps * sig ** 6 / (3 * rc ** 3) + 8 * np.pi * rho * eps * sig ** 12 / (9 * rc ** 9)
    rnn = a / np.sqrt(2)
    ref = 2 * eps * (consts["A12"] * (sig / rnn) ** 12 - consts["A6"] * (sig / rnn) ** 6)
    assert E[0] / 4 + tail == pytest.approx(ref, rel=2e-5)
    assert np.abs(F).max() < 1e-11


@pytest.mark.parametrize("pot,a", [(dict(LJ, shift=1), 5.26), (dict(MO, shift=1), 3.61), (SS, 1.27)])
def test_fcc_energy_vs_lattice_vector_sum(orc, pot, a):
    """Perfect FCC supercell: E/atom equals 1/2 sum_R [phi(|R|) - phi_c] over
    lattice vectors (independent numpy sum), forces vanish, stress isotropic."""
    pos, cell = W.lattice("fcc", (3, 3, 3), a)
    E, F, S = orc.forces([0, len(pos)], pos, cell[None], [[1, 1, 1]], [0], [pot])
    rc = pot["rc"]
    r = _fcc_vectors(a, rc)

    def phi(r):
        if pot["kind"] == 0:
            s, e = pot["p"][0], pot["p"][1]
            return 4 * e * ((s / r) ** 12 - (s / r) ** 6)
        if pot["kind"] == 1:
            D, al, r0 = pot["p"]
            return D * (np.exp(-2 * al * (r - r0)) - 2 * np.exp(-al * (r - r0)))
        s, e, al = pot["p"]
        return np.where(r < s, e / al * np.clip(1 - r / s, 0, None) ** al, 0.0)

    phic = phi(np.array([rc]))[0] if (pot.get("shift") and pot["kind"] != 2) else 0.0
    ref = 0.5 * np.sum(phi(r) - phic)
    assert E[0] / len(pos) == pytest.approx(ref, rel=1e-12, abs=1e-14)
    assert np.abs(F).max() < 1e-10
    assert np.allclose(S[0], np.eye(3) * S[0, 0, 0], atol=1e-12)


def _rattled(seed, pot, kind="fcc", reps=(2, 2, 3), a=5.26, rattle=0.1, strain=0.05):
    rng = np.random.default_rng(seed)
    pos, cell = W.lattice(kind, reps, a)
    e = rng.uniform(-strain, strain, (3, 3)); e = 0.5 * (e + e.T) + np.array([[0, 0.04, 0], [0, 0, 0], [0.03, 0, 0]])
    cell2 = cell @ (np.eye(3) + e)
    pos = pos @ np.linalg.solve(cell, cell2) + rng.normal(0, rattle, pos.shape)
    return pos, cell2


CASES = [(dict(LJ, shift=1), 5.26, "fcc", (2, 2, 3)),     # small cell: multi-image
         (dict(MO, shift=1), 3.61, "fcc", (2, 3, 2)),
         (dict(MO, shift=1), 2.865, "bcc", (2, 2, 2)),
         (SS, 1.03, "bcc", (3, 2, 2))]


@pytest.mark.parametrize("pot,a,kind,reps", CASES)
def test_forces_are_minus_gradient(orc, pot, a, kind, reps):
    pos, cell = _rattled(1, pot, kind, reps, a, rattle=0.03 * a)
    off = [0, len(pos)]
    E, F, S = orc.forces(off, pos, cell[None], [[1, 1, 1]], [0], [pot])
    h = 1e-5 * a
    rng = np.random.default_rng(2)
    for i in rng.choice(len(pos), 4, replace=False):
        for c in range(3):
            xp = pos.copy(); xp[i, c] += h
            xm = pos.copy(); xm[i, c] -= h
            Ep = orc.forces(off, xp, cell[None], [[1, 1, 1]], [0], [pot])[0][0]
            Em = orc.forces(off, xm, cell[None], [[1, 1, 1]], [0], [pot])[0][0]
            assert -(Ep - Em) / (2 * h) == pytest.approx(F[i, c], rel=1e-6, abs=1e-9 * max(1, np.abs(F).max()))
    # Newton's third law
    assert np.abs(F.sum(0)).max() < 1e-12 * max(1.0, np.abs(F).max() * len(pos))


@pytest.mark.parametrize("pot,a,kind,reps", CASES)
def test_stress_is_strain_derivative(orc, pot, a, kind, reps):
    """stress = (1/V) dE/d(eps) with x -> x (I + eps), h -> h (I + eps)."""
    pos, cell = _rattled(3, pot, kind, reps, a, rattle=0.03 * a)
    off = [0, len(pos)]
    E, F, S = orc.forces(off, pos, cell[None], [[1, 1, 1]], [0], [pot])
    V = abs(np.linalg.det(cell))
    d = 1e-6
    for p, q in [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2), (2, 0)]:
        e = np.zeros((3, 3)); e[p, q] = d
        Ep = orc.forces(off, pos @ (np.eye(3) + e), (cell @ (np.eye(3) + e))[None], [[1, 1, 1]], [0], [pot])[0][0]
        Em = orc.forces(off, pos @ (np.eye(3) - e), (cell @ (np.eye(3) - e))[None], [[1, 1, 1]], [0], [pot])[0][0]
        assert (Ep - Em) / (2 * d) / V == pytest.approx(S[0][p, q], rel=1e-6, abs=1e-10)
    assert np.allclose(S[0], S[0].T, atol=1e-14)


def test_autograd_fp64_energy(orc):
    """Independent derivative: PyTorch FP64 autograd of an energy written here
    (explicit image loop) gives the oracle's forces and stress."""
    torch = pytest.importorskip("torch")
    pot = dict(MO, shift=1)
    pos, cell = _rattled(4, pot, "fcc", (2, 2, 2), 3.61, rattle=0.08)
    E, F, S = orc.forces([0, len(pos)], pos, cell[None], [[1, 1, 1]], [0], [pot])
    x = torch.tensor(pos, requires_grad=True)
    strain = torch.zeros(3, 3, dtype=torch.float64, requires_grad=True)
    h = torch.tensor(cell)
    D, al, r0 = pot["p"]; rc = pot["rc"]
    phic = D * (np.exp(-2 * al * (rc - r0)) - 2 * np.exp(-al * (rc - r0)))
    M = torch.eye(3, dtype=torch.float64) + strain
    xs, hs = x @ M, h @ M
    imgs = torch.tensor(list(itertools.product(range(-2, 3), repeat=3)), dtype=torch.float64)
    Et = 0
    for n in imgs:
        d = xs[None, :, :] - xs[:, None, :] + (n @ hs)[None, None, :]
        r = torch.sqrt((d * d).sum(-1) + (1 if n.abs().sum() == 0 else 0) * torch.eye(len(pos), dtype=torch.float64))
        mask = (r < rc) & ~((n.abs().sum() == 0) & torch.eye(len(pos), dtype=torch.bool))
        e = torch.exp(-al * (r - r0))
        Et = Et + 0.5 * torch.where(mask, D * (e * e - 2 * e) - phic, torch.zeros_like(r)).sum()
    gx, gs = torch.autograd.grad(Et, (x, strain))
    assert float(Et) == pytest.approx(E[0], rel=1e-12)
    assert np.allclose(-gx.numpy(), F, atol=1e-11)
    assert np.allclose(gs.numpy() / abs(np.linalg.det(cell)), S[0], atol=1e-12)


def test_invariances_and_batch(orc):
    pot = dict(MO, shift=1)
    pos, cell = _rattled(5, pot, "fcc", (2, 3, 2), 3.61, rattle=0.1)
    off = [0, len(pos)]
    E, F, S = orc.forces(off, pos, cell[None], [[1, 1, 1]], [0], [pot])
    # translation
    E2, F2, S2 = orc.forces(off, pos + np.array([1.7, -3.2, 0.4]), cell[None], [[1, 1, 1]], [0], [pot])
    assert E2[0] == pytest.approx(E[0], rel=1e-12) and np.allclose(F2, F, atol=1e-11)
    # rotation of positions and cell together
    th = 0.7
    Rm = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    E3, F3, S3 = orc.forces(off, pos @ Rm.T, (cell @ Rm.T)[None], [[1, 1, 1]], [0], [pot])
    assert E3[0] == pytest.approx(E[0], rel=1e-12)
    assert np.allclose(F3, F @ Rm.T, atol=1e-11)
    assert np.allclose(S3[0], Rm @ S[0] @ Rm.T, atol=1e-12)
    # permutation within the system
    p = np.random.default_rng(0).permutation(len(pos))
    E4, F4, _ = orc.forces(off, pos[p], cell[None], [[1, 1, 1]], [0], [pot])
    assert E4[0] == pytest.approx(E[0], rel=1e-12) and np.allclose(F4, F[p], atol=1e-11)
    # batch invariance: same system alone and between two others
    pa, ca = _rattled(6, pot, "fcc", (2, 2, 2), 3.61)
    pb, cb = _rattled(7, dict(LJ, shift=1), "fcc", (2, 2, 2), 5.26)
    xs = np.concatenate([pa, pos, pb])
    offs = [0, len(pa), len(pa) + len(pos), len(xs)]
    Eb, Fb, Sb = orc.forces(offs, xs, np.stack([ca, cell, cb]), np.ones((3, 3)), [0, 0, 1], [pot, dict(LJ, shift=1)])
    assert Eb[1] == E[0] and np.array_equal(Fb[offs[1]:offs[2]], F) and np.array_equal(Sb[1], S[0])


def test_fcc_shell_count(orc):
    """LJ argon FCC a = 5.26 within 2.5 sigma: shells 12+6+24+12+24 = 78."""
    pos, cell = W.lattice("fcc", (4, 4, 4), 5.26)
    pairs = orc.neighbors(pos, cell, [1, 1, 1], 8.5125)
    assert len(pairs) == 78 * len(pos)
    r = np.array(sorted(set(np.round(np.linalg.norm(
        pos[pairs[:, 1]] - pos[pairs[:, 0]] + pairs[:, 2:] @ cell, axis=1), 6))))
    assert np.allclose(r, 5.26 * np.sqrt([0.5, 1, 1.5, 2, 2.5]), atol=1e-6)


def test_single_atom_images(orc):
    """One atom in a cubic box smaller than the cutoff: its neighbours are its
    own images n != 0 with |n| L < r (enumerated here directly)."""
    L, r = 2.0, 5.1
    pairs = orc.neighbors(np.array([[0.3, 0.2, 0.1]]), np.eye(3) * L, [1, 1, 1], r)
    m = 4
    ref = {n for n in itertools.product(range(-m, m + 1), repeat=3) if 0 < np.linalg.norm(n) * L < r}
    got = {tuple(p[2:]) for p in pairs}
    assert got == ref and all(p[0] == 0 and p[1] == 0 for p in pairs)


@pytest.mark.parametrize("seed,kind,reps,a,r", [(0, "fcc", (2, 2, 4), 5.26, 9.5), (1, "bcc", (2, 2, 4), 4.175, 9.5),
                                                (2, "fcc", (5, 4, 3), 3.61, 6.5), (3, "fcc", (1, 1, 1), 1.27, 1.3)])
def test_cell_list_equals_brute_force(orc, seed, kind, reps, a, r):
    pos, cell = _rattled(seed, None, kind, reps, a, rattle=0.05 * a)
    pos = pos + np.random.default_rng(seed).uniform(-3, 3, 3) * a   # some atoms outside the box
    b = orc.neighbors(pos, cell, [1, 1, 1], r)
    c = orc.neighbors(pos, cell, [1, 1, 1], r, use_cells=True)

    def key(P):
        d = pos[P[:, 1]] - pos[P[:, 0]] + P[:, 2:] @ cell
        rr = np.linalg.norm(d, axis=1)
        keep = np.abs(rr - r) > 1e-6
        return set(map(tuple, P[keep]))

    assert key(b) == key(c) and len(key(b)) > 0


def test_nonperiodic_axis(orc):
    """A slab periodic in x, y only: no images along z (explicit check)."""
    pos, cell = _rattled(8, None, "fcc", (3, 3, 2), 3.61, rattle=0.05)
    pairs = orc.neighbors(pos, cell, [1, 1, 0], 6.0)
    assert np.all(pairs[:, 4] == 0)
    full = orc.neighbors(pos, cell, [1, 1, 1], 6.0)
    assert len(full) > len(pairs)

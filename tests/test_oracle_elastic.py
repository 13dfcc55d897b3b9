"""Pins of the oracle's stress-strain coefficients (elastic constants; the
paper lists them among the properties to come, Sec. 5) against results that
do not go through the oracle's forces:

* a perfect FCC crystal of a central pair potential at zero pressure obeys
  the Cauchy relation C12 = C44, has cubic symmetry and no normal-shear
  coupling;
* C11 and C12 equal the Born lattice sums (1/2 Omega) sum_R (phi'' -
  phi'/R) R_a R_b R_c R_d / R^2, written out here with numpy;
* the bulk modulus (C11 + 2 C12)/3 equals V d^2E/dV^2 of an energy-volume
  curve of the same crystal (a second route to the same curvature).
The zero-pressure lattice constant is found here from the lattice sum
sum_R phi'(R) R = 0 (no oracle call)."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W

LJ = dict(kind=0, p=(1.0, 1.0, 0.0), rc=2.5, shift=1)
MORSE = dict(W.MORSE_CU)


def _dphi(pot, r):
    """phi'(r), phi''(r) written out from the potentials' textbook forms."""
    if pot["kind"] == 0:
        s, e = pot["p"][0], pot["p"][1]
        x6 = (s / r) ** 6
        return -24 * e / r * (2 * x6 * x6 - x6), 24 * e / r ** 2 * (26 * x6 * x6 - 7 * x6)
    D, al, r0 = pot["p"]
    ex = np.exp(-al * (r - r0))
    return 2 * al * D * (ex - ex * ex), 2 * al * al * D * (2 * ex * ex - ex)


def _fcc_vectors(a, rc, reach=6):
    """Lattice vectors of FCC (conventional constant a) shorter than rc."""
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(-reach, reach + 1)
    cells = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T
    R = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    r = np.linalg.norm(R, axis=1)
    return R[(r > 1e-12) & (r < rc)]


def _zero_pressure_a(pot, a0):
    """The conventional lattice constant where sum_R phi'(R) R = 0 (bisection)."""
    def pressure_sum(a):
        R = _fcc_vectors(a, pot["rc"])
        r = np.linalg.norm(R, axis=1)
        return np.sum(_dphi(pot, r)[0] * r)
    lo, hi = a0 * 0.97, a0 * 1.03
    assert pressure_sum(lo) * pressure_sum(hi) < 0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if pressure_sum(lo) * pressure_sum(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def _born(pot, a):
    """C11, C12 (= C44) from the Born lattice sums at zero stress."""
    R = _fcc_vectors(a, pot["rc"])
    r = np.linalg.norm(R, axis=1)
    d1, d2 = _dphi(pot, r)
    w = (d2 - d1 / r) / r ** 2
    omega = a ** 3 / 4
    return (np.sum(w * R[:, 0] ** 4) / (2 * omega), np.sum(w * R[:, 0] ** 2 * R[:, 1] ** 2) / (2 * omega))


@pytest.mark.parametrize("pot,a0", [(LJ, 1.5496), (MORSE, 3.6616)])
def test_fcc_elastic_constants(orc, pot, a0):
    a = _zero_pressure_a(pot, a0)
    pos, cell = W.lattice("fcc", (4, 4, 4), a)
    off = np.array([0, len(pos)])
    C = orc.elastic_constants(off, pos, cell[None], np.ones((1, 3), np.uint8), [0], [pot], delta=1e-5)[0]
    C11, C12 = _born(pot, a)
    scale = abs(C11)
    assert C[0, 0] == pytest.approx(C11, rel=1e-6)
    assert C[0, 1] == pytest.approx(C12, rel=1e-6)
    assert C[3, 3] == pytest.approx(C12, rel=1e-6)          # Cauchy: C44 = C12 for central forces at zero stress
    assert np.allclose(np.diag(C)[:3], C[0, 0], rtol=1e-7)
    assert np.allclose(np.diag(C)[3:], C[3, 3], rtol=1e-7)
    assert np.allclose(C, C.T, atol=1e-7 * scale)
    assert np.abs(C[:3, 3:]).max() < 1e-7 * scale and np.abs(C[3:, 3:] - np.diag(np.diag(C)[3:])).max() < 1e-7 * scale
    # bulk modulus from the curvature of E(V) of the same crystal
    n = len(pos)
    V0 = np.linalg.det(cell)
    h = 1e-4
    E = []
    for f in (1 - h, 1.0, 1 + h):
        e, _, _ = orc.forces(off, pos * f ** (1 / 3), (cell * f ** (1 / 3))[None], np.ones((1, 3), np.uint8), [0], [pot])
        E.append(e[0])
    d2E = (E[0] - 2 * E[1] + E[2]) / (h * V0) ** 2
    assert (C[0, 0] + 2 * C[0, 1]) / 3 == pytest.approx(V0 * d2E, rel=1e-4)
    assert n == 256

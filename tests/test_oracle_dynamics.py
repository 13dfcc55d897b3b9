"""Pins of the FP64 oracle's integrators, RNG, FIRE, adjoint and RDF."""
import os

import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MO = dict(W.MORSE_CU)
LJR = dict(W.LJ_REDUCED)


def test_philox_known_answers(orc):
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        out = orc.philox4x32_10(w[0:4], w[4:6])
        assert list(out) == w[6:10]


def test_normals_statistics(orc):
    z = np.array([orc.normals3(s, i, 7, 3) for s in range(200) for i in range(100)]).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 6 * np.sqrt(2 / z.size)
    # a different key gives different numbers, the same counter the same numbers
    assert not np.allclose(orc.normals3(5, 1, 7, 3), orc.normals3(5, 1, 7, 4))
    assert np.array_equal(orc.normals3(5, 1, 7, 3), orc.normals3(5, 1, 7, 3))


def _small_batch(seed=0):
    b = W.ragged_mix(seed=seed, n_systems=3, lo=32, hi=108)
    return b


def test_velocity_verlet_time_reversible(orc):
    b = _small_batch()
    dt = 1.0 / W.T0_FS
    x1, v1, E1, K1 = orc.md(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 200)
    x2, v2, E2, K2 = orc.md(b.offsets, x1, -v1, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 200)
    assert np.abs(x2 - b.pos).max() < 1e-9
    assert np.abs(v2 + b.vel).max() < 1e-9


def test_velocity_verlet_energy_conservation(orc):
    b = W.single_lj_argon(seed=0)
    dt = b.meta["dt"]
    E0 = orc.forces(b.offsets, b.pos, b.cell, b.pbc, b.pot_idx, b.pots)[0]
    K0 = 0.5 * (b.mass[:, None] * b.vel ** 2).sum()
    x, v, E, K = orc.md(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 200)
    drift = abs(E[0] + K[0] - E0[0] - K0) / len(b.pos)
    assert drift < 2e-6   # eV/atom over 200 steps of 2 fs (fluctuation of a 2nd-order scheme)
    assert K[0] > 0


def test_baoab_without_friction_is_velocity_verlet(orc):
    b = _small_batch(1)
    dt = 1.0 / W.T0_FS
    xa, va, Ea, Ka = orc.md(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 50)
    xb, vb, Eb, Kb = orc.md(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 50, kind=1,
                            kT=b.kT, gamma=0.0, seed=3, uid=b.uid)
    assert np.abs(xa - xb).max() < 1e-11 and np.abs(va - vb).max() < 1e-11


@pytest.mark.slow
def test_baoab_equipartition(orc):
    """Langevin on every atom thermalises all 3N degrees of freedom:
    <KE> = 3N/2 kT within 4 standard errors of the time average."""
    b = W.single_lj_argon(seed=1, T=80.0)
    kT = W.KB_EV * 120.0
    dt = 2.0 / W.T0_FS
    gamma = 0.05 * W.T0_FS
    x, v = b.pos, b.vel
    x, v, E, K = orc.md(b.offsets, x, v, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 300, kind=1,
                        kT=[kT], gamma=gamma, seed=11, uid=[0], step0=0)
    ks = []
    for blk in range(60):
        x, v, E, K = orc.md(b.offsets, x, v, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 20, kind=1,
                            kT=[kT], gamma=gamma, seed=11, uid=[0], step0=300 + 20 * blk)
        ks.append(K[0])
    ks = np.array(ks)
    target = 1.5 * len(b.pos) * kT
    se = ks.std(ddof=1) / np.sqrt(len(ks) / 2)   # blocks are correlated over ~2 samples
    assert abs(ks.mean() - target) < 4 * se + 1e-12


def test_nhc_conserved_quantity(orc):
    """NVT Nose-Hoover chain, argon heated from 50 K by a 120 K chain: K + U
    changes by electron-volts while the extended energy stays put."""
    b = W.single_lj_argon(seed=2, T=50.0)
    kT, tau, dt = W.KB_EV * 120.0, 200.0 / W.T0_FS, 2.0 / W.T0_FS
    x, v, st = b.pos, b.vel, None
    H, KU = [], []
    for blk in range(10):
        x, v, E, K, st, He = orc.md_nhc(b.offsets, x, v, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 50, [kT], tau,
                                       nhc=st)
        H.append(He[0]); KU.append(E[0] + K[0])
    H, KU = np.array(H), np.array(KU)
    assert KU.max() - KU.min() > 0.5                         # the chain moved real energy
    assert np.abs(H - H[0]).max() < 2e-3 * (KU.max() - KU.min())


def test_nhc_inert_chain_is_velocity_verlet(orc):
    """With enormous thermostat masses the chain does nothing: velocity Verlet."""
    b = W.single_lj_argon(seed=0)
    dt = 2.0 / W.T0_FS
    xa, va, Ea, Ka, st, _ = orc.md_nhc(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 100,
                                       [W.KB_EV * 50.0], 1e9)
    xb, vb, Eb, Kb = orc.md(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 100)
    assert np.abs(xa - xb).max() < 1e-10 and np.abs(va - vb).max() < 1e-10
    assert np.abs(st[0, 3:]).max() < 1e-12


def test_nhc_time_reversible(orc):
    """Reversing the atom and chain velocities retraces the trajectory (the
    factorisation is symmetric)."""
    b = W.single_lj_argon(seed=3, T=60.0)
    kT, tau, dt = W.KB_EV * 90.0, 100.0 / W.T0_FS, 2.0 / W.T0_FS
    st0 = np.array([[0.0, 0.0, 0.0, 0.01, -0.02, 0.005]])
    # 60 steps: long enough to exercise the chain, short enough that chaotic
    # growth of rounding errors stays far below the tolerance
    x1, v1, _, _, st1, _ = orc.md_nhc(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 60,
                                      [kT], tau, nhc=st0)
    back = st1.copy(); back[:, 3:] *= -1
    x2, v2, _, _, st2, _ = orc.md_nhc(b.offsets, x1, -v1, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 60,
                                      [kT], tau, nhc=back)
    assert np.abs(x2 - b.pos).max() < 1e-10
    assert np.abs(v2 + b.vel).max() < 1e-10
    assert np.abs(st2[:, 3:] + st0[:, 3:]).max() < 1e-10       # chain velocities reversed
    assert np.abs(st2[:, :3] - st0[:, :3]).max() < 1e-10       # chain positions back


def test_nhc_canonical_kinetic_energy(orc):
    """A reduced-unit LJ liquid under the chain: <K> = Nf kT / 2 (Nf = 3N - 3)
    within 4 standard errors of block averages."""
    b = W.lj_liquid(seed=5, n_systems=1, reps=(3, 3, 3), kT=1.0, rattle=0.05)
    kT, tau, dt = 1.0, 0.5, 0.005
    x, v, E, K, st, _ = orc.md_nhc(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 4000,
                                   [kT], tau)
    ks = []
    for blk in range(40):
        x, v, E, K, st, _ = orc.md_nhc(b.offsets, x, v, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 250, [kT], tau,
                                       nhc=st)
        ks.append(K[0])
    ks = np.array(ks)
    target = 0.5 * (3 * len(b.pos) - 3) * kT
    se = ks.std(ddof=1) / np.sqrt(len(ks) / 2)
    assert abs(ks.mean() - target) < 4 * se


def test_npt_nph_conserved_quantity(orc):
    """NPT without friction (the MTK equations alone): the piston trades real
    energy with the atoms (K + U moves by several epsilon, the volume by over
    ten per cent) while K + U + W v_e^2/2 + P_ext V stays put.  A wrong sign
    of the virial or a wrong P V term breaks this by orders of magnitude."""
    b = W.lj_liquid(seed=5, n_systems=1, reps=(2, 2, 2), kT=1.0, rattle=0.05)
    V0 = abs(np.linalg.det(b.cell[0]))
    for p_ext in (0.0, 1.0):
        x, v, h, ve = b.pos, b.vel, b.cell, None
        H, KU, V = [], [], []
        for blk in range(40):
            x, v, h, ve, E, K, He, _ = orc.md_npt(b.offsets, x, v, b.mass, h, b.pbc, b.pot_idx, b.pots, 0.005, 50,
                                                 [1.0], 0.0, 0.5, p_ext, baro=ve)
            H.append(He[0]); KU.append(E[0] + K[0]); V.append(abs(np.linalg.det(h[0])))
        H, KU, V = np.array(H), np.array(KU), np.array(V)
        assert KU.max() - KU.min() > 2.0 and V.max() - V.min() > 0.1 * V0
        assert np.abs(H - H[0]).max() < 0.03 * (KU.max() - KU.min())


def test_npt_time_reversible(orc):
    """Without friction, reversing the atom and piston velocities retraces
    positions, cell and velocities (the splitting is symmetric)."""
    b = W.lj_liquid(seed=6, n_systems=1, reps=(2, 2, 2), kT=1.0, rattle=0.05)
    x1, v1, h1, ve1, _, _, _, _ = orc.md_npt(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots,
                                             0.005, 60, [1.0], 0.0, 0.5, 1.0, baro=[0.3])
    assert abs(np.linalg.det(h1[0]) / np.linalg.det(b.cell[0]) - 1) > 0.005     # the cell moved
    x2, v2, h2, ve2, _, _, _, _ = orc.md_npt(b.offsets, x1, -v1, b.mass, h1, b.pbc, b.pot_idx, b.pots,
                                             0.005, 60, [1.0], 0.0, 0.5, 1.0, baro=-ve1)
    assert np.abs(x2 - b.pos).max() < 1e-10 and np.abs(v2 + b.vel).max() < 1e-10
    assert np.abs(h2 - b.cell).max() < 1e-12 and abs(ve2[0] + 0.3) < 1e-10


def test_npt_inert_piston_is_baoab(orc):
    """An enormous piston mass keeps the cell fixed: the atoms follow BAOAB
    with the same noise."""
    b = _small_batch(4)
    dt, gamma = 1.0 / W.T0_FS, 0.01 * W.T0_FS
    kT = np.full(b.n_systems, W.KB_EV * 300.0)
    xa, va, ha, _, Ea, Ka, _, _ = orc.md_npt(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots,
                                             dt, 80, kT, gamma, 1e15, 0.0, seed=9, uid=[5, 6, 7], step0=40)
    xb, vb, Eb, Kb = orc.md(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, b.pot_idx, b.pots, dt, 80, kind=1,
                            kT=kT, gamma=gamma, seed=9, uid=[5, 6, 7], step0=40)
    assert np.abs(ha - b.cell).max() < 1e-12
    assert np.abs(xa - xb).max() < 1e-9 and np.abs(va - vb).max() < 1e-9
    assert np.allclose(Ea, Eb, rtol=1e-9, atol=1e-12)


def test_npt_ideal_gas_volume(orc):
    """Four non-interacting atoms (epsilon = 0) at kT = P_ext = 1: the NPT
    volume distribution is V^N exp(-P V / kT), so <V> = (N + 1) kT / P_ext = 5.
    The MTK coupling factor 1 + 3/Nf is what gives the V^N; with the factor 1
    the mean falls to N kT / P = 4."""
    pos, cell = W.lattice("fcc", (1, 1, 1), 1.6)
    pot = dict(kind=0, p=[1.0, 0.0, 0.0], rc=2.5, shift=1)
    vel = np.random.default_rng(1).normal(size=pos.shape)
    x, v, h, ve = pos, vel, cell[None], None
    V = []
    for blk in range(2000):
        x, v, h, ve, _, _, _, _ = orc.md_npt([0, 4], x, v, np.ones(4), h, [[1, 1, 1]], [0], [pot], 0.005, 100,
                                             [1.0], 1.0, 0.5, 1.0, seed=3, step0=100 * blk, baro=ve)
        V.append(abs(np.linalg.det(h[0])))
    V = np.array(V[20:])
    blocks = V.reshape(-1, 20).mean(1)                       # 99 blocks of 2000 steps, far beyond the correlation time
    se = blocks.std(ddof=1) / np.sqrt(len(blocks))
    assert abs(V.mean() - 5.0) < 4 * se and se < 0.15


def _golden_section(f, a, b, tol=1e-9):
    g = (np.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    while abs(b - a) > tol:
        if f(c) < f(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


def _fcc_energy_per_atom_numpy(pot, a):
    """1/2 sum over FCC lattice vectors of the shifted pair energy (numpy)."""
    import itertools
    rc = pot["rc"]
    m = int(np.ceil(rc / a)) + 1
    g = np.array(list(itertools.product(range(-m, m + 1), repeat=3)), float)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    r = np.linalg.norm((g[:, None, :] + basis[None]).reshape(-1, 3) * a, axis=1)
    r = r[(r > 1e-12) & (r < rc)]
    if pot["kind"] == 1:
        D, al, r0 = pot["p"]
        f = lambda r: D * (np.exp(-2 * al * (r - r0)) - 2 * np.exp(-al * (r - r0)))
    else:
        s, e = pot["p"][:2]
        f = lambda r: 4 * e * ((s / r) ** 12 - (s / r) ** 6)
    return 0.5 * np.sum(f(r) - f(rc))


@pytest.mark.parametrize("pot,a0,astar_lattice_sum", [(MO, 3.61, 3.661615), (LJR, 1.55, 1.549603)])
def test_fire_reaches_fcc_lattice_constant(orc, pot, a0, astar_lattice_sum):
    """Variable-cell FIRE relaxes a rattled, scaled FCC supercell to the lattice
    constant that minimises the independent lattice-vector sum."""
    astar = _golden_section(lambda a: _fcc_energy_per_atom_numpy(pot, a), 0.9 * a0, 1.1 * a0)
    assert astar == pytest.approx(astar_lattice_sum, abs=2e-6)
    rng = np.random.default_rng(5)
    pos, cell = W.lattice("fcc", (2, 2, 2), a0 * 0.98)
    pos = pos + rng.normal(0, 0.02 * a0, pos.shape)
    fr = orc.FireRun([0, len(pos)], pos, cell[None], [[1, 1, 1]], [0], [pot], fmax=1e-6, smax=1e-8 * (1 if pot is MO else 100))
    for _ in range(20):
        E, fm, sm = fr.step(200)
        if fr.converged()[0]:
            break
    assert fr.converged()[0]
    h = fr.cells[0]
    a_fit = np.cbrt(abs(np.linalg.det(h)) / 8)
    assert a_fit == pytest.approx(astar, abs=1e-4 * (1 if pot is MO else 0.3))
    assert E[0] / len(pos) == pytest.approx(_fcc_energy_per_atom_numpy(pot, astar), abs=1e-6)
    # the relaxed cell stays cubic
    assert np.allclose(h / a_fit, 2 * np.eye(3), atol=1e-4)


@pytest.mark.parametrize("p_ext", [0.0, 2.0])
def test_npt_cold_crystal_enthalpy_minimum(orc, p_ext):
    """A perfect FCC crystal at kT = 1e-8 under friction settles at the lattice
    constant that minimises the independent lattice sum's enthalpy per atom,
    u(a) + P_ext a^3 / 4 (a light piston: tau scaled so W = (Nf + 3) kT tau^2 = 24)."""
    astar = _golden_section(lambda a: _fcc_energy_per_atom_numpy(LJR, a) + p_ext * a ** 3 / 4, 1.3, 1.8)
    if p_ext == 0.0:
        assert astar == pytest.approx(1.549603, abs=2e-6)
    pos, cell = W.lattice("fcc", (2, 2, 2), 1.50)
    x, v, h, _, _, K, _, Pi = orc.md_npt([0, 32], pos, np.zeros_like(pos), np.ones(32), cell[None], [[1, 1, 1]], [0],
                                          [LJR], 0.005, 6000, [1e-8], 1.0, 5000.0, p_ext, seed=1)
    a = np.cbrt(abs(np.linalg.det(h[0])) / 8)
    assert a == pytest.approx(astar, rel=5e-6)
    assert Pi[0] == pytest.approx(p_ext, abs=2e-3)
    assert np.allclose(h[0] / a, 2 * np.eye(3), atol=1e-9)   # isotropic scaling keeps the cube


def test_fire_fixed_cell_reduces_forces(orc):
    b = W.fire_stream(seed=9, n_systems=3)
    fr = orc.FireRun(b.offsets, b.pos, b.cell, b.pbc, b.pot_idx, b.pots, variable_cell=0, fmax=1e-4)
    E0, fm0, _ = fr.step(0)
    E1, fm1, _ = fr.step(400)
    assert np.all(E1 < E0) and np.all(fm1 < 1e-2 * fm0 + 1e-4)
    assert np.array_equal(fr.cells, b.cell)


@pytest.mark.parametrize("pi", [0, 1, 2])
def test_forces_backward_finite_differences(orc, pi):
    pots = [dict(W.LJ_AR), dict(W.MORSE_CU), dict(W.SOFT_SPHERE)]
    b = W.ragged_mix(seed=20 + pi, n_systems=2, lo=32, hi=64)
    b.pot_idx[:] = pi
    rng = np.random.default_rng(pi)
    gF = rng.normal(size=b.pos.shape)
    gE = rng.normal(size=2)
    gS = rng.normal(size=(2, 3, 3))

    def L(x, params):
        P = [dict(p, p=tuple(params[k])) for k, p in enumerate(pots)]
        E, F, S = orc.forces(b.offsets, x, b.cell, b.pbc, b.pot_idx, P)
        return (gF * F).sum() + (gE * E).sum() + (gS * S).sum()

    params = np.array([list(p["p"]) for p in pots])
    gx, gth = orc.forces_backward(b.offsets, b.pos, b.cell, b.pbc, b.pot_idx, pots, gF, gE, gS)
    h = 1e-6
    for i in rng.choice(len(b.pos), 5, replace=False):
        for c in range(3):
            xp = b.pos.copy(); xp[i, c] += h
            xm = b.pos.copy(); xm[i, c] -= h
            fd = (L(xp, params) - L(xm, params)) / (2 * h)
            assert gx[i, c] == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1, abs(gx).max()))
    for q in range(3 if pi != 0 else 2):
        hp = 1e-6 * abs(params[pi, q])
        pp = params.copy(); pp[pi, q] += hp
        pm = params.copy(); pm[pi, q] -= hp
        fd = (L(b.pos, pp) - L(b.pos, pm)) / (2 * hp)
        assert gth[pi, q] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_rdf_ideal_gas_and_coordination(orc):
    # ideal gas: g ~ 1 away from r = 0 (average over many random boxes)
    n, L = 400, 12.0
    gs = []
    for s in range(20):
        x, cell = W.random_gas(s, n, L)
        gs.append(orc.rdf([0, n], x, cell[None], [[1, 1, 1]], 5.0, K=50)[0])
    g = np.mean(gs, 0)
    assert abs(g[10:45].mean() - 1) < 0.02
    # FCC: integral of rho g 4 pi r^2 up to between the first and second shell = 12
    pos, cell = W.lattice("fcc", (4, 4, 4), 1.0)
    rmax = 0.85
    K = 170
    g = orc.rdf([0, len(pos)], pos, cell[None], [[1, 1, 1]], rmax, K=K)[0]
    D = rmax / K
    r = (np.arange(K) + 0.5) * D
    rho = (len(pos) - 1) / abs(np.linalg.det(cell))
    assert np.sum(rho * g * 4 * np.pi * r ** 2) * D == pytest.approx(12.0, rel=1e-6)


def test_rdf_backward_finite_differences(orc):
    b = W.lj_liquid(seed=1, n_systems=2, reps=(2, 2, 2), rattle=0.15)
    K, rmax = 40, 2.5
    gg = np.random.default_rng(0).normal(size=(2, K))
    g, gx = orc.rdf(b.offsets, b.pos, b.cell, b.pbc, rmax, K=K, gg=gg)
    h = 1e-6
    for i in [0, 5, 40]:
        for c in range(3):
            xp = b.pos.copy(); xp[i, c] += h
            xm = b.pos.copy(); xm[i, c] -= h
            fd = ((orc.rdf(b.offsets, xp, b.cell, b.pbc, rmax, K=K) - orc.rdf(b.offsets, xm, b.cell, b.pbc, rmax, K=K))
                  * gg).sum() / (2 * h)
            assert gx[i, c] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_trajectory_adjoint_finite_differences(orc):
    """d loss / d (sigma, eps) through 60 NVE steps with frames every 20 steps."""
    b = W.lj_liquid(seed=3, n_systems=2, reps=(2, 2, 3), rattle=0.08, kT=0.5)
    pot = dict(LJR)
    K, rmax, T, every, dt = 50, 2.5, 60, 20, 0.005
    tgt_pot = dict(pot, p=(1.05, 1.0, 0.0))
    _, target, _ = orc.traj_rdf_loss(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, tgt_pot, dt, T, every, rmax, K,
                                     np.zeros(K), grad=False)
    loss, g, gth = orc.traj_rdf_loss(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, pot, dt, T, every, rmax, K, target)
    assert loss > 0
    for q in (0, 1):
        h = 1e-6
        pp = list(pot["p"]); pp[q] += h
        pm = list(pot["p"]); pm[q] -= h
        lp = orc.traj_rdf_loss(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, dict(pot, p=tuple(pp)), dt, T, every,
                               rmax, K, target, grad=False)[0]
        lm = orc.traj_rdf_loss(b.offsets, b.pos, b.vel, b.mass, b.cell, b.pbc, dict(pot, p=tuple(pm)), dt, T, every,
                               rmax, K, target, grad=False)[0]
        # 1e-4 relative: the force jump at rc and the RDF truncation make the loss
        # piecewise smooth; the adjoint differentiates the smooth pieces only
        assert gth[q] == pytest.approx((lp - lm) / (2 * h), rel=1e-4)

"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the method's arithmetic: it only builds lattices,
draws rattles, strains and Maxwell-Boltzmann velocities with numpy
``default_rng``.  Both the CUDA path (tests, bench) and the FP64 oracle take
their inputs from here, so the two never generate inputs separately.

The paper benchmarks FCC Cu supercells of 16-864 atoms under Langevin MD
(arXiv 2508.06628, Sec. 4); these synthetic FCC/BCC supercells of LJ argon,
Morse copper and soft spheres stand in for it.  Units: Angstrom, eV, amu;
the time unit is t0 = sqrt(amu A^2 / eV) = 10.1805 fs.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

T0_FS = 10.180505710759414          # fs per internal time unit
KB_EV = 8.617333262e-5              # eV / K

POT_LJ, POT_MORSE, POT_SOFT_SPHERE = 0, 1, 2

# Potential presets (parameter triples as the C ABI takes them).
LJ_AR = dict(kind=POT_LJ, p=(3.405, 0.0104, 0.0), rc=2.5 * 3.405, shift=1)
MORSE_CU = dict(kind=POT_MORSE, p=(0.3429, 1.3588, 2.866), rc=6.0, shift=1)
SOFT_SPHERE = dict(kind=POT_SOFT_SPHERE, p=(1.0, 1.0, 2.0), rc=1.0, shift=0)
LJ_REDUCED = dict(kind=POT_LJ, p=(1.0, 1.0, 0.0), rc=2.5, shift=1)

MASS = {"Ar": 39.948, "Cu": 63.546, "SS": 1.0, "LJ": 1.0}
# lattice constants (A); BCC at the FCC atomic volume
LATTICE = {("Ar", "fcc"): 5.26, ("Ar", "bcc"): 4.175, ("Cu", "fcc"): 3.61, ("Cu", "bcc"): 2.865,
           ("SS", "fcc"): 1.27, ("SS", "bcc"): 1.03}

_FCC = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
_BCC = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])


def lattice(kind: str, reps, a: float):
    """Cubic FCC/BCC supercell: positions [N,3], cell [3,3] (rows = lattice vectors)."""
    basis = _FCC if kind == "fcc" else _BCC
    n = np.array(reps)
    g = np.stack(np.meshgrid(*[np.arange(k) for k in n], indexing="ij"), -1).reshape(-1, 3)
    frac = (g[:, None, :] + basis[None]).reshape(-1, 3) / n
    cell = np.diag(n * a).astype(np.float64)
    return frac @ cell, cell


def maxwell_boltzmann(rng, mass, kT):
    """Velocities with zero total momentum, rescaled to exactly kT with 3N-3 dof."""
    n = len(mass)
    v = rng.normal(size=(n, 3)) * np.sqrt(kT / mass)[:, None]
    v -= (mass[:, None] * v).sum(0) / mass.sum()
    ke = 0.5 * (mass[:, None] * v * v).sum()
    dof = max(3 * n - 3, 1)
    if ke > 0:
        v *= np.sqrt(0.5 * dof * kT / ke)
    return v


@dataclass
class Batch:
    """Host-side SimState: concatenated atom-wise and stacked system-wise arrays."""
    pos: np.ndarray                 # [N,3] f64
    vel: np.ndarray                 # [N,3] f64 (A / t0)
    mass: np.ndarray                # [N] f64 (amu)
    cell: np.ndarray                # [B,3,3] f64
    pbc: np.ndarray                 # [B,3] u8
    system_idx: np.ndarray          # [N] i32, non-decreasing
    pot_idx: np.ndarray             # [B] i32 index into pots
    pots: list = field(default_factory=list)
    kT: np.ndarray | None = None    # [B] f64 (eV)
    uid: np.ndarray | None = None   # [B] u32 stable system ids (RNG keys)
    meta: dict = field(default_factory=dict)

    @property
    def n_systems(self):
        return int(self.cell.shape[0])

    @property
    def n_atoms(self):
        return int(self.pos.shape[0])

    @property
    def offsets(self):
        counts = np.bincount(self.system_idx, minlength=self.n_systems)
        return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)

    def subset(self, systems):
        systems = np.asarray(systems)
        off = self.offsets
        idx = np.concatenate([np.arange(off[s], off[s + 1]) for s in systems])
        sysidx = np.concatenate([np.full(off[s + 1] - off[s], k, np.int32) for k, s in enumerate(systems)])
        return Batch(self.pos[idx].copy(), self.vel[idx].copy(), self.mass[idx].copy(), self.cell[systems].copy(),
                     self.pbc[systems].copy(), sysidx, self.pot_idx[systems].copy(), list(self.pots),
                     None if self.kT is None else self.kT[systems].copy(),
                     None if self.uid is None else self.uid[systems].copy(), dict(self.meta))


def concat(systems, pots):
    """systems: list of dicts with pos, vel, mass, cell, pot, (kT, uid)."""
    pos = np.concatenate([s["pos"] for s in systems])
    vel = np.concatenate([s["vel"] for s in systems])
    mass = np.concatenate([s["mass"] for s in systems])
    cell = np.stack([s["cell"] for s in systems])
    sysidx = np.concatenate([np.full(len(s["pos"]), k, np.int32) for k, s in enumerate(systems)])
    pot_idx = np.array([s["pot"] for s in systems], np.int32)
    kT = np.array([s.get("kT", 0.0) for s in systems])
    uid = np.array([s.get("uid", k) for k, s in enumerate(systems)], np.uint32)
    return Batch(pos, vel, mass, cell, np.ones((len(systems), 3), np.uint8), sysidx, pot_idx, list(pots), kT, uid)


def _strained(rng, cell, amp):
    e = rng.uniform(-amp, amp, (3, 3))
    e = 0.5 * (e + e.T)
    return cell @ (np.eye(3) + e)


def _reps(rng, kind, lo, hi, max_rep):
    basis = 4 if kind == "fcc" else 2
    combos = [c for c in itertools.product(range(1, max_rep + 1), repeat=3) if lo <= basis * np.prod(c) <= hi]
    return combos[rng.integers(len(combos))]


def single_lj_argon(seed=0, T=50.0):
    """One LJ argon FCC 4x4x4 cubic box (256 atoms, a = 5.26 A), MB velocities at T."""
    rng = np.random.default_rng(seed)
    pos, cell = lattice("fcc", (4, 4, 4), 5.26)
    mass = np.full(len(pos), MASS["Ar"])
    vel = maxwell_boltzmann(rng, mass, KB_EV * T)
    b = concat([dict(pos=pos, vel=vel, mass=mass, cell=cell, pot=0, kT=KB_EV * T)], [LJ_AR])
    b.meta = dict(workload="lj-argon-256", dt=2.0 / T0_FS, steps=1000)
    return b


def ragged_mix(seed=1, n_systems=512, lo=32, hi=2048, T=300.0, rattle=0.05, strain=0.05):
    """Ragged batch: FCC/BCC supercells of n x m x k (32-2048 atoms), each system
    LJ argon, Morse copper or soft sphere with probability 1/3, Gaussian rattle,
    random symmetric strain of the cubic cell, MB velocities at T."""
    rng = np.random.default_rng(seed)
    pots = [LJ_AR, MORSE_CU, SOFT_SPHERE]
    species = ["Ar", "Cu", "SS"]
    systems = []
    for s in range(n_systems):
        p = int(rng.integers(3))
        kind = "fcc" if rng.random() < 0.5 else "bcc"
        reps = _reps(rng, kind, lo, hi, 8 if kind == "fcc" else 10)
        pos, cell = lattice(kind, reps, LATTICE[(species[p], kind)])
        cell2 = _strained(rng, cell, strain)
        pos = pos @ np.linalg.solve(cell, cell2)        # carry the strain to the atoms
        pos = pos + rng.normal(0.0, rattle, pos.shape)
        mass = np.full(len(pos), MASS[species[p]])
        vel = maxwell_boltzmann(rng, mass, KB_EV * T)
        systems.append(dict(pos=pos, vel=vel, mass=mass, cell=cell2, pot=p, kT=KB_EV * T, uid=s))
    b = concat(systems, pots)
    b.meta = dict(workload=f"ragged-mix-{n_systems}", dt=1.0 / T0_FS, gamma=0.01 * T0_FS, steps=5000)
    return b


def fire_stream(seed=2, n_systems=8192, lo=64, hi=864, rattle=0.1, scale=(0.97, 1.03)):
    """Stream of Morse Cu FCC supercells (64-864 atoms), rattled, isotropically scaled."""
    rng = np.random.default_rng(seed)
    systems = []
    for s in range(n_systems):
        reps = _reps(rng, "fcc", lo, hi, 6)
        pos, cell = lattice("fcc", reps, 3.61 * rng.uniform(*scale))
        pos = pos + rng.normal(0.0, rattle, pos.shape)
        mass = np.full(len(pos), MASS["Cu"])
        systems.append(dict(pos=pos, vel=np.zeros_like(pos), mass=mass, cell=cell, pot=0, uid=s))
    b = concat(systems, [MORSE_CU])
    b.meta = dict(workload=f"fire-stream-{n_systems}")
    return b


def lj_liquid(seed=3, n_systems=64, reps=(6, 6, 6), rho=0.8, kT=1.0, rattle=0.0):
    """LJ in reduced units (sigma = eps = m = 1): FCC at density rho with MB
    velocities at kT.  The liquid state is reached by a Langevin pre-run done
    by the caller (either side) on this input."""
    rng = np.random.default_rng(seed)
    a = (4.0 / rho) ** (1.0 / 3.0)
    systems = []
    for s in range(n_systems):
        pos, cell = lattice("fcc", reps, a)
        if rattle:
            pos = pos + rng.normal(0.0, rattle, pos.shape)
        mass = np.ones(len(pos))
        vel = maxwell_boltzmann(rng, mass, kT)
        systems.append(dict(pos=pos, vel=vel, mass=mass, cell=cell, pot=0, kT=kT, uid=s))
    b = concat(systems, [LJ_REDUCED])
    b.meta = dict(workload=f"lj-liquid-{n_systems}x{len(systems[0]['pos'])}", dt=0.005)
    return b


def random_gas(seed, n, L):
    """Uniform random points in a cubic box (ideal gas) for RDF checks."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, (n, 3)), np.diag([L, L, L]).astype(np.float64)

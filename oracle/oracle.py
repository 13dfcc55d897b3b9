"""ctypes shim over the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports this module.

All arrays are numpy; atom-wise arrays are concatenated over systems and
delimited by ``offsets`` (length B+1), system-wise arrays are stacked, as in
TorchSim's SimState (arXiv 2508.06628, Sec. 3).  Cells are [B,3,3] with rows
= lattice vectors.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

POT_LJ, POT_MORSE, POT_SOFT_SPHERE = 0, 1, 2


class OrPot(C.Structure):
    _fields_ = [("kind", C.c_int32), ("shift", C.c_int32), ("p", C.c_double * 3), ("rc", C.c_double)]


class OrFireSys(C.Structure):
    _fields_ = [("dt", C.c_double), ("alpha", C.c_double), ("npos", C.c_int32), ("started", C.c_int32),
                ("converged", C.c_int32), ("nsteps", C.c_int32), ("Fd", C.c_double * 9), ("h0", C.c_double * 9)]


class OrFireParams(C.Structure):
    _fields_ = [("dt_max", C.c_double), ("finc", C.c_double), ("fdec", C.c_double), ("alpha0", C.c_double),
                ("falpha", C.c_double), ("maxstep", C.c_double), ("fmax", C.c_double), ("smax", C.c_double),
                ("p_ext", C.c_double), ("nmin", C.c_int32), ("variable_cell", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.c_void_p
        L.or_neighbors.restype = C.c_int64
        L.or_neighbors.argtypes = [C.c_int, P, P, P, C.c_double, C.c_int, P, C.c_int64]
        L.or_forces.restype = None
        L.or_forces.argtypes = [C.c_int, P, P, P, P, P, P, C.c_int, P, P, P, P]
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_normals3.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, P]
        L.or_md.argtypes = [C.c_int, P, P, P, P, P, P, P, P, C.c_int, C.c_int, C.c_double, C.c_int, P,
                            C.c_double, C.c_uint32, P, C.c_uint64, P, P]
        L.or_md_nhc.argtypes = [C.c_int, P, P, P, P, P, P, P, P, C.c_int, C.c_double, C.c_int, P, C.c_double, P, P,
                                P, P]
        L.or_md_npt.argtypes = [C.c_int, P, P, P, P, P, P, P, P, C.c_int, C.c_double, C.c_int, P, C.c_double,
                                C.c_double, C.c_double, C.c_uint32, P, C.c_uint64, P, P, P, P, P]
        L.or_fire.argtypes = [C.c_int, P, P, P, P, P, P, C.c_int, P, P, P, C.c_int, P, P, P]
        L.or_forces_backward.argtypes = [C.c_int, P, P, P, P, P, P, C.c_int, C.c_int, P, P, P, P, P]
        L.or_rdf.argtypes = [C.c_int, P, P, P, P, C.c_double, C.c_int, C.c_int, P, P, P]
        L.or_traj_rdf_loss.restype = C.c_double
        L.or_traj_rdf_loss.argtypes = [C.c_int, P, P, P, P, P, P, P, C.c_int, C.c_double, C.c_int, C.c_int,
                                       C.c_double, C.c_int, P, P, P]
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_pots(pots):
    """pots: list of dicts {kind, p:(3,), rc, shift} -> ctypes array."""
    arr = (OrPot * len(pots))()
    for k, d in enumerate(pots):
        arr[k].kind = int(d["kind"])
        arr[k].shift = int(d.get("shift", 1))
        p = list(d["p"]) + [0.0] * (3 - len(d["p"]))
        for q in range(3):
            arr[k].p[q] = float(p[q])
        arr[k].rc = float(d["rc"])
    return arr


def num_threads() -> int:
    return int(lib().or_num_threads())


def neighbors(x, cell, pbc, rmax, use_cells=False):
    """Neighbour triples (i, j, n0, n1, n2) of ONE system within rmax (definition:
    multi-image brute force, or the cell-list enumeration of the same set)."""
    x = _f64(x); cell = _f64(cell).reshape(3, 3)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8)
    n = x.shape[0]
    cnt = lib().or_neighbors(n, _p(x), _p(cell), _p(pbc), float(rmax), int(use_cells), None, 0)
    out = np.zeros((max(cnt, 1), 5), np.int32)
    lib().or_neighbors(n, _p(x), _p(cell), _p(pbc), float(rmax), int(use_cells), _p(out), cnt)
    return out[:cnt]


def forces(offsets, x, cells, pbc, pot_of_sys, pots, use_cells=False, per_atom_energy=False):
    """E [B], F [N,3], stress [B,3,3] (and per-atom energies if asked)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    x = _f64(x); cells = _f64(cells)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(B, 3)
    pos = np.ascontiguousarray(pot_of_sys, dtype=np.int32)
    P = make_pots(pots)
    E = np.zeros(B); F = np.zeros_like(x); S = np.zeros((B, 3, 3))
    ea = np.zeros(x.shape[0]) if per_atom_energy else None
    lib().or_forces(B, _p(offsets), _p(x), _p(cells), _p(pbc), _p(pos), C.cast(P, C.c_void_p),
                    int(use_cells), _p(E), _p(F), _p(S), _p(ea))
    if per_atom_energy:
        return E, F, S, ea
    return E, F, S


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def normals3(step, local_atom, seed, uid):
    z = np.zeros(3)
    lib().or_normals3(int(step), int(local_atom), int(seed), int(uid), _p(z))
    return z


def md(offsets, x, v, mass, cells, pbc, pot_of_sys, pots, dt, n_steps, kind=0, kT=None, gamma=0.0,
       seed=0, uid=None, step0=0, use_cells=False):
    """Velocity Verlet (kind 0) or BAOAB Langevin (kind 1) for n_steps.
    Returns new (x, v, E_pot[B], KE[B]); inputs are not modified."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    x = _f64(x).copy(); v = _f64(v).copy(); mass = _f64(mass); cells = _f64(cells)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(B, 3)
    pos = np.ascontiguousarray(pot_of_sys, dtype=np.int32)
    kT = _f64(np.zeros(B) if kT is None else np.broadcast_to(kT, (B,)))
    uid = np.ascontiguousarray(np.arange(B) if uid is None else uid, dtype=np.uint32)
    P = make_pots(pots)
    E = np.zeros(B); KE = np.zeros(B)
    lib().or_md(B, _p(offsets), _p(x), _p(v), _p(mass), _p(cells), _p(pbc), _p(pos), C.cast(P, C.c_void_p),
                int(use_cells), int(kind), float(dt), int(n_steps), _p(kT), float(gamma), int(seed), _p(uid),
                int(step0), _p(E), _p(KE))
    return x, v, E, KE


def md_nhc(offsets, x, v, mass, cells, pbc, pot_of_sys, pots, dt, n_steps, kT, tau, nhc=None, use_cells=False):
    """NVT Nose-Hoover chain (M = 3) for n_steps.  nhc [B, 6] is the chain
    state (xi_1..3, w_1..3), zero if None.  Returns new (x, v, E_pot[B], KE[B],
    nhc[B, 6], H_ext[B] the conserved quantity); inputs are not modified."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    x = _f64(x).copy(); v = _f64(v).copy(); mass = _f64(mass); cells = _f64(cells)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(B, 3)
    pos = np.ascontiguousarray(pot_of_sys, dtype=np.int32)
    kT = _f64(np.broadcast_to(kT, (B,)))
    st = np.zeros((B, 6)) if nhc is None else _f64(nhc).reshape(B, 6).copy()
    P = make_pots(pots)
    E = np.zeros(B); KE = np.zeros(B); H = np.zeros(B)
    lib().or_md_nhc(B, _p(offsets), _p(x), _p(v), _p(mass), _p(cells), _p(pbc), _p(pos), C.cast(P, C.c_void_p),
                    int(use_cells), float(dt), int(n_steps), _p(kT), float(tau), _p(st), _p(E), _p(KE), _p(H))
    return x, v, E, KE, st, H


def md_npt(offsets, x, v, mass, cells, pbc, pot_of_sys, pots, dt, n_steps, kT, gamma, tau, p_ext, seed=0, uid=None,
           step0=0, baro=None, use_cells=False):
    """NPT (isotropic MTK barostat, Langevin atoms and piston) for n_steps.
    baro [B] is the piston velocity v_e (zero if None).  Returns new (x, v,
    cells, baro, E_pot[B], KE[B], H_ext[B], P_inst[B]); inputs are not modified."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    x = _f64(x).copy(); v = _f64(v).copy(); mass = _f64(mass); cells = _f64(cells).reshape(B, 3, 3).copy()
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(B, 3)
    pos = np.ascontiguousarray(pot_of_sys, dtype=np.int32)
    kT = _f64(np.broadcast_to(kT, (B,)))
    uid = np.ascontiguousarray(np.arange(B) if uid is None else uid, dtype=np.uint32)
    ve = np.zeros(B) if baro is None else _f64(baro).reshape(B).copy()
    P = make_pots(pots)
    E = np.zeros(B); KE = np.zeros(B); H = np.zeros(B); Pi = np.zeros(B)
    lib().or_md_npt(B, _p(offsets), _p(x), _p(v), _p(mass), _p(cells), _p(pbc), _p(pos), C.cast(P, C.c_void_p),
                    int(use_cells), float(dt), int(n_steps), _p(kT), float(gamma), float(tau), float(p_ext),
                    C.c_uint32(seed), _p(uid), C.c_uint64(step0), _p(ve), _p(E), _p(KE), _p(H), _p(Pi))
    return x, v, cells, ve, E, KE, H, Pi


FIRE_DEFAULTS = dict(dt0=0.1, dt_max=1.0, finc=1.1, fdec=0.5, alpha0=0.1, falpha=0.99, maxstep=0.2,
                     fmax=1e-3, smax=1e-4, p_ext=0.0, nmin=5, variable_cell=1)


class FireRun:
    """Holds one batch of FIRE systems (variable cell by default) for the oracle."""

    def __init__(self, offsets, x, cells, pbc, pot_of_sys, pots, use_cells=False, **kw):
        prm = dict(FIRE_DEFAULTS); prm.update(kw)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.B = len(self.offsets) - 1
        self.x = _f64(x).copy(); self.cells = _f64(cells).copy()
        self.pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(self.B, 3)
        self.pos = np.ascontiguousarray(pot_of_sys, dtype=np.int32)
        self.P = make_pots(pots)
        self.use_cells = use_cells
        self.st = (OrFireSys * self.B)()
        for s in range(self.B):
            self.st[s].dt = prm["dt0"]; self.st[s].alpha = prm["alpha0"]
            for q in range(9):
                self.st[s].Fd[q] = 1.0 if q in (0, 4, 8) else 0.0
                self.st[s].h0[q] = self.cells[s].reshape(-1)[q]
        self.vel = np.zeros((self.x.shape[0] + 3 * self.B, 3))
        self.prm = OrFireParams(prm["dt_max"], prm["finc"], prm["fdec"], prm["alpha0"], prm["falpha"],
                                prm["maxstep"], prm["fmax"], prm["smax"], prm["p_ext"], prm["nmin"],
                                prm["variable_cell"])

    def step(self, n):
        E = np.zeros(self.B); fm = np.zeros(self.B); sm = np.zeros(self.B)
        lib().or_fire(self.B, _p(self.offsets), _p(self.x), _p(self.cells), _p(self.pbc), _p(self.pos),
                      C.cast(self.P, C.c_void_p), int(self.use_cells), C.cast(self.st, C.c_void_p),
                      _p(self.vel), C.byref(self.prm), int(n), _p(E), _p(fm), _p(sm))
        return E, fm, sm

    def converged(self):
        return np.array([self.st[s].converged for s in range(self.B)], bool)

    def nsteps(self):
        return np.array([self.st[s].nsteps for s in range(self.B)])


def forces_backward(offsets, x, cells, pbc, pot_of_sys, pots, gF, gE=None, gS=None, use_cells=False):
    """Adjoint of (F, E, stress): returns gx [N,3], gtheta [n_pots,3]."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    x = _f64(x); cells = _f64(cells)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(B, 3)
    pos = np.ascontiguousarray(pot_of_sys, dtype=np.int32)
    P = make_pots(pots)
    gF = _f64(gF)
    gE = None if gE is None else _f64(gE)
    gS = None if gS is None else _f64(gS).reshape(B, 9)
    gx = np.zeros_like(x); gth = np.zeros((len(pots), 3))
    lib().or_forces_backward(B, _p(offsets), _p(x), _p(cells), _p(pbc), _p(pos), C.cast(P, C.c_void_p),
                             len(pots), int(use_cells), _p(gF), _p(gE), _p(gS), _p(gx), _p(gth))
    return gx, gth


def rdf(offsets, x, cells, pbc, rmax, K=200, gg=None, use_cells=False):
    """Smeared RDF per system [B,K]; with gg [B,K] also d(sum gg*g)/dx [N,3]."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    x = _f64(x); cells = _f64(cells)
    pbc = np.ascontiguousarray(pbc, dtype=np.uint8).reshape(B, 3)
    g = np.zeros((B, K))
    gx = np.zeros_like(x) if gg is not None else None
    lib().or_rdf(B, _p(offsets), _p(x), _p(cells), _p(pbc), float(rmax), int(K), int(use_cells), _p(g),
                 _p(None if gg is None else _f64(gg)), _p(gx))
    return (g, gx) if gg is not None else g


def traj_rdf_loss(offsets, x0, v0, mass, cells, pbc, pot, dt, T, obs_every, rmax, K, target, grad=True,
                  use_cells=False):
    """NVE trajectory -> averaged smeared RDF -> MSE loss; optional parameter gradient (3,)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    P = make_pots([pot])
    g = np.zeros(K); gth = np.zeros(3) if grad else None
    loss = lib().or_traj_rdf_loss(B, _p(offsets), _p(_f64(x0)), _p(_f64(v0)), _p(_f64(mass)), _p(_f64(cells)),
                                  _p(np.ascontiguousarray(pbc, dtype=np.uint8).reshape(B, 3)),
                                  C.cast(P, C.c_void_p), int(use_cells), float(dt), int(T), int(obs_every),
                                  float(rmax), int(K), _p(_f64(target)), _p(g), _p(gth))
    return loss, g, gth


# Voigt order of stress and strain components: xx, yy, zz, yz, xz, xy
VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def voigt_strain(j, delta):
    """Symmetric strain tensor of Voigt component j with magnitude delta
    (engineering shear: the tensor's off-diagonal entries are delta / 2)."""
    e = np.zeros((3, 3))
    a, b = VOIGT[j]
    if a == b:
        e[a, a] = delta
    else:
        e[a, b] = e[b, a] = 0.5 * delta
    return e


def elastic_constants(offsets, x, cells, pbc, pot_of_sys, pots, delta=1e-5, use_cells=False):
    """Stress-strain coefficients C_ij = d sigma_i / d eps_j [B,6,6] (Voigt,
    eV/A^3) of each system at its configuration, by central differences of
    the stress (forces() sign: sigma = (1/V) dE/d eps) under homogeneous
    strains x -> x (I + eps), h -> h (I + eps) with no internal relaxation (the
    paper names elastic constants among the properties to come, Sec. 5)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    x = _f64(x); cells = _f64(cells).reshape(B, 3, 3)
    C6 = np.zeros((B, 6, 6))
    for j in range(6):
        sig = []
        for sgn in (1.0, -1.0):
            M = np.eye(3) + voigt_strain(j, sgn * delta)
            xs = x.copy()
            for s in range(B):
                xs[offsets[s]:offsets[s + 1]] = x[offsets[s]:offsets[s + 1]] @ M
            _, _, S = forces(offsets, xs, cells @ M, pbc, pot_of_sys, pots, use_cells=use_cells)
            sig.append(S)
        dS = (sig[0] - sig[1]) / (2.0 * delta)
        for i, (a, b) in enumerate(VOIGT):
            C6[:, i, j] = dS[:, a, b]
    return C6

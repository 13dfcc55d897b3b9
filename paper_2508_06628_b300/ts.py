"""Thin Python binding over libts.so (include/ts.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch is used only for
device memory and streams.  There is no fallback: if ``libts.so`` is missing
or CUDA is unavailable, these functions raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libts.so")

TS_OK, TS_ERR_INVALID_ARG, TS_ERR_UNSUPPORTED, TS_ERR_BUDGET, TS_ERR_CUDA = 0, 1, 2, 3, 4
TS_ERR_NEIGHBOR_OVERFLOW, TS_ERR_TIMEOUT, TS_ERR_NONFINITE, TS_ERR_NOT_READY = 5, 6, 7, 8
TS_MIXED, TS_FP64 = 0, 1
TS_NVE, TS_LANGEVIN, TS_NVT_NHC, TS_NPT_LANGEVIN = 0, 1, 2, 3
STATUS_NAMES = {0: "TS_OK", 1: "TS_ERR_INVALID_ARG", 2: "TS_ERR_UNSUPPORTED", 3: "TS_ERR_BUDGET", 4: "TS_ERR_CUDA",
                5: "TS_ERR_NEIGHBOR_OVERFLOW", 6: "TS_ERR_TIMEOUT", 7: "TS_ERR_NONFINITE", 8: "TS_ERR_NOT_READY"}


class TSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("shift", C.c_int32), ("p", C.c_double * 3), ("cutoff", C.c_double),
                ("skin", C.c_double)]


class BatchConfig(C.Structure):
    _fields_ = [("atom_capacity", C.c_int64), ("system_capacity", C.c_int32), ("max_neighbors", C.c_int32),
                ("memory_budget_bytes", C.c_size_t), ("precision", C.c_int32), ("device", C.c_int32),
                ("autotune_cache", C.c_char_p)]


class State(C.Structure):
    _fields_ = [("n_systems", C.c_int32), ("n_atoms", C.c_int64), ("pos", C.c_void_p), ("vel", C.c_void_p),
                ("mass", C.c_void_p), ("cell", C.c_void_p), ("pbc", C.c_void_p), ("system_idx", C.c_void_p),
                ("pot_idx", C.c_void_p), ("uid", C.c_void_p)]


class MDParams(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dt", C.c_double), ("gamma", C.c_double), ("kT", C.c_void_p),
                ("seed", C.c_uint32), ("step0", C.c_uint64), ("tau", C.c_double), ("nhc", C.c_void_p),
                ("p_ext", C.c_double), ("baro", C.c_void_p)]


class FireParams(C.Structure):
    _fields_ = [("dt0", C.c_double), ("dt_max", C.c_double), ("finc", C.c_double), ("fdec", C.c_double),
                ("alpha0", C.c_double), ("falpha", C.c_double), ("maxstep", C.c_double), ("fmax", C.c_double),
                ("smax", C.c_double), ("p_ext", C.c_double), ("nmin", C.c_int32), ("variable_cell", C.c_int32)]


class FireState(C.Structure):
    _fields_ = [("dt", C.c_double), ("alpha", C.c_double), ("npos", C.c_int32), ("started", C.c_int32),
                ("converged", C.c_int32), ("nsteps", C.c_int32), ("Fd", C.c_double * 9), ("h0", C.c_double * 9)]


class Tuning(C.Structure):
    _fields_ = [("item_warps", C.c_int32), ("inner_fraction", C.c_double), ("relist_soon", C.c_double),
                ("bin_factor", C.c_double), ("skin_scale", C.c_double)]


FIRE_STATE_BYTES = C.sizeof(FireState)

_lib = None


def lib():
    """Load libts.so from the package directory (raises if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libts.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, S, I = C.c_void_p, C.c_int, C.c_int
        L.ts_batch_create.argtypes = [C.POINTER(BatchConfig), C.POINTER(Potential), I, C.POINTER(P)]
        L.ts_batch_destroy.argtypes = [P]
        L.ts_last_error.restype = C.c_char_p
        L.ts_last_error.argtypes = [P]
        L.ts_neighbor_build.argtypes = [P, C.POINTER(State), I, P]
        L.ts_neighbor_export.argtypes = [P, P, P, P, P]
        L.ts_batch_max_neighbors.restype = C.c_int32
        L.ts_batch_max_neighbors.argtypes = [P]
        L.ts_pair_forces.argtypes = [P, C.POINTER(State), P, P, P, P]
        L.ts_md_step.argtypes = [P, C.POINTER(State), C.POINTER(MDParams), I, P, P, P]
        L.ts_md_record.argtypes = [P, C.POINTER(State), C.POINTER(MDParams), I, P, P]
        L.ts_fire_init.argtypes = [P, C.POINTER(State), C.POINTER(FireParams), P, P, P]
        L.ts_fire_step.argtypes = [P, C.POINTER(State), P, P, C.POINTER(FireParams), I, P, P, P, P, P]
        L.ts_pair_forces_backward.argtypes = [P, C.POINTER(State), P, P, P, P, P, I, P]
        L.ts_rdf.argtypes = [P, C.POINTER(State), C.c_double, I, P, P]
        L.ts_rdf_backward.argtypes = [P, C.POINTER(State), C.c_double, I, P, P, P]
        L.ts_vv_adjoint_step.argtypes = [P, C.POINTER(State), P, C.c_double, P, P, P, P]
        L.ts_vv_adjoint_segment.argtypes = [P, C.POINTER(State), P, I, C.c_int64, C.c_double, P, P, P, I, C.c_double,
                                            I, P, P]
        L.ts_batch_poll.argtypes = [P, P, I]
        L.ts_autotune.argtypes = [P, C.POINTER(State), C.POINTER(MDParams), I, P]
        L.ts_batch_tuning.argtypes = [P, C.POINTER(Tuning)]
        L.ts_batch_set_tuning.argtypes = [P, C.POINTER(Tuning)]
        L.ts_batch_counters.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.ts_batch_prunes.argtypes = [P, C.POINTER(C.c_int64)]
        L.ts_batch_memory_model.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.ts_profile_pair.argtypes = [P, C.POINTER(State), I, P, C.c_size_t, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int64), P]
        L.ts_bin_pack.argtypes = [P, I, C.c_double, P, C.POINTER(C.c_int32)]
        _lib = L
    return _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA device required: libts.so has no CPU path")
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class DeviceState:
    """SimState in device memory (torch tensors); see ts_state in include/ts.h."""
    pos: object
    vel: object
    mass: object
    cell: object
    pbc: object
    system_idx: object
    pot_idx: object
    uid: object = None
    kT: object = None

    @property
    def n_systems(self):
        return int(self.cell.shape[0])

    @property
    def n_atoms(self):
        return int(self.pos.shape[0])

    def offsets_host(self):
        """System offsets [n_systems + 1] (host numpy) from system_idx."""
        counts = np.bincount(self.system_idx.cpu().numpy(), minlength=self.n_systems)
        return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)

    def c(self):
        self._c = State(self.n_systems, self.n_atoms, _ptr(self.pos), _ptr(self.vel), _ptr(self.mass),
                        _ptr(self.cell), _ptr(self.pbc), _ptr(self.system_idx), _ptr(self.pot_idx), _ptr(self.uid))
        return self._c

    @staticmethod
    def from_host(b, device="cuda"):
        """From a workloads.Batch (numpy) to device tensors."""
        torch = _torch()
        f = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        return DeviceState(f(b.pos, torch.float64), f(b.vel, torch.float64), f(b.mass, torch.float64),
                           f(b.cell, torch.float64), f(b.pbc, torch.uint8), f(b.system_idx, torch.int32),
                           f(b.pot_idx, torch.int32),
                           None if b.uid is None else f(b.uid.astype(np.int64), torch.int64).to(torch.int32),
                           None if b.kT is None else f(b.kT, torch.float64))


def potentials(pots, skins=None):
    arr = (Potential * len(pots))()
    for k, d in enumerate(pots):
        arr[k].kind = int(d["kind"])
        arr[k].shift = int(d.get("shift", 1))
        p = list(d["p"]) + [0.0] * (3 - len(d["p"]))
        for q in range(3):
            arr[k].p[q] = float(p[q])
        arr[k].cutoff = float(d["rc"])
        arr[k].skin = float(d.get("skin", 0.0) if skins is None else skins[k])
    return arr


class Batch:
    """Owns one ts_batch (device scratch sized for the capacities)."""

    def __init__(self, pots, atom_capacity, system_capacity, precision=TS_MIXED, max_neighbors=0, device=0,
                 memory_budget_bytes=0, skins=None, autotune_cache=None):
        self.pots = list(pots)
        self._pots = potentials(self.pots, skins)
        cfg = BatchConfig(int(atom_capacity), int(system_capacity), int(max_neighbors), int(memory_budget_bytes),
                          int(precision), int(device), autotune_cache.encode() if autotune_cache else None)
        h = C.c_void_p()
        st = lib().ts_batch_create(C.byref(cfg), self._pots, len(self.pots), C.byref(h))
        if st != TS_OK:
            raise TSError(st, "ts_batch_create failed")
        self.h = h
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            lib().ts_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != TS_OK:
            raise TSError(st, f"{what}: {lib().ts_last_error(self.h).decode()}")

    def poll(self, stream=None, timeout_ms=-1):
        st = lib().ts_batch_poll(self.h, _stream(stream), int(timeout_ms))
        self._check(st, "ts_batch_poll")

    @property
    def max_neighbors(self):
        return int(lib().ts_batch_max_neighbors(self.h))

    def neighbor_build(self, s: DeviceState, force=False, stream=None):
        self._check(lib().ts_neighbor_build(self.h, C.byref(s.c()), int(force), _stream(stream)), "ts_neighbor_build")

    def neighbor_export(self, s: DeviceState, stream=None):
        torch = _torch()
        M = self.max_neighbors
        j = torch.empty((s.n_atoms, M), dtype=torch.int32, device=s.pos.device)
        img = torch.empty((s.n_atoms, M, 3), dtype=torch.int32, device=s.pos.device)
        cnt = torch.empty((s.n_atoms,), dtype=torch.int32, device=s.pos.device)
        self._check(lib().ts_neighbor_export(self.h, _ptr(j), _ptr(img), _ptr(cnt), _stream(stream)),
                    "ts_neighbor_export")
        return j, img, cnt

    def pair_forces(self, s: DeviceState, F=None, E=None, stress=None, stream=None):
        self._check(lib().ts_pair_forces(self.h, C.byref(s.c()), _ptr(F), _ptr(E), _ptr(stress), _stream(stream)),
                    "ts_pair_forces")

    def md_step(self, s: DeviceState, n_steps, dt, kind=TS_NVE, gamma=0.0, kT=None, seed=0, step0=0, E=None, KE=None,
                stream=None, tau=0.0, nhc=None, p_ext=0.0, baro=None):
        """n_steps MD steps (kind TS_NVE, TS_LANGEVIN, TS_NVT_NHC or
        TS_NPT_LANGEVIN; the chain state ``nhc`` [n_systems, 6] and the piston
        velocities ``baro`` [n_systems] are f64 device tensors updated in
        place; under NPT ``s.cell`` is updated too)."""
        kT = kT if kT is not None else s.kT
        p = MDParams(int(kind), float(dt), float(gamma), _ptr(kT) if kT is not None else None, int(seed), int(step0),
                     float(tau), _ptr(nhc), float(p_ext), _ptr(baro))
        self._check(lib().ts_md_step(self.h, C.byref(s.c()), C.byref(p), int(n_steps), _ptr(E), _ptr(KE),
                                     _stream(stream)), "ts_md_step")

    def md_record(self, s: DeviceState, frames, dt, kind=TS_NVE, gamma=0.0, kT=None, seed=0, step0=0, stream=None,
                  tau=0.0, nhc=None):
        """len(frames) - 1 MD steps recording the positions: ``frames``
        [n_steps + 1, n_atoms, 3] f64 device tensor, row k the positions after
        k steps (TS_NVE, TS_LANGEVIN or TS_NVT_NHC)."""
        kT = kT if kT is not None else s.kT
        p = MDParams(int(kind), float(dt), float(gamma), _ptr(kT) if kT is not None else None, int(seed), int(step0),
                     float(tau), _ptr(nhc), 0.0, None)
        n = int(frames.shape[0]) - 1
        self._check(lib().ts_md_record(self.h, C.byref(s.c()), C.byref(p), n, _ptr(frames), _stream(stream)),
                    "ts_md_record")

    def fire_init(self, s, params, fs, fvel, stream=None):
        self._check(lib().ts_fire_init(self.h, C.byref(s.c()), C.byref(params), _ptr(fs), _ptr(fvel), _stream(stream)),
                    "ts_fire_init")

    def fire_step(self, s, fs, fvel, params, n_steps, converged=None, E=None, fmax=None, smax=None, stream=None):
        self._check(lib().ts_fire_step(self.h, C.byref(s.c()), _ptr(fs), _ptr(fvel), C.byref(params), int(n_steps),
                                       _ptr(converged), _ptr(E), _ptr(fmax), _ptr(smax), _stream(stream)),
                    "ts_fire_step")

    def pair_forces_backward(self, s, gF, gE=None, gS=None, gPos=None, gParams=None, accumulate=False, stream=None):
        self._check(lib().ts_pair_forces_backward(self.h, C.byref(s.c()), _ptr(gF), _ptr(gE), _ptr(gS), _ptr(gPos),
                                                  _ptr(gParams), int(accumulate), _stream(stream)),
                    "ts_pair_forces_backward")

    def rdf(self, s, rmax, K, g, stream=None):
        self._check(lib().ts_rdf(self.h, C.byref(s.c()), float(rmax), int(K), _ptr(g), _stream(stream)), "ts_rdf")

    def rdf_backward(self, s, rmax, K, gg, gPos, stream=None):
        self._check(lib().ts_rdf_backward(self.h, C.byref(s.c()), float(rmax), int(K), _ptr(gg), _ptr(gPos),
                                          _stream(stream)), "ts_rdf_backward")

    def vv_adjoint_step(self, s, x_next, dt, ax, av, gParams, stream=None):
        self._check(lib().ts_vv_adjoint_step(self.h, C.byref(s.c()), _ptr(x_next), float(dt), _ptr(ax), _ptr(av),
                                             _ptr(gParams), _stream(stream)), "ts_vv_adjoint_step")

    def vv_adjoint_segment(self, s, frames, t0, dt, ax, av, gParams, rdf_every=0, rmax=0.0, K=0, gg=None,
                           stream=None):
        """Reverse of len(frames) - 1 NVE steps over frames [n+1, n_atoms, 3]
        (f64 device tensor holding x_t0 ... x_t0+n); see ts.h."""
        n = int(frames.shape[0]) - 1
        self._check(lib().ts_vv_adjoint_segment(self.h, C.byref(s.c()), _ptr(frames), n, int(t0), float(dt),
                                                _ptr(ax), _ptr(av), _ptr(gParams), int(rdf_every), float(rmax),
                                                int(K), _ptr(gg), _stream(stream)), "ts_vv_adjoint_segment")

    def autotune(self, s, dt, kind=TS_LANGEVIN, gamma=0.0, kT=None, seed=0, n_steps=20, stream=None, tau=0.0,
                 nhc=None, p_ext=0.0, baro=None):
        """Tune the batch's launch and list parameters on MD steps of the state
        ``s`` (advanced by the trial steps: pass a copy; under TS_NVT_NHC and
        TS_NPT_LANGEVIN ``nhc`` / ``baro`` and ``s.cell`` advance too); returns
        the chosen tuning as a dict."""
        kT = kT if kT is not None else s.kT
        p = MDParams(int(kind), float(dt), float(gamma), _ptr(kT) if kT is not None else None, int(seed), 0,
                     float(tau), _ptr(nhc), float(p_ext), _ptr(baro))
        self._check(lib().ts_autotune(self.h, C.byref(s.c()), C.byref(p), int(n_steps), _stream(stream)),
                    "ts_autotune")
        return self.tuning()

    def tuning(self):
        t = Tuning()
        self._check(lib().ts_batch_tuning(self.h, C.byref(t)), "ts_batch_tuning")
        return dict(item_warps=t.item_warps, inner_fraction=t.inner_fraction, relist_soon=t.relist_soon,
                    bin_factor=t.bin_factor, skin_scale=t.skin_scale)

    def set_tuning(self, item_warps=8, inner_fraction=0.3, relist_soon=0.5, bin_factor=1.0, skin_scale=1.0):
        t = Tuning(int(item_warps), float(inner_fraction), float(relist_soon), float(bin_factor), float(skin_scale))
        self._check(lib().ts_batch_set_tuning(self.h, C.byref(t)), "ts_batch_set_tuning")

    def profile_pair(self, s, reps=5, flush=None, stream=None):
        ms, pairs, atoms = C.c_double(), C.c_int64(), C.c_int64()
        nb = 0 if flush is None else flush.numel() * flush.element_size()
        self._check(lib().ts_profile_pair(self.h, C.byref(s.c()), int(reps), _ptr(flush), nb, C.byref(ms),
                                          C.byref(pairs), C.byref(atoms), _stream(stream)), "ts_profile_pair")
        return ms.value, pairs.value, atoms.value

    def counters(self):
        a, b = C.c_int64(), C.c_int64()
        lib().ts_batch_counters(self.h, C.byref(a), C.byref(b))
        return a.value, b.value

    def prunes(self):
        """Inner-list prunes so far (one per system and prune)."""
        n = C.c_int64()
        self._check(lib().ts_batch_prunes(self.h, C.byref(n)), "ts_batch_prunes")
        return n.value


def bin_pack(sizes, capacity):
    """ts_bin_pack: first-fit-decreasing bins of ``capacity`` for the memory
    footprints ``sizes``; returns (bin index per system, number of bins).
    Host code only (no GPU needed)."""
    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.float64))
    out = np.zeros(len(sz), np.int32)
    nb = C.c_int32()
    st = lib().ts_bin_pack(sz.ctypes.data if len(sz) else None, len(sz), float(capacity),
                           out.ctypes.data if len(sz) else None, C.byref(nb))
    if st != TS_OK:
        raise TSError(st, "ts_bin_pack")
    return out, nb.value


def default_skins(pots, relax=False):
    """Skin per potential.  For MD (``relax=False``), from step-time sweeps on the 512-system ragged batch
    at 300 K: 1.1 A for LJ argon, 0.88 A for Morse Cu, 1.2 sigma for soft spheres (light, stiff
    particles whose thermal excursions would otherwise force a re-listing every few steps), 0.3 sigma
    for reduced-unit LJ.  Relaxations (``relax=True``) move atoms little and re-list rarely, so shorter
    lists pay there: 0.55 A for Morse Cu and 1.0 sigma for soft spheres (sweep on the FIRE stream)."""
    out = []
    for d in pots:
        if d["kind"] == 2:
            out.append((1.0 if relax else 1.2) * d["p"][0])
        elif d["kind"] == 0:
            out.append(0.3 * d["p"][0] if d["p"][0] < 2 else 1.1)
        else:
            out.append(0.55 if relax else 0.88)
    return out

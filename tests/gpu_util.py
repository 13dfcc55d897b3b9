"""Helpers for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np

from paper_2508_06628_b300 import workloads as W


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def skins_for(pots):
    from paper_2508_06628_b300 import ts
    return ts.default_skins(pots)


def make_batch(hb, precision, extra_atoms=0, extra_sys=0, max_neighbors=0):
    from paper_2508_06628_b300 import ts
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, skins_for(hb.pots))]
    return ts.Batch(pots, hb.n_atoms + extra_atoms, hb.n_systems + extra_sys, precision=precision,
                    max_neighbors=max_neighbors)


def frac_diff(x, y, cell, offsets):
    """Cartesian difference x - y after removing whole lattice vectors, per system."""
    out = np.zeros_like(x)
    for s in range(len(offsets) - 1):
        a, b = offsets[s], offsets[s + 1]
        h = cell[s]
        d = (x[a:b] - y[a:b]) @ np.linalg.inv(h)
        d -= np.round(d)
        out[a:b] = d @ h
    return out


# Mixed precision: the smallest fraction of atoms that must also meet the
# per-atom bound |dF_i| <= max(1e-5 |F_i|, 1e-6), by potential kind (LJ, Morse,
# soft sphere).  The rest may miss it only where FP32 pair arithmetic cannot
# reach it: an atom whose large pair forces cancel (one FP32 rounding of r
# moves a Morse pair force by ~6e-7 eV/A).
MIXED_PER_ATOM_FLOOR = {0: 0.999, 1: 0.99, 2: 0.999}


def kinds_of(hb):
    """Potential kind of every system of a workloads.Batch."""
    return [int(hb.pots[p]["kind"]) for p in hb.pot_idx]


def force_tolerance_ok(F, Fref, offsets, fp64, kinds=None):
    """FP64 mode: per atom |dF_i| <= max(1e-5 |F_i|, 1e-6).  Mixed mode (FP32
    pair arithmetic): per system max_i |dF_i| <= max(1e-5 max_i |F_i|, 1e-6),
    and, when the systems' potential kinds are given, at least
    MIXED_PER_ATOM_FLOOR[kind] of each kind's atoms within the per-atom bound.
    Returns (ok, worst ratio, fraction of atoms passing the per-atom bound)."""
    err = np.linalg.norm(F - Fref, axis=1)
    nrm = np.linalg.norm(Fref, axis=1)
    per_atom = err <= np.maximum(1e-5 * nrm, 1e-6)
    if fp64:
        ratio = (err / np.maximum(1e-5 * nrm, 1e-6)).max()
        return bool(per_atom.all()), float(ratio), float(per_atom.mean())
    worst = 0.0
    for s in range(len(offsets) - 1):
        a, b = offsets[s], offsets[s + 1]
        tol = max(1e-5 * nrm[a:b].max(), 1e-6)
        worst = max(worst, err[a:b].max() / tol)
    ok = worst <= 1.0
    if kinds is not None:
        kind_of_atom = np.repeat(np.asarray(kinds), np.diff(offsets))
        for k, floor in MIXED_PER_ATOM_FLOOR.items():
            sel = kind_of_atom == k
            if sel.any() and per_atom[sel].mean() < floor:
                ok = False
    return ok, float(worst), float(per_atom.mean())


def small_mix(seed, n_systems=10, lo=32, hi=400):
    return W.ragged_mix(seed=seed, n_systems=n_systems, lo=lo, hi=hi)

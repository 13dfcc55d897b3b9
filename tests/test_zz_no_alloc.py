"""ts_pair_forces_noalloc: the entry point for callers that cannot call
cudaMalloc (a host program with a fixed set of buffers and no allocation
after start-up, code inside another framework that owns the device
allocator, a loop that cannot afford cudaMalloc's implicit device
synchronisation).  It must give the oracle's energies, forces and stress --
and the batch path's -- call after call, using only its fixed device table,
and mark systems it cannot evaluate with NaN instead of reading out of range.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2508_06628_b300 import ts
    L = ts.lib()
    L.ts_pair_forces_noalloc.argtypes = [C.POINTER(ts.Potential), C.c_int, C.POINTER(ts.State), C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return ts, L


def _call(torch, ts, L, hb, state, offsets):
    F = torch.full((hb.n_atoms, 3), np.nan, dtype=torch.float64, device="cuda")
    E = torch.full((hb.n_systems,), np.nan, dtype=torch.float64, device="cuda")
    S = torch.full((hb.n_systems, 3, 3), np.nan, dtype=torch.float64, device="cuda")
    off = torch.as_tensor(offsets, dtype=torch.int64, device="cuda")
    pots = ts.potentials(hb.pots)
    st = L.ts_pair_forces_noalloc(pots, len(hb.pots), C.byref(state), C.c_void_p(off.data_ptr()),
                                  C.c_void_p(F.data_ptr()), C.c_void_p(E.data_ptr()), C.c_void_p(S.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, F.cpu().numpy(), E.cpu().numpy(), S.cpu().numpy()


def _fp64_ok(F, E, S, Fr, Er, Sr):
    """The FP64 tolerances of the other tests: per atom max(1e-5 |F|, 1e-6),
    E 1e-9 relative, stress 1e-9 relative."""
    err = np.linalg.norm(F - Fr, axis=1)
    return (np.all(err <= np.maximum(1e-5 * np.linalg.norm(Fr, axis=1), 1e-6)) and
            np.allclose(E, Er, rtol=1e-9, atol=1e-12) and np.allclose(S, Sr, rtol=1e-9, atol=1e-14))


def test_noalloc_matches_oracle_and_batch_path_on_two_calls(orc):
    torch = torch_cuda()
    ts, L = _lib()
    first = None
    for call, seed in enumerate([91, 92]):
        hb = small_mix(seed, n_systems=7, lo=32, hi=300)
        # the batch path in FP64 mode (it also wraps the positions into the cells)
        b = make_batch(hb, ts.TS_FP64)
        s = ts.DeviceState.from_host(hb)
        F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
        E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
        S = torch.zeros((hb.n_systems, 3, 3), dtype=torch.float64, device="cuda")
        b.neighbor_build(s, force=True)
        b.pair_forces(s, F, E, S)
        b.poll()
        st, F2, E2, S2 = _call(torch, ts, L, hb, s.c(), hb.offsets)
        assert st == ts.TS_OK, f"call {call}: status {st}"
        pos = s.pos.cpu().numpy()
        Er, Fr, Sr = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
        assert _fp64_ok(F2, E2, S2, Fr, Er, Sr), f"call {call}: vs the oracle"
        assert _fp64_ok(F2, E2, S2, F.cpu().numpy(), E.cpu().numpy(), S.cpu().numpy()), f"call {call}: vs batch"
        b.close()
        if first is None:
            first = (hb, s, F2, E2, S2)
    # the first input again after the second call: the table keeps the last
    # call's contents, and the fixed-order reductions give the same bits
    hb, s, F1, E1, S1 = first
    st, F3, E3, S3 = _call(torch, ts, L, hb, s.c(), hb.offsets)
    assert st == ts.TS_OK
    assert np.array_equal(F3, F1) and np.array_equal(E3, E1) and np.array_equal(S3, S1)


def test_noalloc_marks_unusable_systems_with_nan(orc):
    """A potential index outside the table and a singular cell: those systems
    get NaN energies, stress and forces; the others are unaffected."""
    torch = torch_cuda()
    ts, L = _lib()
    hb = small_mix(93, n_systems=5, lo=32, hi=200)
    pot_bad = hb.pot_idx.copy()
    pot_bad[1] = 7                      # no such potential (n_pots <= 3)
    cell_bad = hb.cell.copy()
    cell_bad[3, 2] = 0.0                # third lattice vector zero: V = 0
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    pos, cell = dev(hb.pos, torch.float64), dev(cell_bad, torch.float64)
    sidx, pot = dev(hb.system_idx, torch.int32), dev(pot_bad, torch.int32)
    state = ts.State(hb.n_systems, hb.n_atoms, C.c_void_p(pos.data_ptr()), None, None, C.c_void_p(cell.data_ptr()),
                     None, C.c_void_p(sidx.data_ptr()), C.c_void_p(pot.data_ptr()), None)
    st, F, E, S = _call(torch, ts, L, hb, state, hb.offsets)
    assert st == ts.TS_OK
    off = hb.offsets
    for k in (1, 3):
        assert np.isnan(E[k]) and np.all(np.isnan(S[k])) and np.all(np.isnan(F[off[k]:off[k + 1]]))
    good = [0, 2, 4]
    sub = hb.subset(good)
    Er, Fr, Sr = orc.forces(sub.offsets, sub.pos, sub.cell, sub.pbc, sub.pot_idx, sub.pots)
    Fg = np.concatenate([F[off[k]:off[k + 1]] for k in good])
    assert _fp64_ok(Fg, E[good], S[good], Fr, Er, Sr)


def test_noalloc_rejects_too_many_systems():
    torch = torch_cuda()
    ts, L = _lib()
    B = 4097
    dummy = torch.zeros(9 * B, dtype=torch.float64, device="cuda")
    st_c = ts.State(B, B, C.c_void_p(dummy.data_ptr()), None, None, C.c_void_p(dummy.data_ptr()), None,
                    C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()), None)
    pots = ts.potentials([W.LJ_AR])
    st = L.ts_pair_forces_noalloc(pots, 1, C.byref(st_c), C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()),
                                  None, None, None)
    assert st == ts.TS_ERR_BUDGET


def _wrapped(hb, pos):
    """Positions moved into their cells (fractional coordinates in [0, 1))."""
    out = np.empty_like(pos)
    off = hb.offsets
    for k in range(hb.n_systems):
        f = pos[off[k]:off[k + 1]] @ np.linalg.inv(hb.cell[k])
        out[off[k]:off[k + 1]] = (f - np.floor(f)) @ hb.cell[k]
    return out


def test_noalloc_replays_inside_a_captured_graph(orc):
    """After one warm call the entry point can be captured into a CUDA graph in
    global capture mode (in which a cudaMalloc from any thread breaks the
    capture).  Each replay, on positions changed in place, gives the oracle's
    results and the bits of an eager call on the same positions."""
    torch = torch_cuda()
    ts, L = _lib()
    hb = small_mix(94, n_systems=6, lo=32, hi=250)
    rng = np.random.default_rng(94)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    pos = dev(_wrapped(hb, hb.pos), torch.float64)
    cell, sidx, pot = dev(hb.cell, torch.float64), dev(hb.system_idx, torch.int32), dev(hb.pot_idx, torch.int32)
    off = dev(hb.offsets, torch.int64)
    F = torch.empty((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.empty(hb.n_systems, dtype=torch.float64, device="cuda")
    S = torch.empty((hb.n_systems, 3, 3), dtype=torch.float64, device="cuda")
    state = ts.State(hb.n_systems, hb.n_atoms, C.c_void_p(pos.data_ptr()), None, None, C.c_void_p(cell.data_ptr()),
                     None, C.c_void_p(sidx.data_ptr()), C.c_void_p(pot.data_ptr()), None)
    pots = ts.potentials(hb.pots)

    def call():
        return L.ts_pair_forces_noalloc(pots, len(hb.pots), C.byref(state), C.c_void_p(off.data_ptr()),
                                        C.c_void_p(F.data_ptr()), C.c_void_p(E.data_ptr()),
                                        C.c_void_p(S.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))

    assert call() == ts.TS_OK            # the warm call looks up the table's address
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = call()
    assert st == ts.TS_OK
    for rep in range(2):
        p = _wrapped(hb, hb.pos + rng.normal(0.0, 0.02, hb.pos.shape))
        pos.copy_(torch.as_tensor(p))
        F.fill_(np.nan); E.fill_(np.nan); S.fill_(np.nan)
        g.replay()
        torch.cuda.synchronize()
        Fg, Eg, Sg = F.cpu().numpy(), E.cpu().numpy(), S.cpu().numpy()
        Er, Fr, Sr = orc.forces(hb.offsets, p, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
        assert _fp64_ok(Fg, Eg, Sg, Fr, Er, Sr), f"replay {rep}: vs the oracle"
        assert call() == ts.TS_OK
        torch.cuda.synchronize()
        assert (np.array_equal(F.cpu().numpy(), Fg) and np.array_equal(E.cpu().numpy(), Eg) and
                np.array_equal(S.cpu().numpy(), Sg)), f"replay {rep}: vs an eager call"

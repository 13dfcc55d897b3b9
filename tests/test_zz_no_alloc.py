"""ts_pair_forces_noalloc: the entry point for callers that cannot allocate
device memory (fixed-buffer host programs, foreign device allocators,
captured streams).  It must give the same energies, forces and stress as
the batch path, call after call, while using only its fixed device array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_matches_batch_path_on_two_calls():
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    L = ts.lib()
    L.ts_pair_forces_noalloc.argtypes = [C.POINTER(ts.Potential), C.c_int, C.POINTER(ts.State), C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    for call, seed in enumerate([91, 92]):
        hb = small_mix(seed, n_systems=7, lo=32, hi=300)
        # reference: the batch path in FP64 mode
        b = make_batch(hb, ts.TS_FP64)
        s = ts.DeviceState.from_host(hb)
        F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
        E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
        S = torch.zeros((hb.n_systems, 3, 3), dtype=torch.float64, device="cuda")
        b.neighbor_build(s, force=True)
        b.pair_forces(s, F, E, S)
        b.poll()
        # no-allocation path on the same (wrapped) positions
        F2 = torch.full_like(F, np.nan)
        E2 = torch.full_like(E, np.nan)
        S2 = torch.full_like(S, np.nan)
        off = torch.as_tensor(hb.offsets, dtype=torch.int64, device="cuda")
        pots = ts.potentials(hb.pots)
        st = L.ts_pair_forces_noalloc(pots, len(hb.pots), C.byref(s.c()), C.c_void_p(off.data_ptr()),
                                      C.c_void_p(F2.data_ptr()), C.c_void_p(E2.data_ptr()),
                                      C.c_void_p(S2.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        assert st == ts.TS_OK, f"call {call}: status {st}"
        F, E, S, F2, E2, S2 = (t.cpu().numpy() for t in (F, E, S, F2, E2, S2))
        # the FP64 tolerances of the other tests: per atom max(1e-5 |F|, 1e-6), E 1e-9 relative
        err = np.linalg.norm(F2 - F, axis=1)
        assert np.all(err <= np.maximum(1e-5 * np.linalg.norm(F, axis=1), 1e-6)), f"call {call}"
        assert np.allclose(E2, E, rtol=1e-9, atol=1e-12), f"call {call}"
        assert np.allclose(S2, S, rtol=1e-9, atol=1e-14), f"call {call}"
        b.close()


def test_noalloc_rejects_too_many_systems():
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    L = ts.lib()
    L.ts_pair_forces_noalloc.argtypes = [C.POINTER(ts.Potential), C.c_int, C.POINTER(ts.State), C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    B = 4097
    dummy = torch.zeros(9 * B, dtype=torch.float64, device="cuda")
    st_c = ts.State(B, B, C.c_void_p(dummy.data_ptr()), None, None, C.c_void_p(dummy.data_ptr()), None,
                    C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()), None)
    pots = ts.potentials([W.LJ_AR])
    st = L.ts_pair_forces_noalloc(pots, 1, C.byref(st_c), C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()),
                                  None, None, None)
    assert st == ts.TS_ERR_BUDGET

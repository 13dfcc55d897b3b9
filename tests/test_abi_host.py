"""CPU-side checks of the C ABI library: it loads, exports every symbol that
include/ts.h declares, and its host-only batching logic (Fig. 2 memory probe,
in-flight queue of Fig. 3) behaves as the paper describes.  No compute calls."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_06628_b300.csrc import build
    build.build()
    return C.CDLL(os.path.join(ROOT, "paper_2508_06628_b300", "libts.so"))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ts_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_fig2_memory_probe(lib):
    """Fig. 2: model holding ~900 atoms (per-system overhead 15), probes of
    400 and 80 atoms fit 2 and 9 copies; max scaler = min(800, 720) = 720."""
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "fig2_memory_probe.txt")):
        if line.strip() and not line.startswith("#"):
            w = line.split()
            gold[w[0]] = w[1:]
    FITS = C.CFUNCTYPE(C.c_int, C.c_double, C.c_int, C.c_void_p)

    @FITS
    def fits(total, nsys, ctx):
        return int(total + 15 * nsys <= 900)

    sc = (C.c_double * 2)(400, 80)
    nfit = (C.c_int * 2)()
    out = C.c_double()
    lib.ts_estimate_max_scaler.argtypes = [C.c_void_p, C.c_int, FITS, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    st = lib.ts_estimate_max_scaler(sc, 2, fits, None, 1000, nfit, C.byref(out))
    assert st == 0
    assert [nfit[0], nfit[1]] == [int(gold["400"][0]), int(gold["80"][0])]
    assert out.value == float(gold["result"][0])


def test_inflight_queue_fig3(lib):
    """Fig. 3 scenario: 12 structures streamed under a 760-atom budget; the
    active total never exceeds the budget, freed capacity is refilled from
    the stream in order, and every structure runs exactly once."""
    rng = np.random.default_rng(3)
    sizes = rng.integers(40, 400, 12)
    q = C.c_void_p()
    lib.ts_sched_create.argtypes = [C.c_double, C.c_int32, C.c_void_p]
    lib.ts_sched_push.argtypes = [C.c_void_p, C.c_int64, C.c_double]
    lib.ts_sched_fill.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    lib.ts_sched_retire.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    lib.ts_sched_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.ts_sched_create(760.0, 1024, C.byref(q)) == 0
    for i, n in enumerate(sizes):
        assert lib.ts_sched_push(q, i, float(n)) == 0
    ids = (C.c_int64 * 64)()
    nout = C.c_int()
    active, done, order = {}, [], []
    steps_left = {i: int(rng.integers(2, 9)) for i in range(12)}
    for it in range(200):
        assert lib.ts_sched_fill(q, ids, 64, C.byref(nout)) == 0
        for k in range(nout.value):
            active[ids[k]] = sizes[ids[k]]
            order.append(ids[k])
        na, npend, sc = C.c_int32(), C.c_int64(), C.c_double()
        lib.ts_sched_stats(q, C.byref(na), C.byref(npend), C.byref(sc))
        assert sc.value <= 760 + 1e-9 and abs(sc.value - sum(active.values())) < 1e-9
        if not active and npend.value == 0:
            break
        # one "few steps" round: converged systems leave
        fin = []
        for i in list(active):
            steps_left[i] -= 1
            if steps_left[i] == 0:
                fin.append(i)
        arr = (C.c_int64 * max(1, len(fin)))(*fin)
        assert lib.ts_sched_retire(q, arr, len(fin)) == 0
        for i in fin:
            del active[i]
            done.append(i)
    assert sorted(done) == list(range(12)) and order == list(range(12))
    lib.ts_sched_destroy.argtypes = [C.c_void_p]
    lib.ts_sched_destroy(q)


def test_oversized_system_rejected(lib):
    q = C.c_void_p()
    lib.ts_sched_create(760.0, 8, C.byref(q))
    assert lib.ts_sched_push(q, 0, C.c_double(800.0)) == 3   # TS_ERR_BUDGET
    lib.ts_sched_destroy(q)


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2508_06628_b300 import ts
    with pytest.raises(RuntimeError):
        ts._torch()


def test_byte_budget_drives_the_fig2_probe():
    """The runtime's byte-budget admission runs the Fig. 2 probe with the
    engine's byte model as its fit test: with 1 byte per atom, 15 bytes per
    system and a 900-byte budget (the worked example's ~900-atom model),
    probes of 400 and 80 atoms fit 2 and 9 copies and the limit is 720; with
    the density scaler the limit is in scaler units (copies x n^2/V)."""
    from paper_2508_06628_b300 import runtime
    limit, copies = runtime.max_scaler_from_budget([400, 80], [400, 80], 1.0, 15.0, 900.0)
    assert copies == [2, 9] and limit == 720.0
    dens = [400 * 400 / 4000.0, 80 * 80 / 1000.0]           # n_atoms x density of two probe systems
    limit_d, copies_d = runtime.max_scaler_from_budget([400, 80], dens, 1.0, 15.0, 900.0)
    assert copies_d == [2, 9] and limit_d == min(2 * dens[0], 9 * dens[1])
    with pytest.raises(Exception):
        runtime.max_scaler_from_budget([1000], [1000], 1.0, 15.0, 900.0)   # not even one copy fits

"""Benchmark: batched Langevin MD throughput (atom-steps/s) on the ragged
512-system mix (LJ argon / Morse copper / soft spheres, 32-2048 atoms each),
through the C ABI of libts.so.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one MD step of the whole batch: BAOAB kick/drift/noise, skin check
with per-system conditional re-listing, fused pair forces.  Steps run as
calls of ``--inner`` steps (one CUDA-graph replay each); L2 is flushed
(256 MiB write) before every call, outside the timed events.  Rank 0 prints
one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched MD atom-steps/s on 1 B300 vs per-system loop; pair-kernel % HBM peak"
UNIT = "atom-steps/s"
FP32_LANES_PER_SM = 128
FLOP_PER_PAIR = 30          # per ordered pair within the cutoff (force, energy, virial terms)
BYTES_PER_ATOM = 32         # read own position, write own force, per atom-step
# DRAM bytes (read + write) of one forces-only k_pair_small launch (inner lists, rc + 0.45 skin) on
# ragged-mix-512, from one ncu capture of the steady launch; reported only while the kernel's sources
# (ts_pair.cu, then ts_internal.cuh) hash to the value recorded with the capture
PAIR_TRAFFIC = {"bytes": 54_294_272 + 569_344, "source_sha1": "87b3ccc3a3fe858a74ee7694332db1d6d2d1bd4e"}


def pair_traffic():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2508_06628_b300", "csrc")
    h = hashlib.sha1(b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("ts_pair.cu", "ts_internal.cuh")))
    return PAIR_TRAFFIC["bytes"] if h.hexdigest() == PAIR_TRAFFIC["source_sha1"] else None


def n_sm(dev=0):
    """Streaming multiprocessors of the device the bench runs on."""
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), d.get("sm_max_mhz", 2032.0), "measured"
    return 6400.0, 2032.0, "fallback"


def workload(seed=1, n_systems=512):
    from paper_2508_06628_b300 import workloads as W
    return W.ragged_mix(seed=seed, n_systems=n_systems)


class _Nvml:
    """The few read-only NVML calls the clock sampler needs, through ctypes on
    the driver's libnvidia-ml (no Python binding required)."""

    CLOCK_SM = 1

    def __init__(self):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        self.reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def handle(self, pci_bus_id, index=0):
        C = self.C
        h = C.c_void_p()
        if self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), C.byref(h)) != 0:
            if self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
        return h

    def clock(self, h, maximum=False):
        C = self.C
        v = C.c_uint()
        f = self.lib.nvmlDeviceGetMaxClockInfo if maximum else self.lib.nvmlDeviceGetClockInfo
        if f(h, C.c_int(self.CLOCK_SM), C.byref(v)) != 0:
            raise RuntimeError("clock query failed")
        return float(v.value)

    def event_reasons(self, h):
        C = self.C
        v = C.c_ulonglong()
        if self.reasons(h, C.byref(v)) != 0:
            raise RuntimeError("clock-event query failed")
        return int(v.value)


class Clocks:
    """Sample the SM clock and the clock-event reasons through NVML every
    ~1 ms in a host thread while the timed region runs (the region of the
    default line is a few milliseconds, shorter than nvidia-smi's sampling
    period), plus one sample as it opens and one as it closes."""

    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
               "sw_power_cap": 0x4, "hw_power_brake_slowdown": 0x80}

    def __init__(self, device):
        self.samples = []
        self.h = None
        self.error = None
        try:
            import torch
            self.nv = _Nvml()
            pr = torch.cuda.get_device_properties(device)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            self.h = self.nv.handle(bus, 0)
            self.max_mhz = self.nv.clock(self.h, maximum=True)
        except Exception as e:
            self.h = None
            self.error = f"NVML unavailable: {e!r}"

    def _sample(self):
        try:
            self.samples.append((self.nv.clock(self.h), self.nv.event_reasons(self.h)))
        except Exception as e:
            self.error = f"NVML sample failed: {e!r}"

    def _run(self):
        import time as _t
        while not self.stop:
            self._sample()
            _t.sleep(0.001)

    def __enter__(self):
        import threading
        self.stop = False
        self.t = None
        if self.h is not None:
            self._sample()
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *a):
        self.stop = True
        if self.t:
            self.t.join(timeout=5)
            self._sample()

    def summary(self):
        if not self.samples:
            return {"error": self.error} if self.error else None
        sm = [c for c, _ in self.samples]
        mask = 0
        for _, r in self.samples:
            mask |= r
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.max_mhz, "samples": len(self.samples),
                "reasons": sorted(n for n, bit in self.REASONS.items() if mask & bit),
                "how": "NVML SM clock and clock-event reasons, sampled every ~1 ms during the timed region"}


def run_ours(args, rank, world):
    import torch
    from paper_2508_06628_b300 import ts
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    # one workload of 512 systems per GPU, sharded by atom-balanced packing
    # (at N = 1 it is ragged-mix-512 itself)
    from paper_2508_06628_b300 import parallel
    hb_all = workload(seed=1, n_systems=512 * world)
    hb = hb_all if world == 1 else hb_all.subset(parallel.shard_systems(np.diff(hb_all.offsets), world)[rank])
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots))]
    # --tune-cache: the autotuner appends its result there, and a batch created
    # with the file applies its last matching line (with --no-tune: a run with
    # the tuning an earlier run chose)
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, precision=ts.TS_MIXED, device=dev.index,
                 autotune_cache=args.tune_cache)
    s = ts.DeviceState.from_host(hb, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    dt, gamma = hb.meta["dt"], hb.meta["gamma"]
    inner = max(1, min(args.inner, args.steps))
    tuning, tune_s = None, 0.0
    if not args.no_tune:
        # the library's autotuner on a copy of the state, before (and outside) the timed region
        t0 = time.time()
        with torch.cuda.stream(stream):
            trial = ts.DeviceState(*[None if t is None else t.clone() for t in
                                     (s.pos, s.vel, s.mass, s.cell, s.pbc, s.system_idx, s.pot_idx, s.uid, s.kT)])
            tuning = b.autotune(trial, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=11, n_steps=100, stream=stream)
            del trial
        tune_s = time.time() - t0
    else:
        tuning = b.tuning()
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device=dev)
    KE = torch.zeros_like(E)
    step = 0
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        for _ in range(args.warmup):
            b.md_step(s, inner, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=5, step0=step, stream=stream)
            step += inner
        b.poll(stream)
    ncalls = (args.steps + inner - 1) // inner
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ncalls)]
    l0, r0 = b.counters()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(dev)
    with clk, torch.cuda.stream(stream):
        for c in range(ncalls):
            flush.fill_(c & 0xff)
            evs[c][0].record(stream)
            b.md_step(s, inner, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=5, step0=step, stream=stream)
            evs[c][1].record(stream)
            step += inner
        stream.synchronize()
    torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    l1, r1 = b.counters()
    b.poll(stream)
    steps_done = ncalls * inner
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        na = torch.tensor([hb.n_atoms], dtype=torch.float64, device=dev)
        dist.all_reduce(na)
        total_atoms = float(na.item())
    else:
        total_atoms = float(hb.n_atoms)
    value = total_atoms * steps_done / (ms / 1e3)
    out = {"ms": ms, "steps": steps_done, "value": value, "launches": l1 - l0, "relists": r1 - r0,
           "total_atoms": int(total_atoms), "total_systems": int(hb_all.n_systems),
           "tuning": dict(tuning, autotuned=not args.no_tune, tune_seconds=round(tune_s, 2)),
           "n_atoms": hb.n_atoms, "n_systems": hb.n_systems, "inner": inner, "clocks": clk.summary()}
    # --- end to end through the public API with host buffers, on every rank
    # (each its own shard): all ranks' atoms over the slowest rank's time
    e2e_out = e2e(b, s, hb, dev, stream, args, dt, gamma, inner)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_out.pop("ms")], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_out["value"] = total_atoms * e2e_out.pop("steps") / (float(t.item()) / 1e3)
    else:
        e2e_out.pop("ms"); e2e_out.pop("steps")
    out["e2e"] = e2e_out
    if rank != 0:
        return out, None
    # --- dominant kernel: the pair kernel, timed alone with CUDA events on the stream
    # In the timed region L2 is flushed once per call of `inner` steps, so one
    # pair launch in `inner` starts cold and the rest find the positions in L2:
    # time both ways and weight them the same.
    with torch.cuda.stream(stream):
        torch.cuda.nvtx.range_push("pair_kernel_timing")   # the launches a profiler capture selects
        kms_cold, pairs, atoms = b.profile_pair(s, reps=10, flush=flush, stream=stream)
        kms_warm, _, _ = b.profile_pair(s, reps=20, flush=None, stream=stream)
        torch.cuda.nvtx.range_pop()
    kms = (kms_cold + (inner - 1) * kms_warm) / inner
    hbm, smmhz, src = peaks()
    clocks = out["clocks"] or {}
    flops = pairs * FLOP_PER_PAIR
    nsm = n_sm(dev)
    alu_peak = nsm * FP32_LANES_PER_SM * 2 * smmhz * 1e6 / 1e12      # TFLOP/s, FMA = 2
    achieved = flops / (kms / 1e3) / 1e12
    hbm_achieved = atoms * BYTES_PER_ATOM / (kms / 1e3) / 1e9
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                       "frac": achieved / alu_peak, "traffic": pair_traffic(),
                       "kernel": "k_pair_small" + (" + k_pair" if int(np.bincount(hb.system_idx).max()) > 2048 else ""),
                       "kernel_ms": kms, "kernel_ms_cold_l2": kms_cold, "kernel_ms_warm_l2": kms_warm,
                       "pairs_per_launch": pairs, "flop_per_pair": FLOP_PER_PAIR,
                       "peak_source": f"{nsm} SM x 128 FP32 lanes x 2 x {smmhz:.0f} MHz (max SM clock)",
                       "hbm": {"achieved": hbm_achieved, "peak": hbm, "unit": "GB/s", "frac": hbm_achieved / hbm,
                               "bytes_per_atom": BYTES_PER_ATOM, "peak_source": src}}
    # --- forces, energies and stress at the final positions (outside the timed
    # region), for the parity record of the oracle leg
    Ff = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device=dev)
    Ef = torch.zeros(hb.n_systems, dtype=torch.float64, device=dev)
    Sf = torch.zeros((hb.n_systems, 3, 3), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        b.pair_forces(s, Ff, Ef, Sf, stream=stream)
        b.poll(stream)
    out["final"] = {"pos": s.pos.cpu().numpy(), "F": Ff.cpu().numpy(), "E": Ef.cpu().numpy(), "S": Sf.cpu().numpy()}
    # --- per-system launch loop (same kernels, one system per batch, one step per call)
    if not args.no_loop:
        out["per_system_loop"] = per_system_loop(hb, pots, dev, args)
    b.close()
    return out, hb


def per_system_loop(hb, pots, dev, args, n_sample=32, steps=3):
    import torch
    from paper_2508_06628_b300 import ts
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(hb.n_systems, n_sample, replace=False))
    stream = torch.cuda.Stream(device=dev)
    runs = []
    for k in pick:
        sub = hb.subset([k])
        bb = ts.Batch(pots, sub.n_atoms, 1, precision=ts.TS_MIXED, device=dev.index)
        ss = ts.DeviceState.from_host(sub, device=dev)
        with torch.cuda.stream(stream):
            bb.neighbor_build(ss, force=True, stream=stream)
            bb.md_step(ss, 1, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=5, stream=stream)
        runs.append((bb, ss, sub.n_atoms))
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for t in range(steps):
            for bb, ss, n in runs:
                bb.md_step(ss, 1, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=5, step0=t + 1,
                           stream=stream)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    atoms = sum(n for _, _, n in runs)
    for bb, _, _ in runs:
        bb.close()
    return {"value": atoms * steps / (ms / 1e3), "unit": UNIT, "systems_sampled": int(n_sample), "steps": steps,
            "how": "each system its own batch, one ts_md_step(1) call per system per step, sequential"}


def e2e(b, s, hb, dev, stream, args, dt, gamma, inner):
    """Same metric through the public API with the state held on the host in
    pinned buffers (runtime.HostMD): every call copies positions and
    velocities in (H2D), runs its steps and copies the new positions,
    velocities and per-system energies back (D2H), so the trajectory continues
    from call to call.  HostMD splits the systems into two atom-balanced
    groups on two streams, so that one group's copies overlap the other's
    steps; both groups take the main batch's tuning."""
    import torch
    from paper_2508_06628_b300 import runtime, ts
    if hb.uid is None:
        hb.uid = np.arange(hb.n_systems, dtype=np.uint32)
    hm = runtime.HostMD(hb, [dict(p) for p in b.pots], parts=2, device=dev.index, tuning=b.tuning())
    ncalls = max(1, (args.steps + inner - 1) // inner)
    hm.step(inner, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=9)   # warm (lists built)
    hm.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for c in range(ncalls):
        hm.step(inner, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=9, step0=(c + 1) * inner, after=e0 if c == 0 else None)
    hm.join(stream)
    e1.record(stream)
    stream.synchronize()
    hm.synchronize()
    ms = e0.elapsed_time(e1)
    hm.close()
    return {"value": hb.n_atoms * ncalls * inner / (ms / 1e3), "unit": UNIT, "ms": ms, "steps": ncalls * inner,
            "h2d_bytes_per_step": int(hm.h2d_bytes() / inner), "d2h_bytes_per_step": int(hm.d2h_bytes() / inner),
            "how": f"per call of {inner} steps: H2D pos+vel from pinned host, D2H pos+vel+energies; the systems in "
                   f"two atom-balanced groups on two streams (runtime.HostMD), one group's copies beside the "
                   f"other's steps"}


def cpu_baseline(hb, budget_s=15.0, steps=None, warmup=0):
    """FP64 oracle (cell-list mode) on a bounded sample of the same workload:
    one BAOAB step of a random group of 16 systems per step.  steps=None: the
    groups in turn, passing over the batch again, for about budget_s of CPU
    time (at most eight passes); otherwise warmup untimed and then exactly
    `steps` timed steps (the groups taken in turn)."""
    from oracle import oracle
    rng = np.random.default_rng(0)
    order = rng.permutation(hb.n_systems)
    chunk = 16
    groups = [np.sort(order[k:k + chunk]) for k in range(0, hb.n_systems, chunk)]
    total_atoms, total_time, done = 0, 0.0, 0
    t0 = time.time()
    for t in range(warmup + (steps if steps is not None else 8 * len(groups))):
        sub = hb.subset(groups[t % len(groups)])
        t1 = time.time()
        oracle.md(sub.offsets, sub.pos, sub.vel, sub.mass, sub.cell, sub.pbc, sub.pot_idx, sub.pots, hb.meta["dt"],
                  1, kind=1, kT=sub.kT, gamma=hb.meta["gamma"], seed=5, uid=sub.uid, use_cells=True)
        if t >= warmup:
            total_time += time.time() - t1
            total_atoms += sub.n_atoms
            done += 1
        if steps is None and time.time() - t0 > budget_s:
            break
    return {"value": total_atoms * 1 / total_time, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "steps": done, "seconds": total_time,
            "sample": f"{done} steps, each one BAOAB step of a group of {chunk} systems of the batch (random, "
                      f"seed 0, groups in turn), {total_atoms} atom-steps, FP64 cell-list mode"}


def oracle_parity(hb, final, n_pick=8):
    """Error of the GPU result against the FP64 oracle (cell-list mode) on
    n_pick sampled systems at the positions the timed run ended on: forces,
    energies and stress of the mixed-precision path, computed after the timed
    region.  Force tolerance per system: max_i |dF_i| <= max(1e-5 max_i |F_i|,
    1e-6 eV/A); the per-atom bound max(1e-5 |F_i|, 1e-6) is reported as a
    pass fraction; energies and stress as relative errors."""
    from oracle import oracle
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(hb.n_systems, n_pick, replace=False))
    off = hb.offsets
    sub = hb.subset(pick)
    pos = np.concatenate([final["pos"][off[k]:off[k + 1]] for k in pick])
    Er, Fr, Sr = oracle.forces(sub.offsets, pos, sub.cell, sub.pbc, sub.pot_idx, sub.pots, use_cells=True)
    Fg = np.concatenate([final["F"][off[k]:off[k + 1]] for k in pick])
    err = np.linalg.norm(Fg - Fr, axis=1)
    nrm = np.linalg.norm(Fr, axis=1)
    worst, e_rel, s_rel = 0.0, 0.0, 0.0
    so = sub.offsets
    for m, k in enumerate(pick):
        a, e = so[m], so[m + 1]
        worst = max(worst, float(err[a:e].max() / max(1e-5 * nrm[a:e].max(), 1e-6)))
        e_rel = max(e_rel, float(abs(final["E"][k] - Er[m]) / max(abs(Er[m]), 1e-12)))
        s_rel = max(s_rel, float(np.abs(final["S"][k] - Sr[m]).max() / max(np.abs(Sr[m]).max(), 1e-12)))
    return {"reference": "FP64 oracle, cell-list mode", "systems": [int(k) for k in pick],
            "atoms": int(sub.n_atoms), "force_worst_ratio_to_tol": worst,
            "force_per_atom_pass_frac": float(np.mean(err <= np.maximum(1e-5 * nrm, 1e-6))),
            "force_max_abs_err": float(err.max()), "energy_max_rel_err": e_rel, "stress_max_rel_err": s_rel,
            "tolerance": "forces: per system max|dF| <= max(1e-5 max|F|, 1e-6 eV/A); energy <= 1e-6 relative "
                         "(mixed precision)", "when": "after the timed region, at its final positions"}


FLOP_PER_PAIR_BWD = 100   # pair-force backward, per pair within rc (positions and parameters)


def run_row_adjoint(args):
    """The adjoint row: the pair-force backward (gF, gE -> gradients in positions
    and potential parameters) on the MD workload after its warm-up, timed with
    CUDA events around whole backward calls (the call's gradient import,
    pair-backward kernel, export and parameter reductions)."""
    import torch
    from paper_2508_06628_b300 import ts
    dev = torch.device("cuda", 0)
    hb = workload(seed=1)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots))]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, precision=ts.TS_MIXED, device=0)
    s = ts.DeviceState.from_host(hb, device=dev)
    stream = torch.cuda.Stream(device=dev)
    g = torch.Generator(device=dev).manual_seed(3)
    gF = torch.randn((hb.n_atoms, 3), dtype=torch.float64, device=dev, generator=g)
    gE = torch.ones(hb.n_systems, dtype=torch.float64, device=dev)
    gPos = torch.zeros_like(gF)
    gPar = torch.zeros((len(hb.pots), 3), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        b.md_step(s, 20, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=5, stream=stream)
        b.pair_forces(s, None, None, None, stream=stream)
        for _ in range(args.warmup):
            b.pair_forces_backward(s, gF, gE, None, gPos, gPar, stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("backward_calls")   # the launches a profiler capture selects
        e0.record(stream)
        for _ in range(args.steps):
            b.pair_forces_backward(s, gF, gE, None, gPos, gPar, stream=stream)
        e1.record(stream)
        stream.synchronize()
        torch.cuda.nvtx.range_pop()
        _, pairs, _ = b.profile_pair(s, reps=1, flush=None, stream=stream)
    ms = e0.elapsed_time(e1) / args.steps
    b.poll()
    _, smmhz, _ = peaks()
    alu_peak = n_sm(dev) * FP32_LANES_PER_SM * 2 * smmhz * 1e6 / 1e12
    achieved = pairs * FLOP_PER_PAIR_BWD / (ms / 1e3) / 1e12
    b.close()
    return {"metric": "pair-force backward (positions + parameters) atom-evaluations/s", "value": hb.n_atoms / (ms / 1e3),
            "unit": "atom-evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "row": "adjoint",
            "config": {"workload": "ragged-mix-512 after 20 BAOAB steps; upstream gF ~ N(0,1), gE = 1",
                       "n_systems": hb.n_systems, "n_atoms": hb.n_atoms},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "traffic": None, "kernel": "k_pair_bwd (whole backward call timed)",
                         "pairs_per_launch": pairs, "flop_per_pair": FLOP_PER_PAIR_BWD}}


def run_row_fire(args):
    """The FIRE row: variable-cell FIRE on 1024 systems of the relaxation
    stream (Morse Cu FCC, 64-864 atoms, rattled and scaled), timed with CUDA
    events around calls of 10 FIRE steps."""
    import torch
    from paper_2508_06628_b300 import ts, workloads as W
    dev = torch.device("cuda", 0)
    hb = W.fire_stream(seed=2, n_systems=8192).subset(list(range(1024)))
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots, relax=True))]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, precision=ts.TS_MIXED, device=0)
    s = ts.DeviceState.from_host(hb, device=dev)
    stream = torch.cuda.Stream(device=dev)
    # fmax and smax far below reach, so that every system takes every timed step
    P = ts.FireParams(0.1, 1.0, 1.1, 0.5, 0.1, 0.99, 0.2, 1e-12, 1e-12, 0.0, 5, 1)
    conv = torch.zeros(hb.n_systems, dtype=torch.uint8, device=dev)
    fs = torch.zeros(hb.n_systems * ts.FIRE_STATE_BYTES, dtype=torch.uint8, device=dev)
    fv = torch.zeros((hb.n_atoms + 3 * hb.n_systems, 3), dtype=torch.float64, device=dev)
    inner = 10
    ncalls = max(1, (args.steps + inner - 1) // inner)
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        b.fire_init(s, P, fs, fv, stream=stream)
        for _ in range(args.warmup):
            b.fire_step(s, fs, fv, P, inner, stream=stream)
        stream.synchronize()
        l0 = b.counters()[0]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ncalls):
            b.fire_step(s, fs, fv, P, inner, stream=stream)
        e1.record(stream)
        b.fire_step(s, fs, fv, P, 1, converged=conv, stream=stream)
        stream.synchronize()
    assert int(conv.sum()) == 0, "a system converged inside the timed region"
    ms = e0.elapsed_time(e1) / (ncalls * inner)
    launches = b.counters()[0] - l0
    b.poll()
    b.close()
    return {"metric": "batched variable-cell FIRE atom-steps/s", "value": hb.n_atoms / (ms / 1e3),
            "unit": "atom-steps/s", "n_gpus": 1, "steps": ncalls * inner, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "row": "fire", "gpu_launches": launches,
            "config": {"workload": "fire-stream: first 1024 of 8192 Morse Cu FCC supercells of 64-864 atoms, "
                                   "0.1 A rattle, isotropic scale U[0.97, 1.03]; variable cell",
                       "n_systems": hb.n_systems, "n_atoms": hb.n_atoms, "fire_steps_per_call": inner}}


def run_row_ensemble(args, which):
    """The other thermostats and barostat on the MD workload (ragged-mix-512 at
    300 K, dt 1 fs): NVT Nose-Hoover chain (tau 100 fs) or NPT Langevin with the
    isotropic MTK piston (tau 100 fs, 1 GPa: argon above its critical
    temperature and the purely repulsive soft spheres would expand without
    bound at 1 bar), calls of 10 steps timed with CUDA events, L2 flushed
    before every call as in the default line."""
    import torch
    from paper_2508_06628_b300 import ts, workloads as W
    dev = torch.device("cuda", 0)
    hb = workload(seed=1)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots))]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, precision=ts.TS_MIXED, device=0)
    s = ts.DeviceState.from_host(hb, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    dt, gamma, tau = hb.meta["dt"], hb.meta["gamma"], 100.0 / W.T0_FS
    kw = dict(kind=ts.TS_NVT_NHC, tau=tau, nhc=torch.zeros((hb.n_systems, 6), dtype=torch.float64, device=dev)) \
        if which == "nhc" else \
        dict(kind=ts.TS_NPT_LANGEVIN, gamma=gamma, tau=tau, p_ext=1.0 / 160.21766208,   # 1 GPa in eV/A^3
             baro=torch.zeros(hb.n_systems, dtype=torch.float64, device=dev))
    inner = 10
    ncalls = max(1, min(args.steps, 1000) // inner)
    stream = torch.cuda.Stream(device=dev)
    step = 0
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        for _ in range(max(args.warmup, 3)):
            b.md_step(s, inner, dt, seed=5, step0=step, stream=stream, **kw)
            step += inner
        stream.synchronize()
        l0, r0 = b.counters()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ncalls)]
        for c in range(ncalls):
            flush.fill_(c & 0xff)
            evs[c][0].record(stream)
            b.md_step(s, inner, dt, seed=5, step0=step, stream=stream, **kw)
            evs[c][1].record(stream)
            step += inner
        stream.synchronize()
        l1, r1 = b.counters()
    ms = sum(a.elapsed_time(e) for a, e in evs) / (ncalls * inner)
    b.poll()
    b.close()
    name = {"nhc": "NVT Nose-Hoover chain", "npt": "NPT Langevin (isotropic MTK piston)"}[which]
    return _line(f"batched MD atom-steps/s, {name}", hb.n_atoms / (ms / 1e3), UNIT, ms, ncalls * inner,
                 max(args.warmup, 3), "f32",
                 {"workload": "ragged-mix-512 (as the default line), 300 K, dt 1 fs, tau 100 fs" +
                              (", 1 GPa" if which == "npt" else ""), "n_systems": hb.n_systems,
                  "n_atoms": hb.n_atoms, "md_steps_per_call": inner,
                  "l2": "flushed (256 MiB write) before every call, outside the timed events"},
                 row=which, gpu_launches=l1 - l0, relists_in_timed_region=r1 - r0)


def _line(metric, value, unit, ms, steps, warmup, dtype, config, **extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": steps, "warmup": warmup,
         "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
         "data": "synthetic", "config": config}
    d.update(extra)
    return d


def run_row_nve256(args):
    """One 256-atom LJ argon box (FCC 4x4x4, a = 5.26 A, 50 K), NVE velocity
    Verlet at dt = 2 fs, 1000 steps in FP64 as calls of 100 steps; reports the
    relative drift of E + KE beside the throughput, and the oracle on the same
    1000 steps."""
    import torch
    from paper_2508_06628_b300 import ts, workloads as W
    dev = torch.device("cuda", 0)
    hb = W.single_lj_argon(seed=0)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots))]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, precision=ts.TS_FP64, device=0)
    s = ts.DeviceState.from_host(hb, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    KE = torch.zeros_like(E)
    dt, n, inner = hb.meta["dt"], 1000, 100
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        b.md_step(s, 1, dt, kind=ts.TS_NVE, E=E, KE=KE, stream=stream)   # energies at the start
        stream.synchronize()
        H0 = float(E[0] + KE[0])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c in range(n // inner):
            b.md_step(s, inner, dt, kind=ts.TS_NVE, E=E, KE=KE, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / n
    H1 = float(E[0] + KE[0])
    b.poll()
    b.close()
    out = _line("NVE atom-steps/s, one 256-atom LJ argon box", hb.n_atoms / (ms / 1e3), UNIT, ms, n, 1, "f64",
                {"workload": "lj-argon-256: FCC 4x4x4, a = 5.26 A, rc 2.5 sigma shifted, MB 50 K, NVE dt 2 fs",
                 "n_systems": 1, "n_atoms": hb.n_atoms}, row="nve256",
                energy_drift_rel=abs(H1 - H0) / abs(H0))
    if not args.no_cpu:
        from oracle import oracle
        t0 = time.time()
        oracle.md(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots, dt, n, kind=0)
        tc = time.time() - t0
        out["cpu_baseline"] = {"value": hb.n_atoms * n / tc, "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": "the same 1000 NVE steps, FP64 brute force"}
    return out


def run_row_inflight(args):
    """Structural relaxation of a stream of 8192 Morse Cu cells (64-864 atoms,
    0.1 A rattle, cell scaled by U[0.97, 1.03]) by variable-cell FIRE to fmax
    1e-3 eV/A and |sigma| 1e-4 eV/A^3, at most 1024 systems in flight and a
    600 MiB device budget for the batch: converged systems retire and queued
    ones are admitted between rounds of 25 FIRE steps.  Host wall time of the whole
    relaxation, batch set-up included."""
    import torch
    from paper_2508_06628_b300 import runtime, ts, workloads as W
    hb = W.fire_stream(seed=2, n_systems=8192)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots, relax=True))]
    # warm-up on 64 systems of the stream: the first use of each PyTorch
    # kernel of the admission and retirement path costs far more than its run
    budget = 600 << 20    # device bytes of batch scratch
    runtime.relax_inflight(hb.subset(list(range(64))), pots, max_active=1024, n_inner=25, precision=ts.TS_MIXED,
                           memory_budget_bytes=budget)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, log = runtime.relax_inflight(hb, pots, max_active=1024, n_inner=25, precision=ts.TS_MIXED,
                                      memory_budget_bytes=budget, memory_scales_with="n_atoms")
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    assert len(res) == hb.n_systems, "systems left unrelaxed"
    atom_steps = sum(r["atoms"] for r in log) * 25
    out = _line("structures relaxed per second (variable-cell FIRE, in-flight batching)", hb.n_systems / t,
                "structures/s", 1e3 * t / len(log), len(log), 1, "f32",
                {"workload": "fire-stream-8192: Morse Cu FCC 64-864 atoms, 0.1 A rattle, U[0.97, 1.03] scale; "
                             "fmax 1e-3 eV/A, |sigma| 1e-4 eV/A^3; <= 1024 in flight, admission by a 600 MiB device "
                "budget through the Fig. 2 probe (memory scales with n_atoms)",
                 "n_systems": hb.n_systems, "n_atoms": hb.n_atoms, "fire_steps_per_round": 25},
                row="inflight", atom_steps_per_s=atom_steps / t, rounds=len(log), wall_s=t,
                mean_active=float(np.mean([r["active"] for r in log])))
    if not args.no_cpu:
        from oracle import oracle
        sub = hb.subset(list(range(16)))
        fr = oracle.FireRun(sub.offsets, sub.pos, sub.cell, sub.pbc, sub.pot_idx, sub.pots, use_cells=True)
        t0 = time.time()
        fr.step(50)
        tc = time.time() - t0
        out["cpu_baseline"] = {"value": sub.n_atoms * 50 / tc, "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": "first 16 systems of the stream x 50 FIRE steps, "
                                                           "cell-list mode (atom-steps/s)"}
    return out


def run_row_diff(args):
    """The differentiable workload: 64 reduced-LJ liquid boxes of 864 atoms
    (rho* = 0.8, T* = 1.0 after a Langevin pre-run), NVE 2000 steps at dt* =
    0.005; loss = MSE of the trajectory-averaged 200-bin smeared RDF (to rc)
    against a target from sigma' = 1.05; gradient in (sigma, epsilon) by the
    adjoint over the whole trajectory kept on the device (2001 frames, 2.7 GB:
    no recomputation).  Host wall time of one loss and gradient evaluation;
    the same evaluation with the workload's checkpoints every 100 steps is
    timed beside it (wall_s_checkpoint_100)."""
    import torch
    from paper_2508_06628_b300 import grad, ts, workloads as W
    dev = torch.device("cuda", 0)
    hb = W.lj_liquid(seed=3, n_systems=64, reps=(6, 6, 6), rho=0.8, kT=1.0)
    pot = dict(W.LJ_REDUCED, skin=0.3)
    b = ts.Batch([pot], hb.n_atoms, hb.n_systems, precision=ts.TS_MIXED, device=0)
    s = ts.DeviceState.from_host(hb, device=dev)
    b.neighbor_build(s, force=True)
    b.md_step(s, 500, 0.005, kind=ts.TS_LANGEVIN, gamma=1.0, seed=7)       # melt at T* = 1
    T, every, K, rmax = 2000, 100, 200, 2.5
    tuning, tune_s = b.tuning(), 0.0
    if not args.no_tune:
        # the library's autotuner on NVE steps of a copy of the state, outside the timed region
        t0 = time.time()
        tstream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(tstream):
            trial = ts.DeviceState(*[None if t is None else t.clone() for t in
                                     (s.pos, s.vel, s.mass, s.cell, s.pbc, s.system_idx, s.pot_idx, s.uid, s.kT)])
            tuning = b.autotune(trial, 0.005, kind=ts.TS_NVE, n_steps=25, stream=tstream)
            del trial
        torch.cuda.synchronize()
        tune_s = time.time() - t0
    grad.set_params(b, np.array([[1.05, 1.0, 0.0]]))
    target, _ = grad.trajectory_rdf(b, s, 0.005, T, every, rmax, K)
    grad.set_params(b, np.array([[1.0, 1.0, 0.0]]))
    # on a stream of its own, so that the MD calls replay their CUDA graphs
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        # warm-up: one 200-step evaluation (the first use of each PyTorch kernel
        # on the device costs far more than its run); its gradient is reported
        # too, beside the 2000-step one, to show how the adjoint of a chaotic
        # trajectory grows with its length
        _, _, g200 = grad.rdf_loss_and_grad(b, s, 0.005, 200, every, rmax, K, target)
        g200 = g200.cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, g, gth = grad.rdf_loss_and_grad(b, s, 0.005, T, every, rmax, K, target)
        gh = gth.cpu().numpy()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        # the workload's own protocol: checkpoints every 100 steps, each segment
        # recomputed forward and reversed (same loss and gradient up to rounding)
        t0 = time.perf_counter()
        loss_c, _, gth_c = grad.rdf_loss_and_grad(b, s, 0.005, T, every, rmax, K, target, checkpoint=100)
        gh_c = gth_c.cpu().numpy()
        torch.cuda.synchronize()
        t_c = time.perf_counter() - t0
    b.poll()
    b.close()
    out = _line("trajectory-gradient atom-steps/s (NVE forward + adjoint)", hb.n_atoms * T / t, UNIT,
                 1e3 * t / T, T, 1, "f32",
                 {"workload": "lj-liquid-64x864: rho* 0.8, T* 1.0, NVE dt* 0.005, 2000 steps; 200-bin smeared RDF "
                              "to rc vs sigma' = 1.05 target; d loss / d (sigma, epsilon), trajectory kept on the device",
                  "n_systems": hb.n_systems, "n_atoms": hb.n_atoms,
                  "tuning": dict(tuning, autotuned=not args.no_tune, tune_seconds=round(tune_s, 2))},
                 row="diff", wall_s=t, wall_s_checkpoint_100=t_c,
                 checkpointed_vs_resident_max_rel_diff=float(np.max(np.abs(gh_c[0, :2] - gh[0, :2]) /
                                                                    np.maximum(np.abs(gh[0, :2]), 1e-300))),
                 loss=loss, dloss_dsigma=float(gh[0, 0]), dloss_deps=float(gh[0, 1]),
                 dloss_dsigma_200_steps=float(g200[0, 0]), dloss_deps_200_steps=float(g200[0, 1]))
    if not args.no_cpu:
        from oracle import oracle
        sub = hb.subset([0, 1])
        tgt = target.cpu().numpy()
        t0 = time.time()
        oracle.traj_rdf_loss(sub.offsets, sub.pos, sub.vel, sub.mass, sub.cell, sub.pbc, dict(W.LJ_REDUCED), 0.005,
                             100, 100, rmax, K, tgt, grad=True, use_cells=True)
        tc = time.time() - t0
        out["cpu_baseline"] = {"value": sub.n_atoms * 100 / tc, "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": "2 of the 64 systems (lattice start) x 100 steps, "
                                                           "loss and FP64 adjoint gradient, cell lists"}
    return out


def run_row_large(args):
    """Eight reduced-LJ boxes of 2,048,000 atoms (FCC 80x80x80 at rho* = 0.85,
    MB velocities at T* = 1.2, 0.02 sigma rattle), cell-list rebuild on a 0.3
    sigma skin, NVE at dt* = 0.005 in calls of 50 steps after a Langevin pre-run
    and the library's autotuner (on a copy of the state, outside the timed
    region; the skin scale held at 1, since the workload fixes the skin);
    reports the energy drift per atom over the timed steps."""
    import torch
    from paper_2508_06628_b300 import ts, workloads as W
    dev = torch.device("cuda", 0)
    hb = W.lj_liquid(seed=4, n_systems=8, reps=(80, 80, 80), rho=0.85, kT=1.2, rattle=0.02)
    pots = [dict(hb.pots[0], skin=0.3)]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, precision=ts.TS_MIXED, device=0)
    s = ts.DeviceState.from_host(hb, device=dev)
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device=dev)
    KE = torch.zeros_like(E)
    inner = 50
    n = max(inner, (args.large_steps // inner) * inner)
    stream = torch.cuda.Stream(device=dev)
    tuning, tune_s = b.tuning(), 0.0
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        b.md_step(s, 100, 0.005, kind=ts.TS_LANGEVIN, gamma=1.0, seed=3, stream=stream)   # thermalise
        if not args.no_tune:
            t0 = time.time()
            trial = ts.DeviceState(*[None if t is None else t.clone() for t in
                                     (s.pos, s.vel, s.mass, s.cell, s.pbc, s.system_idx, s.pot_idx, s.uid, s.kT)])
            tuning = b.autotune(trial, 0.005, kind=ts.TS_NVE, n_steps=25, stream=stream)
            del trial
            if tuning["skin_scale"] != 1.0:   # the workload fixes the skin
                tuning = dict(tuning, skin_scale=1.0)
                b.set_tuning(**tuning)
            tune_s = time.time() - t0
        b.md_step(s, inner, 0.005, kind=ts.TS_NVE, E=E, KE=KE, stream=stream)
        stream.synchronize()
        H0 = (E + KE).cpu().numpy()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n // inner):
            b.md_step(s, inner, 0.005, kind=ts.TS_NVE, E=E, KE=KE, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / n
    H1 = (E + KE).cpu().numpy()
    b.poll()
    b.close()
    out = _line("NVE atom-steps/s, 8 boxes of 2,048,000 LJ atoms", hb.n_atoms / (ms / 1e3), UNIT, ms, n, 2, "f32",
                {"workload": "lj-large-8x2048000: FCC 80^3 at rho* 0.85, T* 1.2, rc 2.5 shifted, skin 0.3, "
                             "NVE dt* 0.005", "n_systems": hb.n_systems, "n_atoms": hb.n_atoms,
                 "tuning": dict(tuning, autotuned=not args.no_tune, tune_seconds=round(tune_s, 2))},
                row="large", energy_drift_per_atom_max=float(np.abs(H1 - H0).max() / 2048000),
                energy_drift_steps=n)
    if not args.no_cpu:
        from oracle import oracle
        sub = hb.subset([0])
        t0 = time.time()
        oracle.md(sub.offsets, sub.pos, sub.vel, sub.mass, sub.cell, sub.pbc, sub.pot_idx, sub.pots, 0.005, 2, kind=0,
                  use_cells=True)
        tc = time.time() - t0
        out["cpu_baseline"] = {"value": sub.n_atoms * 2 / tc, "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": "one of the 8 boxes (lattice start) x 2 NVE steps, "
                                                           "cell lists"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--inner", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-loop", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (written by tuning, read at create)")
    ap.add_argument("--large-steps", type=int, default=200, help="NVE steps of the large row (the paper's drift "
                                                                  "protocol runs 10,000)")
    ap.add_argument("--row", default="md", choices=["md", "adjoint", "fire", "nve256", "inflight", "diff", "large",
                                                    "nhc", "npt"],
                    help="md: the MD step (the default line); the others: other rows and workloads, one GPU")
    args = ap.parse_args()
    if args.row != "md":
        rows = {"adjoint": run_row_adjoint, "fire": run_row_fire, "nve256": run_row_nve256,
                "inflight": run_row_inflight, "diff": run_row_diff, "large": run_row_large,
                "nhc": lambda a: run_row_ensemble(a, "nhc"), "npt": lambda a: run_row_ensemble(a, "npt")}
        print(json.dumps(rows[args.row](args)))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    hbcfg = {"workload": f"ragged-mix-{512 * world}: FCC/BCC n x m x k supercells of 32-2048 atoms, 1/3 each LJ "
                         "argon, Morse Cu, soft sphere; 0.05 A rattle, +-5% strained triclinic cells; BAOAB 300 K, "
                         "dt 1 fs" + (f"; 512 systems per GPU on average" if world > 1 else ""),
             "n_systems": 512 * world}
    if args.impl == "reference":
        if rank != 0:
            return
        hb = workload(seed=1)
        # each step: one BAOAB step of a 16-system sample of the workload (about
        # half a second on 16 host threads), so that K + W steps end in minutes
        steps = max(1, min(args.steps, 200))
        cb = cpu_baseline(hb, steps=steps, warmup=max(0, min(args.warmup, 20)))
        line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": cb["steps"],
                "warmup": max(0, min(args.warmup, 20)), "ms_per_step": 1e3 * cb["seconds"] / cb["steps"],
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": dict(hbcfg, n_atoms=hb.n_atoms), "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out, hb = run_ours(args, rank, world)
    if rank == 0:
        cb = None if args.no_cpu else cpu_baseline(hb)
        parity = None if args.no_cpu else oracle_parity(hb, out["final"])
        ms_step = out["ms"] / out["steps"]
        line = {"metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": world, "steps": out["steps"],
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(hbcfg, n_atoms=out["total_atoms"], n_systems=out["total_systems"],
                               md_steps_per_call=out["inner"],
                               l2="flushed (256 MiB write) before every call, outside the timed events",
                               precision="FP32 pair arithmetic, FP64 per-system energy/virial, double-float x and v",
                               energy_virial="not evaluated per BAOAB step (the integrator needs forces only); "
                                             "FP64 per-system energy and virial at the last step of a call when "
                                             "asked for (the e2e leg asks every call)",
                               parallelism=(f"one ragged-mix-{512 * world} workload sharded over {world} GPUs "
                                            f"(atom-balanced, no collective in the step)") if world > 1
                                           else "single GPU",
                               tuning=out["tuning"]),
                "roofline": out["roofline"], "cpu_baseline": cb, "parity": parity, "e2e": out["e2e"],
                "gpu_launches": out["launches"], "relists_in_timed_region": out["relists"],
                "clocks": out["clocks"]}
        if "per_system_loop" in out:
            line["per_system_loop"] = out["per_system_loop"]
            line["batched_over_loop"] = out["value"] / world / out["per_system_loop"]["value"]
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

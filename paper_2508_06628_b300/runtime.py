"""The two autobatchers of TorchSim (arXiv 2508.06628, Sec. 3 and Fig. 3).

* In-flight batched relaxation (variable length): sample systems from a
  stream until the memory budget is full, run a few FIRE steps on the whole
  batch, retire converged systems and admit new ones, until every system has
  converged.  Admission decisions come from the library's scheduler
  (ts_sched_*), data movement from ts_batch_compact_admit, the relaxation
  from ts_fire_step; the host reads back one flag per system per round.
* Binned fixed-length MD: pack the systems into as few bins of the maximum
  memory as ts_bin_pack finds and evolve the bins one after another.

Also HostMD: MD of a batch whose state is held in host memory, its systems
split over streams so that one group's copies overlap another's steps.

Orchestration only: every step of the simulations runs in the library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import parallel, ts

FIRE_DEFAULTS = dict(dt0=0.1, dt_max=1.0, finc=1.1, fdec=0.5, alpha0=0.1, falpha=0.99, maxstep=0.2, fmax=1e-3,
                     smax=1e-4, p_ext=0.0, nmin=5, variable_cell=1)


class HostSystems(C.Structure):
    _fields_ = [("n_systems", C.c_int32), ("n_atoms", C.c_int64), ("pos", C.c_void_p), ("mass", C.c_void_p),
                ("cell", C.c_void_p), ("n_per_system", C.c_void_p), ("pot_idx", C.c_void_p), ("uid", C.c_void_p)]


def fire_params(**kw):
    p = dict(FIRE_DEFAULTS)
    p.update(kw)
    return ts.FireParams(*[p[k] for k in ["dt0", "dt_max", "finc", "fdec", "alpha0", "falpha", "maxstep", "fmax",
                                          "smax", "p_ext"]], p["nmin"], p["variable_cell"])


class _Buffers:
    """One device state of the batch capacity (ping-pong partner of another)."""

    def __init__(self, torch, dev, atoms, systems):
        f = lambda *shape, dt=torch.float64: torch.zeros(shape, dtype=dt, device=dev)
        self.pos, self.vel, self.mass = f(atoms, 3), f(atoms, 3), f(atoms)
        self.cell, self.pbc = f(systems, 3, 3), f(systems, 3, dt=torch.uint8)
        self.sidx, self.pot, self.uid = f(atoms, dt=torch.int32), f(systems, dt=torch.int32), f(systems, dt=torch.int32)
        self.fs = f(systems * ts.FIRE_STATE_BYTES, dt=torch.uint8)
        self.fvel = f(atoms + 3 * systems, 3)
        self.n_systems, self.n_atoms = 0, 0

    def state(self):
        return ts.State(self.n_systems, self.n_atoms, *[C.c_void_p(t.data_ptr()) for t in
                        (self.pos, self.vel, self.mass, self.cell, self.pbc, self.sidx, self.pot, self.uid)])

    def device_state(self):
        n, B = self.n_atoms, self.n_systems
        return ts.DeviceState(self.pos[:n], self.vel[:n], self.mass[:n], self.cell[:B], self.pbc[:B], self.sidx[:n],
                              self.pot[:B], self.uid[:B])


def memory_model(pots, precision=ts.TS_MIXED, max_neighbors=0, device=0):
    """(bytes per atom, bytes per system) of the engine's device scratch for
    these potentials and precision (ts_batch_memory_model of a minimal batch)."""
    b = ts.Batch(pots, 32, 1, precision=precision, max_neighbors=max_neighbors, device=device)
    a, s = C.c_double(), C.c_double()
    b._check(ts.lib().ts_batch_memory_model(b.h, C.byref(a), C.byref(s)), "ts_batch_memory_model")
    b.close()
    return a.value, s.value


def max_scaler_from_budget(probe_atoms, probe_scaler, bytes_per_atom, bytes_per_system, budget_bytes,
                           max_systems=1_000_000):
    """The memory probe of Fig. 2 (ts_estimate_max_scaler) with the engine's
    byte model as its out-of-memory test: copies of probe system k fit while
    bytes_per_atom * atoms + bytes_per_system * systems <= budget_bytes, and
    the largest memory scaler is min_k (copies_k * scaler_k).  Host only.
    Returns (max_scaler, copies per probe system)."""
    n = len(probe_atoms)
    FITS = C.CFUNCTYPE(C.c_int, C.c_double, C.c_int, C.c_void_p)
    L = ts.lib()
    L.ts_estimate_max_scaler.argtypes = [C.c_void_p, C.c_int, FITS, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    copies, best = [], float("inf")
    for k in range(n):   # one probe system at a time: the test knows its atom count
        atoms = float(probe_atoms[k])

        @FITS
        def fits(total, nsys, ctx, atoms=atoms):
            return int(bytes_per_atom * atoms * nsys + bytes_per_system * nsys <= budget_bytes)

        sc = (C.c_double * 1)(float(probe_scaler[k]))
        nfit = (C.c_int * 1)()
        out = C.c_double()
        st = L.ts_estimate_max_scaler(sc, 1, fits, None, int(max_systems), nfit, C.byref(out))
        if st != ts.TS_OK:
            raise ts.TSError(st, f"probe system {k} ({atoms:.0f} atoms) does not fit the budget once")
        copies.append(nfit[0])
        best = min(best, out.value)
    return best, copies


def relax_inflight(hb, pots, max_scaler=None, max_active=1024, n_inner=25, precision=ts.TS_MIXED, max_rounds=10000,
                   device=0, on_round=None, memory_budget_bytes=None, memory_scales_with="n_atoms", **fire_kw):
    """Relax every system of the host batch ``hb`` (workloads.Batch) with
    variable-cell FIRE, admitting systems from the stream while their memory
    fits (Sec. 3, Figs. 2-3).  Memory is either an atom budget ``max_scaler``
    (memory scaling with n_atoms), or a device budget ``memory_budget_bytes``
    turned into a limit on the memory scaler ``memory_scales_with``
    (``n_atoms`` or ``n_atoms_x_density``) by the Fig. 2 probe over the
    largest and the densest systems of the stream, with the engine's byte
    model as the probe's fit test; the batch's atom capacity is what the
    budget leaves after max_active systems' overhead, and admission keeps
    both the scaler and the atoms within their limits.  Returns a dict per
    system id with E, fmax, smax, cell and positions at convergence, and the
    round log (each round's admitted, active, atoms and active scaler)."""
    torch = ts._torch()
    dev = torch.device("cuda", device)
    L = ts.lib()
    L.ts_sched_create.argtypes = [C.c_double, C.c_int32, C.c_void_p]
    L.ts_sched_push.argtypes = [C.c_void_p, C.c_int64, C.c_double]
    L.ts_sched_fill.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    L.ts_sched_retire.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    L.ts_sched_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.ts_sched_destroy.argtypes = [C.c_void_p]
    L.ts_batch_compact_admit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    prm = fire_params(**fire_kw)
    off = hb.offsets
    n_of = np.diff(off)
    scaler = memory_sizes(hb, memory_scales_with)
    if memory_budget_bytes is None:
        if max_scaler is None:
            raise ValueError("give max_scaler or memory_budget_bytes")
        if memory_scales_with != "n_atoms":
            raise ValueError("an atom budget (max_scaler) admits by n_atoms; give memory_budget_bytes otherwise")
        atoms_cap, limit = int(max_scaler), float(max_scaler)
        share = scaler              # in atoms, against the atom budget
    else:
        per_atom, per_sys = memory_model(pots, precision, device=device)
        # what the budget leaves after the systems' overhead, less the layout's
        # rounding of the slot count up to a whole warp
        atoms_cap = int((memory_budget_bytes - per_sys * max_active) / per_atom) - 32
        if atoms_cap < int(n_of.max()):
            raise ts.TSError(ts.TS_ERR_BUDGET, "the budget does not hold the largest system beside the others' overhead")
        probes = sorted({int(np.argmax(n_of)), int(np.argmax(scaler))})
        limit, _ = max_scaler_from_budget(n_of[probes], scaler[probes], per_atom, per_sys, memory_budget_bytes)
        # the scheduler sees one share per system: the larger of its part of
        # the scaler limit and its part of the atom capacity (a sum of these
        # within 1 keeps both sums within their limits)
        share = np.maximum(scaler / limit, n_of / atoms_cap)
    b = ts.Batch(pots, atoms_cap, max_active, precision=precision, device=device,
                 memory_budget_bytes=int(memory_budget_bytes or 0))
    q = C.c_void_p()
    assert L.ts_sched_create(limit if memory_budget_bytes is None else 1.0, int(max_active), C.byref(q)) == 0
    for i in range(hb.n_systems):
        st = L.ts_sched_push(q, i, float(share[i]))
        if st != 0:
            raise ts.TSError(st, f"system {i} ({n_of[i]} atoms) exceeds the budget")
    bufs = [_Buffers(torch, dev, atoms_cap, max_active), _Buffers(torch, dev, atoms_cap, max_active)]
    cur = 0
    ids_active = []
    results, log = {}, []
    ids = (C.c_int64 * max_active)()
    nout = C.c_int()
    stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream)
    conv = torch.zeros(max_active, dtype=torch.uint8, device=dev)
    E = torch.zeros(max_active, dtype=torch.float64, device=dev)
    fm, sm = torch.zeros_like(E), torch.zeros_like(E)
    keep = np.ones(max_active, np.uint8)
    for rnd in range(max_rounds):
        assert L.ts_sched_fill(q, ids, max_active, C.byref(nout)) == 0
        new = [ids[k] for k in range(nout.value)]
        src, dst = bufs[cur], bufs[1 - cur]
        add = None
        if new:
            pos = np.ascontiguousarray(np.concatenate([hb.pos[off[i]:off[i + 1]] for i in new]))
            mass = np.ascontiguousarray(np.concatenate([hb.mass[off[i]:off[i + 1]] for i in new]))
            cell = np.ascontiguousarray(hb.cell[new])
            nps = np.ascontiguousarray(n_of[new].astype(np.int32))
            potidx = np.ascontiguousarray(hb.pot_idx[new].astype(np.int32))
            uid = np.ascontiguousarray(np.array(new, np.uint32))
            keepalive = (pos, mass, cell, nps, potidx, uid)
            add = HostSystems(len(new), int(pos.shape[0]), *[C.c_void_p(a.ctypes.data) for a in keepalive])
        kmask = np.ascontiguousarray(keep[:src.n_systems])
        if not new and not any(kmask):
            break
        sst = src.state()
        dstc = dst.state()
        st = L.ts_batch_compact_admit(b.h, C.byref(sst) if src.n_systems else None,
                                      C.c_void_p(kmask.ctypes.data) if src.n_systems else None,
                                      C.byref(add) if add else None, C.byref(dstc),
                                      C.c_void_p(src.fs.data_ptr()), C.c_void_p(src.fvel.data_ptr()),
                                      C.c_void_p(dst.fs.data_ptr()), C.c_void_p(dst.fvel.data_ptr()), C.byref(prm), sp)
        b._check(st, "ts_batch_compact_admit")
        dst.n_systems, dst.n_atoms = dstc.n_systems, dstc.n_atoms
        ids_active = [i for i, k in zip(ids_active, kmask) if k] + new
        cur = 1 - cur
        buf = bufs[cur]
        s = buf.device_state()
        b.fire_step(s, buf.fs, buf.fvel, prm, n_inner, conv, E, fm, sm)
        c = conv[:buf.n_systems].cpu().numpy().astype(bool)
        log.append(dict(round=rnd, active=len(ids_active), atoms=buf.n_atoms, admitted=len(new), converged=int(c.sum()),
                        scaler=float(scaler[np.asarray(ids_active, dtype=np.int64)].sum()) if ids_active else 0.0))
        if on_round:
            on_round(log[-1])
        done = np.nonzero(c)[0]
        if len(done):
            # gather the converged systems' rows on the device and copy only those
            offs = np.concatenate([[0], np.cumsum(n_of[np.asarray(ids_active, dtype=np.int64)])])
            didx = torch.as_tensor(done, device=dev)
            sc = torch.stack([E[didx], fm[didx], sm[didx]]).cpu().numpy()
            cellh = buf.cell[didx].cpu().numpy()
            rows = np.concatenate([np.arange(offs[k], offs[k + 1]) for k in done])
            posh = buf.pos[torch.as_tensor(rows, device=dev)].cpu().numpy()
            o = 0
            for m, k in enumerate(done):
                i = ids_active[k]
                n = int(offs[k + 1] - offs[k])
                results[i] = dict(E=sc[0, m], fmax=sc[1, m], smax=sc[2, m], cell=cellh[m], pos=posh[o:o + n],
                                  round=rnd)
                o += n
            arr = (C.c_int64 * len(done))(*[ids_active[k] for k in done])
            assert L.ts_sched_retire(q, arr, len(done)) == 0
        keep[:buf.n_systems] = (~c).astype(np.uint8)
    L.ts_sched_destroy(q)
    b.close()
    return results, log


def memory_sizes(hb, memory_scales_with="n_atoms"):
    """Memory footprint of every system in the units of the maximum memory
    (Sec. 3): ``n_atoms``, or ``n_atoms_x_density`` (atoms times atoms per
    A^3, for neighbour counts that grow with density)."""
    n = np.diff(hb.offsets).astype(np.float64)
    if memory_scales_with == "n_atoms":
        return n
    if memory_scales_with == "n_atoms_x_density":
        vol = np.abs(np.linalg.det(hb.cell))
        return n * n / vol
    raise ValueError(f"unknown memory_scales_with {memory_scales_with!r}")


def run_binned(hb, pots, max_scaler, n_steps, dt, kind=ts.TS_LANGEVIN, gamma=0.0, seed=0, inner=10,
               memory_scales_with="n_atoms", precision=ts.TS_MIXED, device=0):
    """Fixed-length MD of every system of ``hb`` (BinningAutobatcher, Sec. 3,
    Fig. 3): pack the systems into bins of ``max_scaler`` (ts_bin_pack) and
    evolve the bins one after another, each for ``n_steps`` steps, through one
    reused batch.  Returns ({system id: dict(pos, vel, E, KE, bin)}, bins)."""
    torch = ts._torch()
    dev = torch.device("cuda", device)
    bins, n_bins = ts.bin_pack(memory_sizes(hb, memory_scales_with), max_scaler)
    members = [np.nonzero(bins == k)[0] for k in range(n_bins)]
    n_of = np.diff(hb.offsets)
    atom_cap = int(max(n_of[m].sum() for m in members))
    sys_cap = int(max(len(m) for m in members))
    b = ts.Batch(pots, atom_cap, sys_cap, precision=precision, device=device)
    stream = torch.cuda.Stream(device=dev)
    results = {}
    for k, ids in enumerate(members):
        sub = hb.subset(ids)
        s = ts.DeviceState.from_host(sub, device=dev)
        E = torch.zeros(sub.n_systems, dtype=torch.float64, device=dev)
        KE = torch.zeros_like(E)
        with torch.cuda.stream(stream):
            b.neighbor_build(s, force=True, stream=stream)   # a new set of systems: new layout
            done = 0
            while done < n_steps:
                m = min(inner, n_steps - done)
                b.md_step(s, m, dt, kind=kind, gamma=gamma, seed=seed, step0=done, E=E, KE=KE, stream=stream)
                done += m
            b.poll(stream)
        stream.synchronize()
        pos, vel, Eh, KEh = s.pos.cpu().numpy(), s.vel.cpu().numpy(), E.cpu().numpy(), KE.cpu().numpy()
        off = sub.offsets
        for j, i in enumerate(ids):
            results[int(i)] = dict(pos=pos[off[j]:off[j + 1]], vel=vel[off[j]:off[j + 1]], E=Eh[j], KE=KEh[j], bin=k)
    b.close()
    return results, bins


def relax_inflight_sharded(hb, pots, group=None, device=None, **kw):
    """relax_inflight over several GPUs, one process per GPU: this rank relaxes
    its shard of the stream (systems balanced by atom count) on its own GPU
    and the results, keyed by the index in ``hb``, are gathered on every rank
    (one all-gather after the work; no collective during it).  ``device``:
    this rank's CUDA device (default: the current one)."""
    torch = ts._torch()
    dev = torch.cuda.current_device() if device is None else device
    return parallel.run_sharded(hb, lambda sub: relax_inflight(sub, pots, device=dev, **kw)[0], group)


def run_binned_sharded(hb, pots, max_scaler, n_steps, dt, group=None, device=None, **kw):
    """run_binned over several GPUs, one process per GPU: this rank bins and
    evolves its shard (systems balanced by atom count); results keyed by the
    index in ``hb`` are gathered on every rank."""
    torch = ts._torch()
    dev = torch.cuda.current_device() if device is None else device
    return parallel.run_sharded(hb, lambda sub: run_binned(sub, pots, max_scaler, n_steps, dt, device=dev, **kw)[0],
                                group)


class HostMD:
    """MD of a batch whose state is held in host memory.

    Each call copies positions and velocities to the device, runs n steps
    there and copies them back, with the per-system energies, so the
    trajectory lives on the host between calls (a caller that reads or edits
    it between calls, or whose data does not fit the device).  The systems are
    split into ``parts`` atom-balanced groups (parallel.shard_systems), each
    its own device batch and CUDA stream with its own pinned host buffers, so
    that one group's copies overlap another group's steps.  Every system keeps
    its index in ``hb`` as its noise id, so its trajectory is the one a single
    batch of all systems gives, up to the summation order of re-listed
    neighbour lists (each group gathers its own re-listings).

    ``tuning``: ts_batch_set_tuning fields for every group (default: the
    library's).  Orchestration only: every step runs in the library."""

    def __init__(self, hb, pots, parts=2, precision=ts.TS_MIXED, device=0, tuning=None):
        torch = ts._torch()
        self._torch = torch
        self.dev = torch.device("cuda", device)
        self.n_systems, self.n_atoms = hb.n_systems, hb.n_atoms
        self.offsets = np.asarray(hb.offsets)
        uid = np.asarray(hb.uid if hb.uid is not None else np.arange(hb.n_systems), np.uint32)
        parts = max(1, min(int(parts), hb.n_systems))
        self.groups = []
        for ids in parallel.shard_systems(np.diff(self.offsets), parts):
            if len(ids) == 0:
                continue
            sub = hb.subset(ids)
            sub.uid = uid[ids]
            b = ts.Batch(pots, sub.n_atoms, sub.n_systems, precision=precision, device=device)
            if tuning:
                b.set_tuning(**tuning)
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            E = torch.zeros(sub.n_systems, dtype=torch.float64, device=self.dev)
            self.groups.append(dict(ids=np.asarray(ids), off=sub.offsets, b=b, s=ts.DeviceState.from_host(sub, self.dev),
                                    stream=torch.cuda.Stream(device=self.dev), pos=pin(sub.pos), vel=pin(sub.vel),
                                    E=E, KE=torch.zeros_like(E), E_h=pin(np.zeros(sub.n_systems)),
                                    KE_h=pin(np.zeros(sub.n_systems))))

    def h2d_bytes(self):
        """Bytes copied to the device per call (positions and velocities)."""
        return 2 * 24 * self.n_atoms

    def d2h_bytes(self):
        """Bytes copied back per call (positions, velocities, E and KE)."""
        return 2 * 24 * self.n_atoms + 2 * 8 * self.n_systems

    def step(self, n_steps, dt, kind=ts.TS_LANGEVIN, gamma=0.0, seed=0, step0=0, after=None):
        """Enqueue one call on every group's stream (returns before it ends):
        copy in, ``n_steps`` steps of ts_md_step, copy out.  ``after``: a CUDA
        event every group waits for first (optional)."""
        for g in self.groups:
            st = g["stream"]
            if after is not None:
                st.wait_event(after)
            with self._torch.cuda.stream(st):
                g["s"].pos.copy_(g["pos"], non_blocking=True)
                g["s"].vel.copy_(g["vel"], non_blocking=True)
                g["b"].md_step(g["s"], n_steps, dt, kind=kind, gamma=gamma, seed=seed, step0=step0, E=g["E"],
                               KE=g["KE"], stream=st)
                g["pos"].copy_(g["s"].pos, non_blocking=True)
                g["vel"].copy_(g["s"].vel, non_blocking=True)
                g["E_h"].copy_(g["E"], non_blocking=True)
                g["KE_h"].copy_(g["KE"], non_blocking=True)

    def join(self, stream):
        """Make ``stream`` wait for every call enqueued so far."""
        for g in self.groups:
            ev = self._torch.cuda.Event()
            ev.record(g["stream"])
            stream.wait_event(ev)

    def synchronize(self):
        for g in self.groups:
            g["stream"].synchronize()
            g["b"].poll(g["stream"])

    def state(self):
        """(pos, vel, E, KE) in the order of ``hb``, as numpy arrays, after
        the calls enqueued so far."""
        self.synchronize()
        pos = np.empty((self.n_atoms, 3)); vel = np.empty((self.n_atoms, 3))
        E = np.empty(self.n_systems); KE = np.empty(self.n_systems)
        for g in self.groups:
            gp, gv = g["pos"].numpy(), g["vel"].numpy()
            for j, i in enumerate(g["ids"]):
                a, e, ga = self.offsets[i], self.offsets[i + 1], g["off"][j]
                pos[a:e] = gp[ga:ga + e - a]; vel[a:e] = gv[ga:ga + e - a]
            E[g["ids"]] = g["E_h"].numpy(); KE[g["ids"]] = g["KE_h"].numpy()
        return pos, vel, E, KE

    def set_state(self, pos=None, vel=None):
        """Replace positions and/or velocities ([n_atoms, 3] in the order of
        ``hb``) in the host buffers; the next call starts from them.  Waits
        for the calls enqueued so far first, since their copies back write
        these buffers."""
        self.synchronize()
        for name, a in (("pos", pos), ("vel", vel)):
            if a is None:
                continue
            a = np.asarray(a, dtype=np.float64)
            if a.shape != (self.n_atoms, 3):
                raise ValueError(f"{name}: shape {a.shape}, expected ({self.n_atoms}, 3)")
            for g in self.groups:
                buf = g[name].numpy()
                for j, i in enumerate(g["ids"]):
                    a0, e, ga = self.offsets[i], self.offsets[i + 1], g["off"][j]
                    buf[ga:ga + e - a0] = a[a0:e]

    def close(self):
        for g in self.groups:
            g["b"].close()
        self.groups = []

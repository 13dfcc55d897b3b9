"""Differentiable simulation on top of libts.so (TorchSim, arXiv 2508.06628,
Sec. 2: backpropagating an observable of a whole trajectory, a radial
distribution function, to the potential parameters).

Orchestration only: forces, their adjoint, the smeared RDF and its gradient,
the MD steps and the reverse velocity-Verlet steps all run in the library's
CUDA kernels.  The loss itself (an MSE on a 200-bin histogram) is the user's
and is computed here with torch on the host-side tensors.
"""
from __future__ import annotations

import numpy as np

from . import parallel, ts


def _torch():
    return ts._torch()


class PairForces:
    """``F, E, stress = PairForces.apply(pos, params, batch, state)``.

    pos [N,3] f64 and params [n_pots,3] f64 are differentiable; backward
    calls ts_pair_forces_backward (gradients through F, E and stress)."""

    @staticmethod
    def _fn():
        torch = _torch()

        class _PF(torch.autograd.Function):
            @staticmethod
            def forward(ctx, pos, params, batch, state):
                set_params(batch, params)
                state.pos = pos.detach().contiguous()
                N, B = state.n_atoms, state.n_systems
                F = torch.zeros((N, 3), dtype=torch.float64, device=pos.device)
                E = torch.zeros(B, dtype=torch.float64, device=pos.device)
                S = torch.zeros((B, 3, 3), dtype=torch.float64, device=pos.device)
                batch.pair_forces(state, F, E, S)
                ctx.batch, ctx.state = batch, state
                ctx.save_for_backward(state.pos, params)
                return F, E, S

            @staticmethod
            def backward(ctx, gF, gE, gS):
                pos, params = ctx.saved_tensors
                b, s = ctx.batch, ctx.state
                s.pos = pos
                set_params(b, params)
                gF = torch.zeros_like(pos) if gF is None else gF.contiguous()
                gPos = torch.zeros_like(pos)
                gPar = torch.zeros_like(params)
                b.pair_forces_backward(s, gF, None if gE is None else gE.contiguous(),
                                       None if gS is None else gS.contiguous(), gPos, gPar)
                return gPos, gPar, None, None

        return _PF

    @classmethod
    def apply(cls, pos, params, batch, state):
        return cls._fn().apply(pos, params, batch, state)


def set_params(batch, params):
    """Push parameters [n_pots,3] (tensor or array) into the batch's potentials."""
    p = params.detach().cpu().numpy() if hasattr(params, "detach") else np.asarray(params)
    pots = [dict(d, p=tuple(float(v) for v in p[k])) for k, d in enumerate(batch.pots)]
    arr = ts.potentials(pots)
    st = ts.lib().ts_batch_set_potentials(batch.h, arr, len(pots))
    batch._check(st, "ts_batch_set_potentials")
    batch.pots = pots


def rdf_mse_upstream(g, target, n_total, n_frames):
    """The loss (1/K) sum_k (g_k - target_k)^2 of the system- and frame-averaged
    RDF g, and its derivative with respect to each system's RDF at each
    observed frame, 2 (g - target) / (K n_total n_frames) (the same row for
    every system).  numpy or torch arrays."""
    K = g.shape[-1]
    d = g - target
    return float((d * d).sum() / K), 2.0 * d / (K * n_total * n_frames)


def trajectory_rdf(batch, state, dt, T, every, rmax, K, checkpoint=None, store=False, group=None, frames=None):
    """NVE velocity Verlet for T steps from ``state`` (not modified); smeared
    RDF averaged over systems and the frames t = every, 2 every, ..., T.
    With several ranks (torch.distributed, ``group``) ``state`` holds this
    rank's systems and the average runs over every rank's systems: one
    all-reduce of the K bin sums.  ``frames`` (optional f64 device tensor
    [T + 1, n_atoms, 3]) receives every frame of the trajectory.  Returns
    (g [K] tensor, checkpoints list of (t, x, v))."""
    torch = _torch()
    n_total = int(parallel.allreduce_sum([state.n_systems], group)[0])
    checkpoint = checkpoint or every
    x = state.pos.clone()
    v = state.vel.clone()
    s = ts.DeviceState(x, v, state.mass, state.cell, state.pbc, state.system_idx, state.pot_idx, state.uid)
    g = torch.zeros(K, dtype=torch.float64, device=x.device)
    gs = torch.zeros((state.n_systems, K), dtype=torch.float64, device=x.device)
    ckpts = [(0, x.clone(), v.clone())] if store else []
    nfr = T // every
    t = 0
    while t < T:
        nxt = min(T, (t // every + 1) * every, (t // checkpoint + 1) * checkpoint)
        if frames is not None:
            batch.md_record(s, frames[t:nxt + 1], dt, kind=ts.TS_NVE)
        else:
            batch.md_step(s, nxt - t, dt, kind=ts.TS_NVE)
        t = nxt
        if t % every == 0:
            batch.rdf(s, rmax, K, gs)
            g += gs.sum(0) / (n_total * nfr)
        if store and t % checkpoint == 0 and t < T:
            ckpts.append((t, s.pos.clone(), s.vel.clone()))
    if parallel.rank_world(group)[1] > 1:
        g = torch.as_tensor(parallel.allreduce_sum(g.cpu().numpy(), group), device=x.device)
    return g, ckpts


def rdf_loss_and_grad(batch, state, dt, T, every, rmax, K, target, checkpoint=None, group=None,
                      store_budget_bytes=None):
    """Loss = (1/K) sum_k (g_k - target_k)^2 of the trajectory-averaged smeared
    RDF, and d loss / d params [n_pots,3] by the discrete adjoint of velocity
    Verlet.  With ``checkpoint=None`` the whole trajectory (T + 1 frames of
    24 bytes per atom) stays on the device when it fits in
    ``store_budget_bytes`` (default: half the free device memory), and one
    reverse sweep runs over it; otherwise, or with an explicit interval, the
    forward pass keeps checkpoints every ``checkpoint`` steps (100 by default)
    and the reverse recomputes each segment forward before reversing it.
    With several ranks (``group``), ``state`` holds this rank's systems: the
    averaged RDF takes one all-reduce of K sums, and the parameter gradient
    one all-reduce of n_pots x 3 sums (for one LJ potential, dL/dsigma and
    dL/depsilon); every rank returns the global loss and gradient."""
    torch = _torch()
    N = state.n_atoms
    stored = None
    if checkpoint is None:
        need = (T + 1) * N * 3 * 8
        budget = store_budget_bytes
        if budget is None:
            budget = torch.cuda.mem_get_info(state.pos.device)[0] // 2
        if need <= budget:
            stored = torch.empty((T + 1, N, 3), dtype=torch.float64, device=state.pos.device)
        else:
            checkpoint = 100
    if stored is not None:
        g, _ = trajectory_rdf(batch, state, dt, T, every, rmax, K, group=group, frames=stored)
        ckpts = [(0, None, None)]
    else:
        g, ckpts = trajectory_rdf(batch, state, dt, T, every, rmax, K, checkpoint, store=True, group=group)
    target = torch.as_tensor(target, dtype=torch.float64, device=g.device)
    nfr = T // every
    n_total = int(parallel.allreduce_sum([state.n_systems], group)[0])
    loss, up = rdf_mse_upstream(g, target, n_total, nfr)
    gg = up.expand(state.n_systems, K).contiguous()
    ax = torch.zeros((N, 3), dtype=torch.float64, device=g.device)
    av = torch.zeros_like(ax)
    gth = torch.zeros((len(batch.pots), 3), dtype=torch.float64, device=g.device)
    bounds = [c[0] for c in ckpts] + [T]
    if stored is not None:   # one sweep over the stored trajectory, nothing recomputed
        batch.vv_adjoint_segment(state, stored, 0, dt, ax, av, gth, rdf_every=every, rmax=rmax, K=K, gg=gg)
        ckpts = []
    frames = None
    for seg in range(len(ckpts) - 1, -1, -1):
        t0, x0, v0 = ckpts[seg]
        t1 = bounds[seg + 1]
        # the segment recomputed forward with every frame recorded (one
        # library call), then reversed in one library call (RDF gradients at
        # the observed frames)
        if frames is None or frames.shape[0] < t1 - t0 + 1:
            frames = torch.empty((t1 - t0 + 1, N, 3), dtype=torch.float64, device=g.device)
        fr = frames[:t1 - t0 + 1]
        s = ts.DeviceState(x0.clone(), v0.clone(), state.mass, state.cell, state.pbc, state.system_idx,
                           state.pot_idx, state.uid)
        batch.md_record(s, fr, dt, kind=ts.TS_NVE)
        batch.vv_adjoint_segment(state, fr, t0, dt, ax, av, gth, rdf_every=every, rmax=rmax, K=K, gg=gg)
    if parallel.rank_world(group)[1] > 1:
        gth = torch.as_tensor(parallel.allreduce_sum(gth.cpu().numpy(), group), device=g.device)
    return loss, g, gth


def fit_rdf(batch, state, target, dt, T, every, rmax, K, iters=10, lr=0.02, fit=((0, 0), (0, 1)),
            checkpoint=100, on_iter=None):
    """Differentiable fitting of potential parameters to a target RDF (Sec. 2,
    ref. [19]): Adam on the entries ``fit`` (pot index, parameter index) of the
    batch's parameters, every iteration a fresh trajectory from ``state``
    (not modified) and its checkpointed adjoint (rdf_loss_and_grad).  Steps
    are scaled by each parameter's starting magnitude (``lr`` is relative);
    the step is halved whenever the loss rises (the moments carry the search
    past a minimum otherwise).  Returns (the parameters with the lowest loss
    [n_pots, 3] numpy, history of (loss, parameters))."""
    params = np.array([list(p["p"]) for p in batch.pots], dtype=np.float64)
    mask = np.zeros_like(params)
    for q, c in fit:
        mask[q, c] = 1.0
    scale = np.abs(params) * mask
    m = np.zeros_like(params)
    v = np.zeros_like(params)
    b1, b2, eps = 0.9, 0.999, 1e-12
    history = []
    best = (np.inf, params.copy())
    for it in range(iters):
        set_params(batch, params)
        loss, _, gth = rdf_loss_and_grad(batch, state, dt, T, every, rmax, K, target, checkpoint=checkpoint)
        history.append((loss, params.copy()))
        if on_iter:
            on_iter(it, loss, params)
        if len(history) > 1 and loss > history[-2][0]:
            lr *= 0.5
        if loss < best[0]:
            best = (loss, params.copy())
        g = gth.cpu().numpy() * scale              # gradient in relative units of each parameter
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** (it + 1))
        vh = v / (1 - b2 ** (it + 1))
        params = params - lr * scale * mh / (np.sqrt(vh) + eps)
    set_params(batch, best[1])
    return best[1], history


def hessian_vector_product(batch, state, v, stream=None):
    """H v, H = d2E/dx2 of the batch's potential energy (block diagonal over
    systems), for a direction v [n_atoms, 3] (device, FP64).  The pair-force
    adjoint with gF = v returns d<v, F>/dx = (dF/dx)^T v = -H v (F = -dE/dx,
    H symmetric), so one backward launch gives one product (second-order work
    of the kind phonon and elastic-constant codes need, Sec. 5).  The
    neighbour list must be current (call neighbor_build first)."""
    torch = _torch()
    g = torch.zeros_like(state.pos)
    batch.pair_forces_backward(state, v.contiguous(), None, None, gPos=g, stream=stream)
    return -g


def hessian_blocks(batch, state, stream=None):
    """The Hessian block of every system, [3 n_s, 3 n_s] numpy arrays (A, eV/A^2),
    from 3 * max_s n_s products: product (a, c) displaces local atom a along
    axis c in every system at once."""
    torch = _torch()
    off = state.offsets_host()
    n = np.diff(off)
    N = int(off[-1])
    blocks = [np.zeros((3 * k, 3 * k)) for k in n]
    for a in range(int(n.max())):
        for c in range(3):
            v = torch.zeros((N, 3), dtype=torch.float64, device=state.pos.device)
            rows = torch.as_tensor(off[:-1][n > a] + a, device=v.device)
            v[rows, c] = 1.0
            hv = hessian_vector_product(batch, state, v, stream=stream).cpu().numpy()
            for s in np.nonzero(n > a)[0]:
                blocks[s][:, 3 * a + c] = hv[off[s]:off[s + 1]].reshape(-1)
    return blocks


def gamma_frequencies(block, mass):
    """Phonon angular frequencies at Gamma of one system (rad per internal time
    unit; sqrt of the eigenvalues of M^-1/2 H M^-1/2, negative for unstable
    modes), from its Hessian block and masses [n_s]."""
    w = 1.0 / np.sqrt(np.repeat(np.asarray(mass, np.float64), 3))
    d = 0.5 * (block + block.T) * w[:, None] * w[None, :]
    lam = np.linalg.eigvalsh(d)
    return np.sign(lam) * np.sqrt(np.abs(lam))


# Voigt order of stress and strain components: xx, yy, zz, yz, xz, xy
VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def elastic_constants(pots, state, delta=1e-5, precision=ts.TS_FP64, device=None):
    """Stress-strain coefficients C_ij = d sigma_i / d eps_j [B,6,6] (Voigt
    xx, yy, zz, yz, xz, xy; eV/A^3; engineering shear strains) of every
    system of ``state`` at its configuration, by central differences of the
    stress under the homogeneous strains x -> x (I + eps), h -> h (I + eps),
    eps = +-delta along each Voigt component, without internal relaxation
    (elastic constants are among the second-order properties the paper lists
    as next, Sec. 5).  All 12 strained copies of every system are evaluated
    in one batched ts_pair_forces call in a batch of their own; at zero
    stress C is the elastic-constant matrix.  ``state`` is not modified."""
    torch = _torch()
    pos, cell = state.pos, state.cell
    dev = pos.device if device is None else device
    B, N = state.n_systems, state.n_atoms
    M = torch.zeros((12, 3, 3), dtype=torch.float64, device=dev)
    for j, (a, b) in enumerate(VOIGT):
        for c, sgn in enumerate((1.0, -1.0)):
            e = torch.zeros((3, 3), dtype=torch.float64)
            if a == b:
                e[a, a] = sgn * delta
            else:
                e[a, b] = e[b, a] = 0.5 * sgn * delta
            M[2 * j + c] = (torch.eye(3, dtype=torch.float64) + e).to(dev)
    copies = torch.arange(12, device=dev, dtype=torch.int32)
    big = ts.DeviceState(
        torch.einsum("na,cab->cnb", pos.to(dev), M).reshape(12 * N, 3).contiguous(),
        None, state.mass.to(dev).repeat(12).contiguous(),
        torch.einsum("sab,cbd->csad", cell.to(dev), M).reshape(12 * B, 3, 3).contiguous(),
        state.pbc.to(dev).repeat(12, 1).contiguous(),
        (state.system_idx.to(dev)[None, :] + B * copies[:, None]).reshape(-1).contiguous(),
        state.pot_idx.to(dev).repeat(12).contiguous(), None)
    b = ts.Batch(pots, 12 * N, 12 * B, precision=precision, device=dev.index if dev.index is not None else 0)
    S = torch.zeros((12 * B, 3, 3), dtype=torch.float64, device=dev)
    b.pair_forces(big, None, None, S)
    b.poll()
    b.close()
    S = S.view(12, B, 3, 3)
    C = torch.zeros((B, 6, 6), dtype=torch.float64, device=dev)
    for j in range(6):
        dS = (S[2 * j] - S[2 * j + 1]) / (2.0 * delta)
        for i, (a, b_) in enumerate(VOIGT):
            C[:, i, j] = dS[:, a, b_]
    return C

"""GPU parity of the differentiable path: pair-force adjoint, smeared RDF and
its gradient, and the trajectory gradient through velocity Verlet."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import frac_diff, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_pair_backward_matches_oracle(orc, precision):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(71, n_systems=6, lo=32, hi=300)
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    rng = np.random.default_rng(0)
    gF = rng.normal(size=(hb.n_atoms, 3))
    gE = rng.normal(size=hb.n_systems)
    gS = rng.normal(size=(hb.n_systems, 3, 3))
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
    gx = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    gp = torch.zeros((len(hb.pots), 3), dtype=torch.float64, device="cuda")
    b.pair_forces_backward(s, t(gF), t(gE), t(gS), gx, gp)
    b.poll()
    pos = s.pos.cpu().numpy()
    gxr, gpr = orc.forces_backward(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots, gF, gE, gS)
    gx, gp = gx.cpu().numpy(), gp.cpu().numpy()
    rel = 1e-9 if precision == 1 else 1e-4
    scale = np.abs(gxr).max()
    assert np.abs(gx - gxr).max() <= rel * scale
    assert np.all(np.abs(gp - gpr) <= rel * np.abs(gpr) + rel * 1e-2 * np.abs(gpr).max())


@pytest.mark.parametrize("with_stress", [False, True])
def test_pair_backward_small_and_large_systems(orc, with_stress):
    """Mixed precision: without a stress upstream the systems of up to 2048
    atoms take the shared-memory backward and a 2304-atom system the gather
    kernel in the same call; with one, every system takes the gather kernel.
    Both against the oracle."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    rng = np.random.default_rng(9)
    p, c = W.lattice("fcc", (8, 8, 9), 5.26)
    c2 = c @ (np.eye(3) + np.array([[0, 0.03, 0], [0.01, 0, 0], [0, 0.02, 0]]))
    p = p @ np.linalg.solve(c, c2) + rng.normal(0, 0.05, p.shape)
    big = dict(pos=p, vel=np.zeros_like(p), mass=np.full(len(p), 39.948), cell=c2, pot=0)
    small = small_mix(19, n_systems=5, lo=32, hi=600)
    systems = [dict(pos=small.pos[small.offsets[k]:small.offsets[k + 1]],
                    vel=np.zeros((small.offsets[k + 1] - small.offsets[k], 3)),
                    mass=small.mass[small.offsets[k]:small.offsets[k + 1]], cell=small.cell[k],
                    pot=int(small.pot_idx[k])) for k in range(5)]
    hb = W.concat(systems[:2] + [big] + systems[2:], small.pots)
    b = make_batch(hb, 0)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    gF = rng.normal(size=(hb.n_atoms, 3))
    gE = rng.normal(size=hb.n_systems)
    gS = rng.normal(size=(hb.n_systems, 3, 3)) if with_stress else None
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
    gx = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    gp = torch.zeros((len(hb.pots), 3), dtype=torch.float64, device="cuda")
    b.pair_forces_backward(s, t(gF), t(gE), t(gS) if with_stress else None, gx, gp)
    b.poll()
    gxr, gpr = orc.forces_backward(hb.offsets, s.pos.cpu().numpy(), hb.cell, hb.pbc, hb.pot_idx, hb.pots, gF, gE,
                                   gS if with_stress else np.zeros((hb.n_systems, 3, 3)), use_cells=True)
    gx, gp = gx.cpu().numpy(), gp.cpu().numpy()
    assert np.abs(gx - gxr).max() <= 1e-4 * np.abs(gxr).max()
    assert np.all(np.abs(gp - gpr) <= 1e-4 * np.abs(gpr) + 1e-6 * np.abs(gpr).max())
    b.close()


def backward_after_md(hb, precision, with_stress):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    rng = np.random.default_rng(6)
    gF, gE, gS = rng.normal(size=(hb.n_atoms, 3)), rng.normal(size=hb.n_systems), rng.normal(size=(hb.n_systems, 3, 3))
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
    gx = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    gp = torch.zeros((len(hb.pots), 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        b.md_step(s, 40, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=4, stream=stream)
        b.pair_forces_backward(s, t(gF), t(gE), t(gS) if with_stress else None, gx, gp, stream=stream)
        b.poll(stream)
    stream.synchronize()
    out = s.pos.cpu().numpy(), gx.cpu().numpy(), gp.cpu().numpy(), b.prunes(), (gF, gE, gS if with_stress else None)
    b.close()
    return out


@pytest.mark.parametrize("precision,with_stress", [(0, False), (0, True), (1, False), (1, True)])
def test_pair_backward_after_md_uses_inner_lists(orc, monkeypatch, precision, with_stress):
    """After MD steps the backward reads the pruned (inner) lists; with
    TS_INNER=1 the inner list is the whole Verlet list, so the two runs must
    agree bit for bit, and both with the oracle at the final positions."""
    hb = small_mix(72, n_systems=8, lo=32, hi=500)
    xa, gxa, gpa, pa, (gF, gE, gS) = backward_after_md(hb, precision, with_stress)
    monkeypatch.setenv("TS_INNER", "1")
    xb, gxb, gpb, _, _ = backward_after_md(hb, precision, with_stress)
    assert pa > 0
    assert np.array_equal(xa, xb)
    assert np.array_equal(gxa, gxb) and np.array_equal(gpa, gpb)
    gxr, gpr = orc.forces_backward(hb.offsets, xa, hb.cell, hb.pbc, hb.pot_idx, hb.pots, gF, gE, gS)
    rel = 1e-9 if precision == 1 else 1e-4
    assert np.abs(gxa - gxr).max() <= rel * np.abs(gxr).max()
    assert np.all(np.abs(gpa - gpr) <= rel * np.abs(gpr) + rel * 1e-2 * np.abs(gpr).max())


@pytest.mark.parametrize("precision", [0, 1])
def test_rdf_and_its_gradient(orc, precision):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = W.lj_liquid(seed=2, n_systems=3, reps=(3, 3, 3), rattle=0.12)
    pots = [dict(hb.pots[0], skin=0.3)]
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, precision=precision)
    s = ts.DeviceState.from_host(hb)
    K, rmax = 200, 2.5
    g = torch.zeros((hb.n_systems, K), dtype=torch.float64, device="cuda")
    b.neighbor_build(s, force=True)
    b.rdf(s, rmax, K, g)
    gg = np.random.default_rng(1).normal(size=(hb.n_systems, K))
    gx = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    b.rdf_backward(s, rmax, K, torch.as_tensor(gg, device="cuda"), gx)
    b.poll()
    pos = s.pos.cpu().numpy()
    gr, gxr = orc.rdf(hb.offsets, pos, hb.cell, hb.pbc, rmax, K=K, gg=gg)
    rel = 1e-5 if precision == 0 else 1e-9
    assert np.abs(g.cpu().numpy() - gr).max() <= rel * np.abs(gr).max() + 1e-12
    assert np.abs(gx.cpu().numpy() - gxr).max() <= (1e-4 if precision == 0 else 1e-8) * np.abs(gxr).max()


@pytest.mark.parametrize("precision,checkpoint", [(1, 20), (0, 20), (1, None), (0, None)])
def test_trajectory_gradient_matches_oracle(orc, precision, checkpoint):
    """d loss / d (sigma, eps) through 60 NVE steps with RDF frames every 20
    steps: the GPU adjoint with checkpoints every 20 steps (segments
    recomputed) or over the whole trajectory kept on the device (one sweep)
    vs the oracle's stored-trajectory adjoint."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import grad, ts
    hb = W.lj_liquid(seed=3, n_systems=2, reps=(2, 2, 3), rattle=0.08, kT=0.5)
    pot = dict(W.LJ_REDUCED)
    K, rmax, T, every, dt = 50, 2.5, 60, 20, 0.005
    _, target, _ = orc.traj_rdf_loss(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, dict(pot, p=(1.05, 1.0, 0.0)),
                                     dt, T, every, rmax, K, np.zeros(K), grad=False)
    lr, gr, gthr = orc.traj_rdf_loss(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, pot, dt, T, every, rmax, K,
                                     target)
    b = ts.Batch([dict(pot, skin=0.4)], hb.n_atoms, hb.n_systems, precision=precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    loss, g, gth = grad.rdf_loss_and_grad(b, s, dt, T, every, rmax, K, target, checkpoint=checkpoint)
    b.poll()
    gth = gth.cpu().numpy()[0]
    rel = 1e-7 if precision == 1 else 1e-4
    assert loss == pytest.approx(lr, rel=rel * 10)
    assert np.abs(g.cpu().numpy() - gr).max() <= rel * 10 * np.abs(gr).max()
    for q in (0, 1):
        assert gth[q] == pytest.approx(gthr[q], rel=rel)


def test_pair_forces_autograd_function(orc):
    """torch.autograd through PairForces: d(sum w.F)/dx and /dparams equal the
    ABI adjoint, and a finite difference of the energy in eps."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import grad, ts
    hb = small_mix(81, n_systems=3, lo=32, hi=128)
    b = make_batch(hb, 1)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    pos = s.pos.clone().requires_grad_(True)
    params = torch.tensor([list(p["p"]) for p in hb.pots], dtype=torch.float64, device="cuda", requires_grad=True)
    F, E, S = grad.PairForces.apply(pos, params, b, s)
    E.sum().backward()
    # dE/dx = -F
    assert torch.allclose(pos.grad, -F.detach(), atol=1e-10)
    # dE/deps of the LJ potential by central differences
    h = 1e-6
    Es = []
    for sgn in (1, -1):
        p2 = params.detach().clone()
        p2[0, 1] += sgn * h * p2[0, 1]
        _, E2, _ = grad.PairForces.apply(s.pos.clone(), p2, b, s)
        Es.append(E2.sum().item())
    fd = (Es[0] - Es[1]) / (2 * h * params[0, 1].item())
    assert params.grad[0, 1].item() == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("precision", [1, 0])
def test_adjoint_segment_equals_step_loop(precision):
    """ts_vv_adjoint_segment over 30 stored frames with RDF gradients at every
    10th frame gives the adjoints and parameter gradient of the same reverse
    steps issued one call at a time: the segment merges the half kicks of
    adjacent reverse steps (one backward pass per frame with weight dt instead
    of two with dt/2), which changes only the order of the additions, so the
    results agree to rounding.  On a side stream the first call is issued
    directly, the second captured as a CUDA graph and launched, the third
    replayed: each equals the directly issued call bit for bit, call for call
    (a later call starts from the lists the previous one left)."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = W.lj_liquid(seed=5, n_systems=3, reps=(2, 2, 3), rattle=0.08, kT=0.5)
    pot = dict(W.LJ_REDUCED, skin=0.4)
    K, rmax, dt, n, every, t0 = 50, 2.5, 0.005, 30, 10, 40
    rng = np.random.default_rng(11)
    gg = torch.as_tensor(rng.normal(size=(hb.n_systems, K)), device="cuda")
    ax0 = torch.as_tensor(rng.normal(size=(hb.n_atoms, 3)), device="cuda")
    av0 = torch.as_tensor(rng.normal(size=(hb.n_atoms, 3)), device="cuda")

    def setup():
        b = ts.Batch([pot], hb.n_atoms, hb.n_systems, precision=precision)
        s = ts.DeviceState.from_host(hb)
        b.neighbor_build(s, force=True)
        frames = torch.empty((n + 1, hb.n_atoms, 3), dtype=torch.float64, device="cuda")
        frames[0].copy_(s.pos)
        for m in range(1, n + 1):
            b.md_step(s, 1, dt, kind=ts.TS_NVE)
            frames[m].copy_(s.pos)
        return b, s, frames

    def segment(b, s, frames, stream=None):
        ax, av = ax0.clone(), av0.clone()
        gth = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
        b.vv_adjoint_segment(s, frames, t0, dt, ax, av, gth, rdf_every=every, rmax=rmax, K=K, gg=gg, stream=stream)
        b.poll(stream)
        return ax.cpu().numpy(), av.cpu().numpy(), gth.cpu().numpy()

    b, s, frames = setup()
    res_seg = segment(b, s, frames)      # legacy default stream: issued directly
    res_seg2 = segment(b, s, frames)
    res_seg3 = segment(b, s, frames)
    b.close()

    b, s, frames = setup()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        res_dir = segment(b, s, frames, stream)
        res_cap = segment(b, s, frames, stream)
        res_rep = segment(b, s, frames, stream)
    b.close()
    for a, a2, a3, c, d, e in zip(res_seg, res_seg2, res_seg3, res_dir, res_cap, res_rep):
        assert np.array_equal(a, c) and np.array_equal(a2, d) and np.array_equal(a3, e)

    b, s, frames = setup()
    ax, av = ax0.clone(), av0.clone()
    gth = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    for m in range(n, 0, -1):
        if (t0 + m) % every == 0:
            sn = ts.DeviceState(frames[m], None, s.mass, s.cell, s.pbc, s.system_idx, s.pot_idx, s.uid)
            b.rdf_backward(sn, rmax, K, gg, ax)
        st = ts.DeviceState(frames[m - 1], None, s.mass, s.cell, s.pbc, s.system_idx, s.pot_idx, s.uid)
        b.vv_adjoint_step(st, frames[m], dt, ax, av, gth)
    b.poll()
    res_loop = ax.cpu().numpy(), av.cpu().numpy(), gth.cpu().numpy()
    b.close()
    assert np.abs(res_seg[0]).max() > 0 and np.abs(res_seg[2]).max() > 0
    for a, c in zip(res_seg, res_loop):
        assert np.abs(a - c).max() <= 1e-11 * np.abs(c).max()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_md_record_rows_equal_shorter_calls(orc, precision, kind):
    """ts_md_record (velocity Verlet, BAOAB, Nose-Hoover chain): row k of the
    frames equals the positions after a ts_md_step call of k steps from the
    same state (bit for bit), its last row equals the returned positions, and
    in FP64 mode the rows follow the oracle's trajectory."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(83, n_systems=5, lo=32, hi=400)
    dt, n, tau = hb.meta["dt"], 12, 50.0
    kT = torch.as_tensor(hb.kT, dtype=torch.float64, device="cuda")

    def md_kw():   # the chain state starts at zero for every run
        kw = dict(kind=kind, gamma=hb.meta["gamma"] if kind == 1 else 0.0, seed=4, kT=kT)
        if kind == 2:
            kw.update(tau=tau, nhc=torch.zeros((hb.n_systems, 6), dtype=torch.float64, device="cuda"))
        return kw

    def fresh():
        b = make_batch(hb, precision)
        s = ts.DeviceState.from_host(hb)
        b.neighbor_build(s, force=True)
        return b, s

    b, s = fresh()
    frames = torch.full((n + 1, hb.n_atoms, 3), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    md = md_kw()
    with torch.cuda.stream(stream):
        b.md_record(s, frames, dt, stream=stream, **md)
        b.poll(stream)
    torch.cuda.synchronize()
    fr = frames.cpu().numpy()
    assert np.isfinite(fr).all()
    assert np.array_equal(fr[n], s.pos.cpu().numpy())
    # the replayed graph writes into another buffer: the frames base is read on the device
    frames2 = torch.full_like(frames, float("nan"))
    with torch.cuda.stream(stream):
        b.md_record(s, frames2, dt, stream=stream, step0=n, **md)
        b.poll(stream)
    torch.cuda.synchronize()
    fr2 = frames2.cpu().numpy()
    assert np.isfinite(fr2).all() and np.array_equal(fr2[0], fr[n]) and np.array_equal(fr2[n], s.pos.cpu().numpy())
    assert np.array_equal(frames.cpu().numpy(), fr)
    b.close()
    for k in (1, 5, n):
        b, s = fresh()
        b.md_step(s, k, dt, **md_kw())
        b.poll()
        assert np.array_equal(fr[k], s.pos.cpu().numpy()), k
        b.close()
    if precision == 1:
        for k in (1, n):
            if kind == 2:
                xr = orc.md_nhc(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots, dt, k,
                                hb.kT, tau)[0]
            else:
                xr = orc.md(hb.offsets, hb.pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots, dt, k,
                            kind=kind, kT=hb.kT, gamma=hb.meta["gamma"] if kind == 1 else 0.0, seed=4,
                            uid=hb.uid)[0]
            assert np.abs(frac_diff(fr[k], xr, hb.cell, hb.offsets)).max() < 1e-9
    # NPT is not recorded
    b, s = fresh()
    with pytest.raises(ts.TSError) as ei:
        b.md_record(s, frames, dt, kind=ts.TS_NPT_LANGEVIN)
    assert ei.value.status == ts.TS_ERR_INVALID_ARG
    b.close()

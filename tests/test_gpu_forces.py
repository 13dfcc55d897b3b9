"""GPU parity of the neighbour build and the fused pair kernel against the FP64
oracle, through the C ABI (libts.so)."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import force_tolerance_ok, kinds_of, frac_diff, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def run_forces(hb, precision, max_neighbors=0):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision, max_neighbors=max_neighbors)
    s = ts.DeviceState.from_host(hb)
    F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    S = torch.zeros((hb.n_systems, 3, 3), dtype=torch.float64, device="cuda")
    b.neighbor_build(s, force=True)
    b.pair_forces(s, F, E, S)
    b.poll()
    return b, s, F.cpu().numpy(), E.cpu().numpy(), S.cpu().numpy(), s.pos.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("seed", [11, 12])
def test_pair_forces_parity(orc, precision, seed):
    hb = small_mix(seed)
    b, s, F, E, S, pos = run_forces(hb, precision)
    # the wrapped positions are the input positions up to lattice vectors
    assert np.abs(frac_diff(pos, hb.pos, hb.cell, hb.offsets)).max() < 1e-9
    Er, Fr, Sr = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F, Fr, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    if precision == 1:
        assert np.allclose(E, Er, rtol=1e-9, atol=1e-12)
        assert np.allclose(S, Sr, rtol=1e-9, atol=1e-14)
    else:
        assert np.all(np.abs(E - Er) <= 1e-6 * np.abs(Er) + 1e-9)
        for k in range(hb.n_systems):
            assert np.abs(S[k] - Sr[k]).max() <= 1e-5 * np.abs(Sr[k]).max() + 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_pair_sets_identical(orc, precision):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(21, n_systems=8, lo=32, hi=256)
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    j, img, cnt = b.neighbor_export(s)
    b.poll()
    j, img, cnt, pos = j.cpu().numpy(), img.cpu().numpy(), cnt.cpu().numpy(), s.pos.cpu().numpy()
    off = hb.offsets
    for k in range(hb.n_systems):
        a, e = off[k], off[k + 1]
        pot = hb.pots[hb.pot_idx[k]]
        rl = (pot["rc"] if pot["kind"] != 2 else pot["p"][0]) + ts.default_skins([pot])[0]
        ref = orc.neighbors(pos[a:e], hb.cell[k], [1, 1, 1], rl)
        h = hb.cell[k]

        def near_cut(i, jj, n):
            d = pos[a + jj] - pos[a + i] + np.asarray(n) @ h
            return abs(np.linalg.norm(d) - rl) < 1e-6

        R = {(int(p[0]), int(p[1]), *map(int, p[2:])) for p in ref if not near_cut(p[0], p[1], p[2:])}
        G = set()
        for i in range(a, e):
            for q in range(cnt[i]):
                t = (i - a, int(j[i, q]) - a, *map(int, img[i, q]))
                if not near_cut(t[0], t[1], t[2:]):
                    G.add(t)
        assert G == R, f"system {k}: {len(G ^ R)} pairs differ"


def test_batch_invariance_and_determinism():
    hb = small_mix(31, n_systems=6)
    _, _, F1, E1, S1, _ = run_forces(hb, 0)
    _, _, F2, E2, S2, _ = run_forces(hb, 0)
    assert np.array_equal(F1, F2) and np.array_equal(E1, E2) and np.array_equal(S1, S2)
    sub = hb.subset([3])
    _, _, Fs, Es, Ss, _ = run_forces(sub, 0)
    o = hb.offsets
    assert np.array_equal(Fs, F1[o[3]:o[4]]) and Es[0] == E1[3] and np.array_equal(Ss[0], S1[3])


@pytest.mark.parametrize("precision", [0, 1])
def test_edge_cases(orc, precision):
    """1-atom cells (self images only), tiny triclinic cells reaching 4
    images, a ragged tail of 33 atoms, and a dilute system in one bin."""
    rng = np.random.default_rng(5)
    systems = []
    # one atom in a 3 A sheared cube with LJ argon: r_list 9.51 A -> reach 4 (self images only)
    systems.append(dict(pos=np.array([[0.3, 0.2, 0.1]]), vel=np.zeros((1, 3)), mass=np.array([39.948]),
                        cell=np.eye(3) * 3.0 + np.array([[0, 0.2, 0], [0, 0, 0], [0.1, 0, 0]]), pot=0))
    # 33 atoms of Cu in a sheared cell
    p, c = W.lattice("fcc", (2, 2, 2), 3.61)
    p = np.concatenate([p, p[:1] + 1.8])
    c = c @ (np.eye(3) + np.array([[0, 0.08, 0], [0.02, 0, 0], [0, 0.05, 0]]))
    systems.append(dict(pos=p + rng.normal(0, 0.05, p.shape), vel=np.zeros_like(p), mass=np.full(33, 63.546), cell=c, pot=1))
    # dilute soft spheres: a few atoms in a big box, with overlaps
    q = rng.uniform(0, 3.0, (5, 3))
    systems.append(dict(pos=q, vel=np.zeros_like(q), mass=np.ones(5), cell=np.eye(3) * 3.0, pot=2))
    hb = W.concat(systems, [W.LJ_AR, W.MORSE_CU, W.SOFT_SPHERE])
    b, s, F, E, S, pos = run_forces(hb, precision, max_neighbors=256)
    Er, Fr, Sr = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F, Fr, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    assert np.allclose(E, Er, rtol=1e-6 if precision == 0 else 1e-9, atol=1e-9)


def test_bad_system_idx_is_rejected():
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(41, n_systems=3)
    b = make_batch(hb, 0)
    s = ts.DeviceState.from_host(hb)
    s.system_idx = s.system_idx.flip(0).contiguous()
    with pytest.raises(ts.TSError) as e:
        b.neighbor_build(s, force=True)
    assert e.value.status == ts.TS_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_large_system_path(orc, precision):
    """A 2304-atom system (multi-kernel re-listing path) next to small ones
    (fused per-system path): pair sets and forces match the oracle."""
    rng = np.random.default_rng(8)
    p, c = W.lattice("fcc", (8, 8, 9), 5.26)
    c2 = c @ (np.eye(3) + np.array([[0, 0.03, 0], [0.01, 0, 0], [0, 0.02, 0]]))
    p = p @ np.linalg.solve(c, c2) + rng.normal(0, 0.05, p.shape)
    big = dict(pos=p, vel=np.zeros_like(p), mass=np.full(len(p), 39.948), cell=c2, pot=0)
    small = small_mix(17, n_systems=3, lo=32, hi=200)
    systems = [big] + [dict(pos=small.pos[small.offsets[k]:small.offsets[k + 1]], vel=np.zeros((small.offsets[k + 1] - small.offsets[k], 3)),
                            mass=small.mass[small.offsets[k]:small.offsets[k + 1]], cell=small.cell[k], pot=int(small.pot_idx[k]))
                       for k in range(3)]
    hb = W.concat(systems, small.pots)
    b, s, F, E, S, pos = run_forces(hb, precision)
    Er, Fr, Sr = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots, use_cells=True)
    ok, worst, frac = force_tolerance_ok(F, Fr, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    assert np.all(np.abs(E - Er) <= (1e-6 if precision == 0 else 1e-9) * np.abs(Er) + 1e-9)
    # MD steps through both re-listing paths keep the state consistent
    torch = torch_cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.md_step(s, 30, 2.0 / W.T0_FS, kind=0, stream=stream)
        b.pair_forces(s, None, None, None, stream=stream)
        b.poll(stream)
    F2 = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    b.pair_forces(s, F2)
    b.poll()
    pos2 = s.pos.cpu().numpy()
    _, Fr2, _ = orc.forces(hb.offsets, pos2, hb.cell, hb.pbc, hb.pot_idx, hb.pots, use_cells=True)
    ok, worst, frac = force_tolerance_ok(F2.cpu().numpy(), Fr2, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)

"""The autotuner of the hot path's launch and list parameters (pair work-item
size, cell-list bin edge, skin scale, inner-list radius, re-list hysteresis):
it picks a valid configuration by timing MD steps, caches it, a new batch
applies the cache at create, and every configuration it can pick gives the
oracle's pair sets and forces."""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import force_tolerance_ok, frac_diff, kinds_of, make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def _copy_state(s):
    from paper_2508_06628_b300 import ts
    c = lambda t: None if t is None else t.clone()
    return ts.DeviceState(c(s.pos), c(s.vel), c(s.mass), c(s.cell), c(s.pbc), c(s.system_idx), c(s.pot_idx),
                          c(s.uid), c(s.kT))


def test_autotune_picks_caches_and_reloads(tmp_path, orc):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = W.ragged_mix(seed=5, n_systems=24, lo=32, hi=512)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots))]
    cache = str(tmp_path / "tune.txt")
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, autotune_cache=cache)
    s = ts.DeviceState.from_host(hb)
    trial = _copy_state(s)   # the trial steps advance the state they are given
    best = b.autotune(trial, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=3, n_steps=10)
    assert best["item_warps"] in (4, 8) and best["bin_factor"] in (1.0, 0.5)
    assert best["inner_fraction"] in (0.2, 0.3, 0.45, 0.5, 1.0) and best["relist_soon"] in (0.4, 0.5, 0.6)
    assert best["skin_scale"] in (1.0, 0.9, 0.8)
    key, iw, inner, soon, binf, scale = open(cache).read().split("\n")[-2].split()
    assert "pots=012" in key and "fp64=0" in key
    assert (int(iw), float(inner), float(soon), float(binf), float(scale)) == (
        best["item_warps"], best["inner_fraction"], best["relist_soon"], best["bin_factor"], best["skin_scale"])
    b.close()
    # a new batch of the same configuration starts from the cached tuning
    b2 = ts.Batch(pots, hb.n_atoms, hb.n_systems, autotune_cache=cache)
    assert b2.tuning() == best
    F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    b2.neighbor_build(s, force=True)
    b2.pair_forces(s, F, E)
    b2.poll()
    pos = s.pos.cpu().numpy()
    Er, Fr, _ = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F.cpu().numpy(), Fr, hb.offsets, False, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    assert np.all(np.abs(E.cpu().numpy() - Er) <= 1e-6 * np.abs(Er) + 1e-9)
    b2.close()


def test_tuning_rejects_values_outside_its_ranges():
    torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(31, n_systems=3, lo=32, hi=128)
    b = make_batch(hb, ts.TS_MIXED)
    for bad in (dict(item_warps=6), dict(bin_factor=0.7), dict(inner_fraction=0.0), dict(relist_soon=1.5),
                dict(skin_scale=0.0), dict(skin_scale=1.2)):
        with pytest.raises(ts.TSError) as ei:
            b.set_tuning(**bad)
        assert ei.value.status == ts.TS_ERR_INVALID_ARG
    b.close()


def test_cache_line_without_skin_scale_reads_as_one(tmp_path):
    """A cache line of the earlier five-field format (no skin_scale) applies
    with the skins unscaled."""
    torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(37, n_systems=3, lo=32, hi=128)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, ts.default_skins(hb.pots))]
    probe = ts.Batch(pots, hb.n_atoms, hb.n_systems, autotune_cache=str(tmp_path / "none.txt"))
    probe.close()
    cache = tmp_path / "tune.txt"
    # the key a batch of this configuration looks up (kinds, log2 capacities, precision)
    na, ns = int(hb.n_atoms).bit_length() - 1, int(hb.n_systems).bit_length() - 1
    kinds = "".join(str(p["kind"]) for p in pots)
    cache.write_text(f"pots={kinds};log2atoms={na};log2systems={ns};fp64=0 4 0.2 0.6 0.5\n")
    b = ts.Batch(pots, hb.n_atoms, hb.n_systems, autotune_cache=str(cache))
    assert b.tuning() == dict(item_warps=4, inner_fraction=0.2, relist_soon=0.6, bin_factor=0.5, skin_scale=1.0)
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_half_bins_small_items_pair_sets_forces_and_md(orc, precision):
    """Bins of half the list radius (two-bin stencils), four-warp items, the
    skins scaled by 0.8, a tight inner list and a late hysteresis: pair sets
    equal the oracle's brute force at the scaled list radius, forces match the
    oracle, and BAOAB steps follow the oracle."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(41, n_systems=8, lo=32, hi=600)
    b = make_batch(hb, precision)
    b.set_tuning(item_warps=4, inner_fraction=0.2, relist_soon=0.6, bin_factor=0.5, skin_scale=0.8)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    j, img, cnt = b.neighbor_export(s)
    F = torch.zeros((hb.n_atoms, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    b.pair_forces(s, F, E)
    b.poll()
    j, img, cnt, pos = j.cpu().numpy(), img.cpu().numpy(), cnt.cpu().numpy(), s.pos.cpu().numpy()
    off = hb.offsets
    for k in range(hb.n_systems):
        a, e = off[k], off[k + 1]
        pot = hb.pots[hb.pot_idx[k]]
        rl = (pot["rc"] if pot["kind"] != 2 else pot["p"][0]) + 0.8 * ts.default_skins([pot])[0]
        ref = orc.neighbors(pos[a:e], hb.cell[k], [1, 1, 1], rl)
        h = hb.cell[k]
        near = lambda i, jj, n: abs(np.linalg.norm(pos[a + jj] - pos[a + i] + np.asarray(n) @ h) - rl) < 1e-6
        R = {(int(p[0]), int(p[1]), *map(int, p[2:])) for p in ref if not near(p[0], p[1], p[2:])}
        G = {(i - a, int(j[i, q]) - a, *map(int, img[i, q])) for i in range(a, e) for q in range(cnt[i])}
        G = {t for t in G if not near(t[0], t[1], t[2:])}
        assert G == R, f"system {k}: {len(G ^ R)} pairs differ"
    Er, Fr, _ = orc.forces(hb.offsets, pos, hb.cell, hb.pbc, hb.pot_idx, hb.pots)
    ok, worst, frac = force_tolerance_ok(F.cpu().numpy(), Fr, hb.offsets, precision == 1, kinds=kinds_of(hb))
    assert ok, (worst, frac)
    # BAOAB through the tuned layout (one CUDA-graph call) against the oracle
    steps = 10 if precision == 1 else 3
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.md_step(s, steps, hb.meta["dt"], kind=ts.TS_LANGEVIN, gamma=hb.meta["gamma"], seed=9, stream=stream)
        b.poll(stream)
    xr, _, _, _ = orc.md(hb.offsets, pos, hb.vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots, hb.meta["dt"],
                         steps, kind=1, kT=hb.kT, gamma=hb.meta["gamma"], seed=9, uid=hb.uid)
    tol = 1e-9 if precision == 1 else 1e-6
    assert np.abs(frac_diff(s.pos.cpu().numpy(), xr, hb.cell, hb.offsets)).max() < tol
    b.close()


@pytest.mark.parametrize("kind", ["nhc", "npt"])
def test_autotune_under_chain_and_barostat(orc, kind):
    """The tuner saves and restores the chain state (NHC) or the cell and the
    piston velocities (NPT) between its trials: it runs clean, leaves finite
    state, and the tuned batch's next steps still follow the oracle (FP64
    chain state and cell, short mixed run)."""
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    hb = small_mix(43, n_systems=6, lo=32, hi=300)
    b = make_batch(hb, ts.TS_MIXED)
    s = ts.DeviceState.from_host(hb)
    B = hb.n_systems
    kT = torch.as_tensor(hb.kT, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        if kind == "nhc":
            st = torch.zeros((B, 6), dtype=torch.float64, device="cuda")
            best = b.autotune(s, hb.meta["dt"], kind=ts.TS_NVT_NHC, kT=kT, n_steps=5, stream=stream, tau=50.0, nhc=st)
        else:
            st = torch.zeros(B, dtype=torch.float64, device="cuda")
            best = b.autotune(s, hb.meta["dt"], kind=ts.TS_NPT_LANGEVIN, gamma=0.01, kT=kT, n_steps=5, stream=stream,
                              tau=100.0, p_ext=6.2e-3, baro=st)
        b.poll(stream)
    torch.cuda.synchronize()
    assert best["item_warps"] in (4, 8)
    assert torch.isfinite(st).all() and torch.isfinite(s.pos).all() and torch.isfinite(s.cell).all()
    # the tuned batch continues: a few steps from the current state against the oracle
    pos, vel, cell = s.pos.cpu().numpy(), s.vel.cpu().numpy(), s.cell.cpu().numpy()
    st0 = st.cpu().numpy().copy()
    with torch.cuda.stream(stream):
        if kind == "nhc":
            b.md_step(s, 3, hb.meta["dt"], kind=ts.TS_NVT_NHC, kT=kT, tau=50.0, nhc=st, stream=stream)
        else:
            b.md_step(s, 3, hb.meta["dt"], kind=ts.TS_NPT_LANGEVIN, gamma=0.01, kT=kT, tau=100.0, p_ext=6.2e-3,
                      baro=st, seed=0, stream=stream)
        b.poll(stream)
    torch.cuda.synchronize()
    assert torch.isfinite(s.pos).all() and torch.isfinite(st).all()
    if kind == "nhc":
        xr, _, _, _, nr, _ = orc.md_nhc(hb.offsets, pos, vel, hb.mass, hb.cell, hb.pbc, hb.pot_idx, hb.pots,
                                        hb.meta["dt"], 3, hb.kT, 50.0, nhc=st0)
        assert np.abs(frac_diff(s.pos.cpu().numpy(), xr, hb.cell, hb.offsets)).max() < 1e-6
        assert np.allclose(st.cpu().numpy(), nr, rtol=1e-4, atol=1e-9)
    b.close()

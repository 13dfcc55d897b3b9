"""BinningAutobatcher on the GPU (Sec. 3, Fig. 3): a fixed-length BAOAB run
of systems packed into bins and evolved bin after bin gives every system the
trajectory it has in one batch of all systems.  With the re-list hysteresis
off (TS_SOON=1) a system's re-listings depend on the system alone, so the
results agree bit for bit."""
import numpy as np
import pytest

from tests.gpu_util import make_batch, small_mix, skins_for, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_binned_run_matches_one_batch(monkeypatch, precision):
    monkeypatch.setenv("TS_SOON", "1")
    torch = torch_cuda()
    from paper_2508_06628_b300 import runtime, ts
    hb = small_mix(81, n_systems=10, lo=32, hi=400)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, skins_for(hb.pots))]
    dt, gamma, steps = hb.meta["dt"], hb.meta["gamma"], 30
    res, bins = runtime.run_binned(hb, pots, 900, steps, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=3,
                                   precision=precision)
    n_bins = bins.max() + 1
    assert n_bins >= 2
    loads = np.bincount(bins, weights=np.diff(hb.offsets), minlength=n_bins)
    assert (loads <= 900).all()
    # all systems in one batch
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    E = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    KE = torch.zeros_like(E)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        for c in range(steps // 10):
            b.md_step(s, 10, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=3, step0=10 * c, E=E, KE=KE, stream=stream)
        b.poll(stream)
    stream.synchronize()
    pos, vel, Eh, KEh = s.pos.cpu().numpy(), s.vel.cpu().numpy(), E.cpu().numpy(), KE.cpu().numpy()
    off = hb.offsets
    for k in range(hb.n_systems):
        r = res[k]
        assert np.array_equal(r["pos"], pos[off[k]:off[k + 1]])
        assert np.array_equal(r["vel"], vel[off[k]:off[k + 1]])
        assert r["E"] == Eh[k] and r["KE"] == KEh[k]
    b.close()

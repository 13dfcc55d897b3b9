"""Host-resident MD (runtime.HostMD): the state lives in pinned host buffers,
every call copies it in and out, and the systems run as two groups on two
streams.  Each system keeps its index as its noise id, and with the re-list
hysteresis off (TS_SOON=1) a system's re-listings depend on the system alone,
so every system's trajectory, energy and kinetic energy equal those of one
device-resident batch of all systems bit for bit."""
import numpy as np
import pytest

from tests.gpu_util import make_batch, skins_for, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,parts", [(0, 2), (1, 2), (0, 3)])
def test_host_md_matches_one_batch(monkeypatch, precision, parts):
    monkeypatch.setenv("TS_SOON", "1")
    torch = torch_cuda()
    from paper_2508_06628_b300 import runtime, ts
    hb = small_mix(17, n_systems=9, lo=32, hi=600)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, skins_for(hb.pots))]
    dt, gamma, inner, calls = hb.meta["dt"], hb.meta["gamma"], 10, 3
    hm = runtime.HostMD(hb, pots, parts=parts, precision=precision)
    assert len(hm.groups) == parts
    assert sorted(np.concatenate([g["ids"] for g in hm.groups]).tolist()) == list(range(hb.n_systems))
    for c in range(calls):
        hm.step(inner, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=5, step0=c * inner)
    pos, vel, E, KE = hm.state()
    hm.close()
    # one device-resident batch of every system
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    Ed = torch.zeros(hb.n_systems, dtype=torch.float64, device="cuda")
    KEd = torch.zeros_like(Ed)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for c in range(calls):
            b.md_step(s, inner, dt, kind=ts.TS_LANGEVIN, gamma=gamma, seed=5, step0=c * inner, E=Ed, KE=KEd,
                      stream=stream)
        b.poll(stream)
    stream.synchronize()
    assert np.array_equal(pos, s.pos.cpu().numpy())
    assert np.array_equal(vel, s.vel.cpu().numpy())
    assert np.array_equal(E, Ed.cpu().numpy()) and np.array_equal(KE, KEd.cpu().numpy())
    assert np.isfinite(pos).all() and not np.array_equal(pos, hb.pos)
    b.close()


def test_host_md_state_edits_between_calls(monkeypatch):
    """The host buffers are the state: a velocity the caller zeroes between
    calls is what the next call starts from."""
    monkeypatch.setenv("TS_SOON", "1")
    torch_cuda()
    from paper_2508_06628_b300 import runtime, ts
    hb = small_mix(23, n_systems=4, lo=32, hi=200)
    pots = [dict(p, skin=s) for p, s in zip(hb.pots, skins_for(hb.pots))]
    hm = runtime.HostMD(hb, pots, parts=2)
    hm.step(5, hb.meta["dt"], kind=ts.TS_NVE)
    pos0, vel0, _, _ = hm.state()
    # set_state scatters caller-ordered arrays into the groups' buffers
    moved = pos0 + np.arange(hb.n_atoms)[:, None] * 1e-7
    hm.set_state(pos=moved)
    assert np.array_equal(hm.state()[0], moved)
    hm.set_state(pos=pos0, vel=np.zeros_like(vel0))
    hm.step(1, hb.meta["dt"], kind=ts.TS_NVE, step0=5)
    _, vel1, _, KE1 = hm.state()
    with pytest.raises(ValueError):
        hm.set_state(vel=np.zeros((hb.n_atoms + 1, 3)))
    hm.close()
    # from rest, one velocity-Verlet step leaves v = dt F / m: nonzero, and far
    # below the thermal velocities the systems had before (the call did not
    # start from the device's own copy of the state)
    assert np.abs(vel1).max() > 0
    assert np.sqrt((vel1 ** 2).mean()) < 0.2 * np.sqrt((vel0 ** 2).mean())
    assert (KE1 > 0).all()

"""The re-listing paths agree with each other.

* The list build runs one warp per atom when a pass re-lists few atoms and
  one warp per 32 atoms when it re-lists many (more than 32768).  Both visit
  a system's stencil in the same order, so the lists are identical, order
  included.
* A re-listing pass runs its list build and the re-listed systems' pair
  forces on a second stream, beside the pair forces of the systems that keep
  their lists.  The trajectory is bit-identical to the serial pass.
"""
import numpy as np
import pytest

from paper_2508_06628_b300 import workloads as W
from tests.gpu_util import make_batch, small_mix, torch_cuda

pytestmark = pytest.mark.gpu


def export_lists(hb, precision):
    torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    b.neighbor_build(s, force=True)
    j, img, cnt = b.neighbor_export(s)
    b.poll()
    out = j.cpu().numpy(), img.cpu().numpy(), cnt.cpu().numpy()
    b.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_build_modes_give_identical_lists(precision):
    hb = W.ragged_mix(seed=71, n_systems=56, lo=400, hi=2048)
    assert hb.n_atoms > 32768          # the first build of the whole batch: one warp per 32 atoms
    j, img, cnt = export_lists(hb, precision)
    off = hb.offsets
    assert cnt.min() > 0
    for k in range(0, hb.n_systems, 7):  # each system alone: one warp per atom
        a, e = off[k], off[k + 1]
        j1, img1, cnt1 = export_lists(hb.subset([k]), precision)
        assert np.array_equal(cnt[a:e], cnt1)
        m = cnt1.max()
        live = np.arange(m)[None, :] < cnt1[:, None]
        assert np.array_equal(np.where(live, j[a:e, :m] - a, -1), np.where(live, j1[:, :m], -1))
        assert np.array_equal(img[a:e, :m][live], img1[:, :m][live])


def md_run(hb, precision, steps=120):
    torch = torch_cuda()
    from paper_2508_06628_b300 import ts
    b = make_batch(hb, precision)
    s = ts.DeviceState.from_host(hb)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.neighbor_build(s, force=True, stream=stream)
        _, r0 = b.counters()
        for c in range(steps // 10):
            b.md_step(s, 10, hb.meta["dt"], kind=1, gamma=hb.meta["gamma"], seed=4, step0=10 * c, stream=stream)
        b.poll(stream)
    stream.synchronize()
    _, r1 = b.counters()
    out = s.pos.cpu().numpy(), s.vel.cpu().numpy(), r1 - r0
    b.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_overlapped_relist_matches_serial(monkeypatch, precision):
    hb = small_mix(73, n_systems=12, lo=32, hi=600)
    xa, va, na = md_run(hb, precision)
    monkeypatch.setenv("TS_OVERLAP_RELIST", "0")
    xb, vb, nb = md_run(hb, precision)
    assert na > 0 and na == nb          # re-listing passes happened, the same ones
    assert np.array_equal(xa, xb)
    assert np.array_equal(va, vb)

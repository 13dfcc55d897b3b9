"""BinningAutobatcher packing (ts_bin_pack, Sec. 3 and Fig. 3): host logic, no GPU.

Pins: every bin within capacity and every system in exactly one bin; the bin
count against the exact optimum found by brute force on small instances
(first fit decreasing uses at most 11/9 OPT + 6/9 bins, Dosa 2007, and is
optimal on the instances below); the Fig. 2 example (80-atom systems under a
720-atom maximum: 9 per bin); error codes."""
import itertools

import numpy as np
import pytest

from paper_2508_06628_b300 import ts


def exact_bins(sizes, cap):
    """Fewest bins by exhaustive search over assignments (tiny instances only)."""
    n = len(sizes)
    order = sorted(range(n), key=lambda k: -sizes[k])
    best = n
    loads = []

    def place(i):
        nonlocal best
        if len(loads) >= best:
            return
        if i == n:
            best = len(loads)
            return
        s = sizes[order[i]]
        for b in range(len(loads)):
            if loads[b] + s <= cap:
                loads[b] += s
                place(i + 1)
                loads[b] -= s
        loads.append(s)
        place(i + 1)
        loads.pop()

    place(0)
    return best


def check_valid(sizes, cap, bins, nb):
    assert len(bins) == len(sizes)
    assert set(bins.tolist()) == set(range(nb))          # no empty bin
    loads = np.bincount(bins, weights=sizes, minlength=nb)
    assert (loads <= cap + 1e-9).all()


@pytest.mark.parametrize("seed", range(12))
def test_bin_pack_within_ffd_bound_of_optimum(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    sizes = rng.integers(1, 60, n).astype(float)
    cap = float(rng.integers(60, 120))
    bins, nb = ts.bin_pack(sizes, cap)
    check_valid(sizes, cap, bins, nb)
    opt = exact_bins(sizes.tolist(), cap)
    assert opt <= nb <= 11 / 9 * opt + 6 / 9


def test_bin_pack_optimal_cases():
    # perfectly packable: pairs summing to the capacity
    sizes = [70, 30, 60, 40, 55, 45, 90, 10]
    bins, nb = ts.bin_pack(sizes, 100)
    check_valid(np.array(sizes, float), 100, bins, nb)
    assert nb == 4
    # the worked example of the engine's memory probe: 80-atom systems, 720-atom maximum
    bins, nb = ts.bin_pack([80] * 20, 720)
    assert nb == 3 and np.bincount(bins).tolist() == [9, 9, 2]
    # decreasing order, ties by index: the largest system opens bin 0
    bins, _ = ts.bin_pack([10, 50, 50, 10], 60)
    assert bins[1] == 0 and bins[2] == 1 and bins[0] == 0 and bins[3] == 1


def test_bin_pack_large_ragged_batch():
    rng = np.random.default_rng(3)
    sizes = rng.integers(32, 2049, 8192).astype(float)
    cap = 40000.0
    bins, nb = ts.bin_pack(sizes, cap)
    check_valid(sizes, cap, bins, nb)
    lower = int(np.ceil(sizes.sum() / cap))
    assert nb <= lower + 1                                 # many small items: FFD is near the volume bound


def test_bin_pack_errors():
    with pytest.raises(ts.TSError) as e:
        ts.bin_pack([10, 200], 100)
    assert e.value.status == ts.TS_ERR_BUDGET
    with pytest.raises(ts.TSError) as e:
        ts.bin_pack([10, 0], 100)
    assert e.value.status == ts.TS_ERR_INVALID_ARG
    with pytest.raises(ts.TSError):
        ts.bin_pack([10], 0.0)
    bins, nb = ts.bin_pack([], 100)
    assert nb == 0 and len(bins) == 0


def test_memory_sizes_units():
    from paper_2508_06628_b300 import runtime, workloads as W
    hb = W.ragged_mix(seed=2, n_systems=6)
    n = np.diff(hb.offsets)
    assert np.array_equal(runtime.memory_sizes(hb), n.astype(float))
    d = runtime.memory_sizes(hb, "n_atoms_x_density")
    vol = np.abs(np.linalg.det(hb.cell))
    assert np.allclose(d, n * n / vol)
    with pytest.raises(ValueError):
        runtime.memory_sizes(hb, "n_bonds")


def test_exact_bins_helper_is_exact():
    # the brute force itself, checked on instances with a known optimum
    assert exact_bins([50, 50, 50, 50], 100) == 2
    assert exact_bins([60, 60, 60], 100) == 3
    assert exact_bins([34, 33, 33, 34, 33, 33], 100) == 2
    # against an enumeration of all assignments for a 5-item case
    sizes, cap = [45, 35, 30, 25, 15], 75
    best = min(len(set(a)) for a in itertools.product(range(5), repeat=5)
               if all(sum(s for s, b in zip(sizes, a) if b == k) <= cap for k in set(a)))
    assert exact_bins(sizes, cap) == best

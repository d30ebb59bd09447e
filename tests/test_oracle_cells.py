"""Pins of the oracle's cell-list candidate builder (Sec. 3.2.2 builds the
neighbour list from cells; Sec. 4 adds the skin) against its brute-force
O(N^2) builder, which is itself pinned to a k-d tree ball query: the two must
give the same candidates in the same order, bit for bit, on systems of at
most 2,000 atoms."""
import numpy as np
import pytest


def _same(O, x, box, rlist, cap):
    a = O.candidates(x, box, rlist, cap, method="cells")
    b = O.candidates(x, box, rlist, cap, method="brute")
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2]
    return a


@pytest.mark.parametrize("rlist", [6.0, 6.2, 8.0])
def test_cells_equal_brute_force_water(oracle, synth, rlist):
    w = synth.sub_box_water(9, 27.96)          # 2,187 atoms at 1 g/cm^3
    x, box = w["coords"][:2000], w["box"]      # 2,000 atoms (a hole does no harm)
    nc, cand, over = _same(oracle, x, box, rlist, 512)
    assert over == 0 and nc.min() > 0


def test_cells_equal_brute_force_copper(oracle, synth):
    x, t, box = synth.copper_fcc(8)            # 2,048 atoms, L = 29.07 A, 3 cells of 8 A
    _same(oracle, x[:2000], box, 8.0, 512)


def test_cells_equal_brute_force_zero_jitter_lattice(oracle, synth):
    """Perfect FCC: every shell is an exact tie and many pairs sit exactly at
    the cell edges' multiples."""
    x, t, box = synth.copper_fcc(8, jitter_frac=0.0)
    nc, cand, _ = _same(oracle, x[:2000], box, 8.0, 512)
    _same(oracle, x[:2000], box, 3.634 * np.sqrt(2), 512)     # the 4th shell sits at rlist


def test_cells_boxes_outside_unit_cell_and_anisotropic(oracle):
    rng = np.random.default_rng(3)
    box = np.array([19.0, 25.5, 31.0])
    x = rng.uniform(-1.5, 2.5, (1500, 3)) * box     # coordinates far outside [0, L)
    _same(oracle, x, box, 6.0, 256)
    # box edges a hair above 3 rlist and exactly 4 rlist (3 cells of 8 A)
    box = np.array([18.000001, 24.0, 18.000001])
    x = rng.uniform(0, 1, (1200, 3)) * box
    x[:40] = np.round(x[:40] / 6.0) * 6.0           # atoms on the cell faces
    _same(oracle, x, box, 6.0, 256)


def test_cells_capacity_overflow_matches(oracle):
    rng = np.random.default_rng(4)
    box = np.array([20.0, 20.0, 20.0])
    x = rng.uniform(0, 1, (1800, 3)) * box
    nc, cand, over = _same(oracle, x, box, 6.0, 96)
    assert over > 0 and nc.max() == 96


def test_cells_subset_of_centres(oracle, synth):
    w = synth.sub_box_water(9, 27.96)
    x, box = w["coords"], w["box"]
    full = oracle.candidates(x, box, 8.0, 512, method="cells")
    part = oracle.candidates(x, box, 8.0, 512, method="cells", ncentre=700)
    np.testing.assert_array_equal(part[0][:700], full[0][:700])
    np.testing.assert_array_equal(part[1][:700], full[1][:700])
    assert np.all(part[0][700:] == 0)


def test_cells_refuse_small_boxes(oracle, synth):
    w = synth.workload("water192")               # 12.42 A: 2 cells of 6 A
    with pytest.raises(ValueError):
        oracle.candidates(w["coords"], w["box"], 6.0, 192, method="cells")
    a = oracle.candidates(w["coords"], w["box"], 6.0, 192)          # auto falls back
    b = oracle.candidates(w["coords"], w["box"], 6.0, 192, method="brute")
    np.testing.assert_array_equal(a[1], b[1])

"""Host-side logic of the student trainer (no GPU needed).

The trainer works in units of the labels' RMS force by dividing every type's
output layer (w_o, b_o) by the same factor; that is exact only because the
atomic energy is affine in the output layer (Eq. fitting: E_i = h w_o + b_o),
so E and F scale by the same factor.  These tests check the flat-vector
slices the trainer rescales and that property, the latter on the oracle.
"""
import numpy as np
import pytest

from paper_2004_11658_gb300 import student as S
from paper_2004_11658_gb300 import synth as Y


@pytest.mark.parametrize("desc", [Y.WATER_MODEL, Y.WATER_STUDENT], ids=["full", "student"])
def test_output_slices_are_wo_then_bo(desc):
    shapes = dict(Y.layer_shapes(desc))
    sl = S._output_slices(desc)
    assert len(sl) == desc["ntypes"]
    for a, s in enumerate(sl):
        wo = S.param_offset(desc, f"fit{a}.wo")
        bo = S.param_offset(desc, f"fit{a}.bo")
        assert shapes[f"fit{a}.wo"] == (desc["fit"][-1],) and shapes[f"fit{a}.bo"] == (1,)
        assert (s.start, s.stop) == (wo, bo + 1)
        assert bo == wo + desc["fit"][-1]
    # the slices are disjoint and inside the vector
    n = Y.n_params(desc)
    marks = np.zeros(n, dtype=int)
    for s in sl:
        marks[s] += 1
    assert marks.max() == 1 and marks.sum() == desc["ntypes"] * (desc["fit"][-1] + 1)


def test_param_offset_unknown_name():
    with pytest.raises(KeyError):
        S.param_offset(Y.WATER_MODEL, "fit9.wo")


def test_output_layer_scaling_scales_energy_and_force(oracle):
    """E and F are linear in (w_o, b_o) of all types together: scaling those
    slices by c scales E, every E_i, F and the virial by c.  The output biases
    are set nonzero first, so that a slice missing b_o fails."""
    w = Y.workload("water192")
    desc = w["model"]
    P = Y.model_params(desc, 0)
    sl = S._output_slices(desc)
    for a, s in enumerate(sl):
        P[s.stop - 1] = -0.3 + 0.1 * a
    c = 0.37
    Pc = P.copy()
    for s in sl:
        Pc[s] *= c
    a = oracle.evaluate(desc, P, w["coords"], w["types"], w["box"])
    b = oracle.evaluate(desc, Pc, w["coords"], w["types"], w["box"])
    assert b["energy"] == pytest.approx(c * a["energy"], rel=1e-13)
    np.testing.assert_allclose(b["atom_energy"], c * a["atom_energy"], rtol=1e-13, atol=0)
    fmax = np.abs(a["force"]).max()
    np.testing.assert_allclose(b["force"], c * a["force"], rtol=0, atol=1e-13 * fmax)
    vmax = np.abs(np.asarray(a["virial"])).max()
    np.testing.assert_allclose(b["virial"], c * np.asarray(a["virial"]), rtol=0, atol=1e-13 * vmax)
    # scaling w_o alone leaves the biases' share unscaled
    Pw = P.copy()
    for s in sl:
        Pw[s.start:s.stop - 1] *= c
    d = oracle.evaluate(desc, Pw, w["coords"], w["types"], w["box"])
    assert abs(d["energy"] - c * a["energy"]) > 1e-3 * abs(a["energy"])

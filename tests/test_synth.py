"""The seeded synthetic inputs follow their stated recipe: rigid water
(O-H 0.96 A, H-O-H 104.5 deg) at about 1 g/cm^3, FCC copper with a = 3.634 A
(Sec. 4), Maxwell-Boltzmann velocities with no centre-of-mass momentum at
exactly T0 over 3N - 3 degrees of freedom, and reproducible seeds."""
import numpy as np
import pytest

from paper_2004_11658_gb300 import synth as Y

_AMU_G = 1.66053906660e-24          # g
_KB_EV = 1.380649e-23 / 1.602176634e-19
_AMU_A2_FS2_IN_EV = 1.66053906660e-27 * 1e10 / 1.602176634e-19


def _min_image(d, L):
    return d - L * np.round(d / L)


@pytest.mark.parametrize("name", ["water192", "water12288"])
def test_water_is_rigid_molecules_at_unit_density(name):
    w = Y.workload(name)
    x, t, L = w["coords"], w["types"], w["box"]
    assert list(t[:6]) == [0, 1, 1, 0, 1, 1] and len(x) % 3 == 0
    O, H1, H2 = x[0::3], x[1::3], x[2::3]
    d1, d2 = _min_image(H1 - O, L), _min_image(H2 - O, L)
    r1, r2 = np.linalg.norm(d1, axis=1), np.linalg.norm(d2, axis=1)
    np.testing.assert_allclose(r1, 0.96, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r2, 0.96, rtol=0, atol=1e-12)
    ang = np.degrees(np.arccos((d1 * d2).sum(1) / (r1 * r2)))
    np.testing.assert_allclose(ang, 104.5, rtol=0, atol=1e-9)
    assert np.all((x >= 0) & (x < L))
    mass_g = len(O) * (2 * w["masses"][1] + w["masses"][0]) * _AMU_G
    rho = mass_g / (np.prod(L) * 1e-24)
    assert rho == pytest.approx(1.0, rel=0.01)


def test_copper_fcc_lattice():
    w = Y.workload("cu32000")
    x, L = w["coords"], w["box"]
    assert len(x) == 4 * 20 ** 3
    np.testing.assert_allclose(L, 20 * 3.634)
    # every atom within a few jitter widths of an FCC site of a = 3.634 A
    a = 3.634
    frac = np.mod(x / a, 1.0)
    sites = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    d = _min_image(frac[:, None, :] - sites[None], 1.0) * a
    nearest = np.linalg.norm(d, axis=2).min(axis=1)
    assert nearest.max() < 6 * 0.01 * a * np.sqrt(3)
    assert np.std(nearest) > 0.0                      # the jitter is there


@pytest.mark.parametrize("T0", [300.0, 330.0])
def test_maxwell_velocities_exact_temperature_zero_momentum(T0):
    w = Y.workload("water192")
    m = np.array(w["masses"])[w["types"]]
    v = Y.maxwell_velocities(m, T0, seed=2)
    p = (m[:, None] * v).sum(0)
    assert np.abs(p).max() < 1e-12 * (m[:, None] * np.abs(v)).sum()
    ke = 0.5 * float((m[:, None] * v * v).sum()) * _AMU_A2_FS2_IN_EV
    T = 2 * ke / ((3 * len(m) - 3) * _KB_EV)
    assert T == pytest.approx(T0, rel=1e-9)


def test_seeds_are_reproducible():
    a, b = Y.workload("water192"), Y.workload("water192")
    np.testing.assert_array_equal(a["coords"], b["coords"])
    c = Y.workload("water192", seed_geom=2)
    assert not np.array_equal(a["coords"], c["coords"])
    P0, P1 = Y.model_params(Y.WATER_MODEL, 0), Y.model_params(Y.WATER_MODEL, 0)
    np.testing.assert_array_equal(P0, P1)
    assert len(P0) == Y.n_params(Y.WATER_MODEL)

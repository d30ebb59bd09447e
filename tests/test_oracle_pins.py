"""Pins of the CPU oracle to facts other than itself (no GPU needed).

Each test checks the oracle against something the paper or the mathematics
fixes: closed forms of special cases, brute force on tiny inputs, a library
routine, invariances (Sec. 2: translation, rotation, permutation), F = -grad E
(Remark 2), the virial as the strain derivative, smoothness at rcut (Sec. 2),
sel independence (padding rows are zero, Algorithm 2) and velocity-Verlet
properties (Sec. 4).
"""
import math

import numpy as np
import pytest

pytestmark = []


def views(S, desc, P):
    out, off = {}, 0
    for name, shape in S.layer_shapes(desc):
        n = int(np.prod(shape))
        out[name] = P[off:off + n].reshape(shape)
        off += n
    assert off == len(P)
    return out


# ----------------------------------------------------------- switching --

def test_switch_closed_forms(oracle):
    rs, rc = 0.5, 6.0
    for r in (0.05, 0.3, 0.4999):
        s, ds = oracle.switch(r, rs, rc)
        assert s == 1.0 / r and ds == pytest.approx(-1.0 / r ** 2, rel=1e-15)
    for r in (6.0, 6.5, 100.0):
        assert oracle.switch(r, rs, rc) == (0.0, 0.0)
    # w(r) = r s(r): 1 at rs, 1/2 at the midpoint (the quintic step is odd
    # about u = 1/2), 0 at rc
    w = lambda r: r * oracle.switch(r, rs, rc)[0]
    assert w(rs) == pytest.approx(1.0, abs=1e-15)
    assert w(0.5 * (rs + rc)) == pytest.approx(0.5, abs=1e-14)
    assert w(rc - 1e-12) == pytest.approx(0.0, abs=1e-12)
    # C2: w', w'' vanish at both ends (one-sided differences from inside)
    h = 1e-4
    for r0, sgn in ((rs, 1.0), (rc, -1.0)):
        d1 = (w(r0 + sgn * 2 * h) - w(r0 + sgn * h)) / h
        d2 = (w(r0 + sgn * 3 * h) - 2 * w(r0 + sgn * 2 * h) + w(r0 + sgn * h)) / h ** 2
        assert abs(d1) < 1e-6 and abs(d2) < 1e-3
    # ds/dr against central differences in every region
    for r in (0.3, 0.6, 2.0, 3.25, 5.9):
        s, ds = oracle.switch(r, rs, rc)
        fd = (oracle.switch(r + 1e-6, rs, rc)[0] - oracle.switch(r - 1e-6, rs, rc)[0]) / 2e-6
        assert ds == pytest.approx(fd, rel=1e-7, abs=1e-9)


# ----------------------------------------------------- neighbour lists --

def test_candidates_match_kdtree(oracle, synth):
    spatial = pytest.importorskip("scipy.spatial")
    w = synth.workload("water192")
    x, L = w["coords"], w["box"]
    rl = 6.0
    ncand, cand, over = oracle.candidates(x, L, rl, 192)
    assert over == 0
    tree = spatial.cKDTree(x, boxsize=L)
    ref = tree.query_ball_point(x, r=rl)
    for i in range(len(x)):
        got = set(cand[i, :ncand[i]].tolist())
        exp = set(ref[i]) - {i}
        assert got == exp


def _py_format(x, types, L, sel, rcut, rlist):
    """Algorithm 1 by brute force in pure Python on a tiny system."""
    N = len(x)
    nm = sum(sel)
    off = [sum(sel[:a]) for a in range(len(sel))]
    nlist = [[-1] * nm for _ in range(N)]
    nreal = [[0] * len(sel) for _ in range(N)]
    ovf = [0] * N
    for i in range(N):
        S = []
        for j in range(N):
            if j == i:
                continue
            d = []
            for a in range(3):
                v = x[j][a] - x[i][a]
                n = round(v / L[a])            # round half to even, like rint
                d.append(v - L[a] * n)
            r = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
            if r <= rcut:          # L(i) of Sec. 2 (the skin only widens the candidates)
                S.append((int(types[j]), math.floor(r * 1e8), j, r))
        S.sort(key=lambda t: (t[0], t[1], t[2]))
        cnt = [0] * len(sel)
        for (a, q, j, r) in S:
            if cnt[a] < sel[a]:
                nlist[i][off[a] + cnt[a]] = j
                cnt[a] += 1
            else:
                ovf[i] += 1
        nreal[i] = cnt
    return np.array(nlist), np.array(nreal), np.array(ovf)


@pytest.mark.parametrize("sel", [(6, 9), (2, 3)])
def test_format_matches_brute_force(oracle, sel):
    rng = np.random.default_rng(5)
    N, L = 40, np.array([9.0, 9.5, 10.0])
    x = rng.uniform(0, 1, (N, 3)) * L
    x[7] = x[3] + np.array([0.4, 0.0, 0.0])   # a close pair
    types = rng.integers(0, 2, N).astype(np.int32)
    rcut, skin = 3.0, 1.0
    ncand, cand, _ = oracle.candidates(x, L, rcut + skin, 64)
    nl, nr, ov = oracle.format_nlist(x, types, L, ncand, cand, sel, rcut)
    enl, enr, eov = _py_format(x.tolist(), types, L.tolist(), list(sel), rcut, rcut + skin)
    np.testing.assert_array_equal(nl, enl)
    np.testing.assert_array_equal(nr, enr)
    np.testing.assert_array_equal(ov, eov)
    if sel == (2, 3):
        assert ov.sum() > 0


def test_format_tie_break_by_index(oracle):
    # two neighbours of atom 0 at exactly the same distance: smaller index first
    x = np.array([[5.0, 5.0, 5.0], [6.0, 5.0, 5.0], [4.0, 5.0, 5.0], [5.0, 6.5, 5.0]])
    L = np.array([20.0, 20.0, 20.0])
    types = np.zeros(4, dtype=np.int32)
    ncand, cand, _ = oracle.candidates(x, L, 4.0, 8)
    nl, nr, _ = oracle.format_nlist(x, types, L, ncand, cand, (4,), 4.0)
    assert nl[0].tolist() == [1, 2, 3, -1]
    assert nr[0].tolist() == [3]
    # the list holds L(i) only: with rcut 1.2 A atom 3 (1.5 A away) is left out
    nl, nr, _ = oracle.format_nlist(x, types, L, ncand, cand, (4,), 1.2)
    assert nl[0].tolist() == [1, 2, -1, -1]
    assert nr[0].tolist() == [2]


# ------------------------------------------------- closed-form energies --

SMALL = dict(ntypes=1, sel=(4,), rcut=4.0, rcut_smth=1.0, emb=(2, 4, 8), m2=2, fit=(3,), desc_scale_nm=1)


def _zero_emb_weights(S, desc, seed, keep_W0=False):
    P = S.model_params(desc, seed, fit_in_gain=30.0)
    V = views(S, desc, P)
    for name, arr in V.items():
        if name.startswith("emb") and ".W" in name and not (keep_W0 and name.endswith(".W0")):
            arr[...] = 0.0
    return P, V


def _fit_energy(V, a, D):
    h = np.tanh(D.ravel() @ V[f"fit{a}.W1"] + V[f"fit{a}.b1"])
    return float(h @ V[f"fit{a}.wo"] + V[f"fit{a}.bo"][0])


def test_single_neighbour_closed_form(oracle, synth):
    """One neighbour, embedding weights 0: G is the constant built from the
    biases and the skips, D = 2 (s/N_m)^2 G_< (x) G (|(1, x/r, y/r, z/r)|^2 = 2)."""
    desc = SMALL
    P, V = _zero_emb_weights(synth, desc, 3)
    h0 = np.tanh(V["emb00.b0"])
    h1 = np.concatenate([h0, h0]) + np.tanh(V["emb00.b1"])
    G = np.concatenate([h1, h1]) + np.tanh(V["emb00.b2"])
    L = np.array([30.0, 30.0, 30.0])
    r = 2.5
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r * 0.6, 10.0 + r * 0.8, 10.0]])
    out = oracle.evaluate(desc, P, x, np.zeros(2, np.int32), L)
    s, _ = oracle.switch(r, desc["rcut_smth"], desc["rcut"])
    nm = 4
    D = 2.0 * (s / nm) ** 2 * np.outer(G[:2], G)
    e0 = _fit_energy(V, 0, D)
    assert out["atom_energy"] == pytest.approx([e0, e0], rel=1e-13)


def test_two_neighbour_angle_closed_form(oracle, synth):
    """Constant G: D = G_a G_b / N_m^2 * |sum_k s_k (1, u_k)|^2
    = G_a G_b / N_m^2 * ((s1 + s2)^2 + s1^2 + s2^2 + 2 s1 s2 cos(theta))."""
    desc = SMALL
    P, V = _zero_emb_weights(synth, desc, 4)
    h0 = np.tanh(V["emb00.b0"])
    h1 = np.concatenate([h0, h0]) + np.tanh(V["emb00.b1"])
    G = np.concatenate([h1, h1]) + np.tanh(V["emb00.b2"])
    L = np.array([40.0, 40.0, 40.0])
    r1, r2, th = 1.7, 3.1, 1.1
    c = np.array([20.0, 20.0, 20.0])
    x = np.array([c, c + r1 * np.array([1.0, 0, 0]), c + r2 * np.array([np.cos(th), np.sin(th), 0.0])])
    out = oracle.evaluate(desc, P, x, np.zeros(3, np.int32), L)
    s1 = oracle.switch(r1, 1.0, 4.0)[0]
    s2 = oracle.switch(r2, 1.0, 4.0)[0]
    q = (s1 + s2) ** 2 + s1 ** 2 + s2 ** 2 + 2 * s1 * s2 * np.cos(th)
    D = q / 16.0 * np.outer(G[:2], G)
    assert out["atom_energy"][0] == pytest.approx(_fit_energy(V, 0, D), rel=1e-12)


def test_layer0_dependence_closed_form(oracle, synth):
    """W0 != 0, deeper weights 0: G = ((h0,h0)+tanh(b1), (h0,h0)+tanh(b1)) + tanh(b2)
    with h0 = tanh(s W0 + b0) (Eqs. embedding-first, embedding-rest)."""
    desc = SMALL
    P, V = _zero_emb_weights(synth, desc, 5, keep_W0=True)
    L = np.array([30.0, 30.0, 30.0])
    r = 0.8   # below rcut_smth: s = 1/r
    x = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0 + r]])
    out = oracle.evaluate(desc, P, x, np.zeros(2, np.int32), L)
    s = 1.0 / r
    h0 = np.tanh(s * V["emb00.W0"] + V["emb00.b0"])
    h1 = np.concatenate([h0, h0]) + np.tanh(V["emb00.b1"])
    G = np.concatenate([h1, h1]) + np.tanh(V["emb00.b2"])
    D = 2.0 * (s / 4) ** 2 * np.outer(G[:2], G)
    assert out["atom_energy"][0] == pytest.approx(_fit_energy(V, 0, D), rel=1e-13)


def test_type_pair_nets_closed_form(oracle, synth):
    """Remark 1: atom i of type a uses G^{a, alpha_j} and N_a; the neighbour
    sits in the slot block of its own type."""
    desc = dict(SMALL, ntypes=2, sel=(2, 3))
    P, V = _zero_emb_weights(synth, desc, 6)
    L = np.array([30.0, 30.0, 30.0])
    r = 2.2
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    t = np.array([0, 1], np.int32)
    out = oracle.evaluate(desc, P, x, t, L)
    assert out["nlist"].tolist() == [[-1, -1, 1, -1, -1], [0, -1, -1, -1, -1]]
    s = oracle.switch(r, 1.0, 4.0)[0]
    for a, b in ((0, 1), (1, 0)):
        h0 = np.tanh(V[f"emb{a}{b}.b0"])
        h1 = np.concatenate([h0, h0]) + np.tanh(V[f"emb{a}{b}.b1"])
        G = np.concatenate([h1, h1]) + np.tanh(V[f"emb{a}{b}.b2"])
        D = 2.0 * (s / 5) ** 2 * np.outer(G[:2], G)
        assert out["atom_energy"][a] == pytest.approx(_fit_energy(V, a, D), rel=1e-13)


def test_unscaled_descriptor_flag(oracle, synth):
    """desc_scale_nm = 0 is the paper's unscaled Eq. descrpt: D grows by N_m^2."""
    desc0 = dict(SMALL, desc_scale_nm=0)
    P, V = _zero_emb_weights(synth, desc0, 3)
    L = np.array([30.0, 30.0, 30.0])
    x = np.array([[10.0, 10.0, 10.0], [12.0, 10.0, 10.0]])
    o0 = oracle.evaluate(desc0, P, x, np.zeros(2, np.int32), L, want_descriptor=True)
    o1 = oracle.evaluate(SMALL, P, x, np.zeros(2, np.int32), L, want_descriptor=True)
    np.testing.assert_allclose(o0["descriptor"], 16.0 * o1["descriptor"], rtol=1e-14)


# ------------------------------------------------------------ invariances --

@pytest.fixture(scope="module")
def water(synth):
    w = synth.workload("water192")
    P = synth.model_params(w["model"], 0)
    return w, P


def _cluster(w, radius=7.0):
    x = w["coords"]
    L = w["box"]
    c = L / 2
    d = x - c
    keep = np.where(np.linalg.norm(d, axis=1) < radius)[0]
    xc = d[keep] + 40.0
    return xc, w["types"][keep], np.array([80.0, 80.0, 80.0])


def test_translation_invariance(oracle, water):
    w, P = water
    a = oracle.evaluate(w["model"], P, w["coords"], w["types"], w["box"])
    x2 = np.mod(w["coords"] + np.array([1.37, -2.11, 0.73]), w["box"])
    b = oracle.evaluate(w["model"], P, x2, w["types"], w["box"])
    assert b["energy"] == pytest.approx(a["energy"], rel=1e-12)
    np.testing.assert_allclose(b["force"], a["force"], atol=1e-10 * np.abs(a["force"]).max())


def test_rotation_invariance_cluster(oracle, water):
    w, P = water
    x, t, L = _cluster(w)
    a = oracle.evaluate(w["model"], P, x, t, L)
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    c = np.array([40.0, 40.0, 40.0])
    xr = (x - c) @ Q.T + c
    b = oracle.evaluate(w["model"], P, xr, t, L)
    assert b["energy"] == pytest.approx(a["energy"], rel=1e-12)
    np.testing.assert_allclose(b["force"], a["force"] @ Q.T, atol=1e-10 * np.abs(a["force"]).max())
    # descriptor itself is rotation invariant
    da = oracle.evaluate(w["model"], P, x, t, L, want_descriptor=True)["descriptor"]
    db = oracle.evaluate(w["model"], P, xr, t, L, want_descriptor=True)["descriptor"]
    np.testing.assert_allclose(db, da, atol=1e-13 * np.abs(da).max())


def test_permutation_invariance(oracle, water):
    w, P = water
    rng = np.random.default_rng(12)
    perm = rng.permutation(len(w["coords"]))
    a = oracle.evaluate(w["model"], P, w["coords"], w["types"], w["box"])
    b = oracle.evaluate(w["model"], P, w["coords"][perm], w["types"][perm], w["box"])
    assert b["energy"] == pytest.approx(a["energy"], rel=1e-12)
    np.testing.assert_allclose(b["force"], a["force"][perm], atol=1e-11 * np.abs(a["force"]).max())
    np.testing.assert_allclose(b["atom_energy"], a["atom_energy"][perm], rtol=1e-11)


# ------------------------------------------------- forces and the virial --

def test_force_sum_zero_and_virial_symmetric(oracle, water):
    w, P = water
    a = oracle.evaluate(w["model"], P, w["coords"], w["types"], w["box"])
    F = a["force"]
    assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).max() * len(F)
    V = a["virial"]
    assert np.abs(V - V.T).max() < 1e-12 * np.abs(V).max()
    rms = np.sqrt((F ** 2).mean())
    assert 0.002 < rms < 5.0   # the seeded model gives RMS forces of ~0.01 eV/A


def test_forces_are_minus_gradient(oracle, water):
    """Remark 2 (F = -grad E): Richardson-extrapolated central differences."""
    w, P = water
    x0 = w["coords"]
    a = oracle.evaluate(w["model"], P, x0, w["types"], w["box"])
    F = a["force"]
    rng = np.random.default_rng(13)
    atoms = rng.choice(len(x0), 4, replace=False)

    def fd(i, c, h):
        xp = x0.copy()
        xp[i, c] += h
        xm = x0.copy()
        xm[i, c] -= h
        ep = oracle.evaluate(w["model"], P, xp, w["types"], w["box"])["energy"]
        em = oracle.evaluate(w["model"], P, xm, w["types"], w["box"])["energy"]
        return (ep - em) / (2 * h)

    scale = np.abs(F).max()
    for i in atoms:
        for c in range(3):
            d1, d2 = fd(i, c, 2e-4), fd(i, c, 1e-4)
            rich = (4 * d2 - d1) / 3
            assert abs(rich + F[i, c]) < 2e-8 * scale
            assert abs(d2 + F[i, c]) < 2e-6 * scale


def test_virial_cluster_equals_r_times_f(oracle, water):
    w, P = water
    x, t, L = _cluster(w)
    a = oracle.evaluate(w["model"], P, x, t, L)
    V = x.T @ a["force"]      # sum_i r_i (x) F_i
    np.testing.assert_allclose(a["virial"], V, atol=1e-10 * np.abs(V).max())


def test_virial_is_strain_derivative(oracle, water):
    """Xi[a][b] = -dE/d(eps[b][a]) under x -> (I + eps) x (isolated cluster,
    any strain) and under diagonal strains of the periodic box."""
    w, P = water
    x, t, L = _cluster(w, radius=6.0)
    V = oracle.evaluate(w["model"], P, x, t, L)["virial"]
    c = np.array([40.0, 40.0, 40.0])
    h = 1e-5
    for (p, q) in ((0, 0), (1, 2), (2, 1), (0, 1)):
        e = np.zeros((3, 3))
        e[p, q] = h
        ep = oracle.evaluate(w["model"], P, (x - c) @ (np.eye(3) + e).T + c, t, L)["energy"]
        em = oracle.evaluate(w["model"], P, (x - c) @ (np.eye(3) - e).T + c, t, L)["energy"]
        dE = (ep - em) / (2 * h)
        assert dE == pytest.approx(-V[q, p], abs=1e-6 * np.abs(V).max())
    # periodic box, diagonal strain
    xw, Lw = w["coords"], w["box"]
    Vp = oracle.evaluate(w["model"], P, xw, w["types"], Lw)["virial"]
    for a_ in range(3):
        s = np.ones(3)
        s[a_] += h
        ep = oracle.evaluate(w["model"], P, xw * s, w["types"], Lw * s)["energy"]
        s[a_] -= 2 * h
        em = oracle.evaluate(w["model"], P, xw * s, w["types"], Lw * s)["energy"]
        assert (ep - em) / (2 * h) == pytest.approx(-Vp[a_, a_], abs=1e-6 * np.abs(Vp).max())


# -------------------------------------------------------------- smoothness --

def test_smooth_through_rcut(oracle, synth):
    desc = SMALL
    P = synth.model_params(desc, 8, fit_in_gain=30.0)
    L = np.array([30.0, 30.0, 30.0])

    def energy(r):
        x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        return oracle.evaluate(desc, P, x, np.zeros(2, np.int32), L)["energy"]

    rc = desc["rcut"]
    far = energy(rc + 0.5)
    assert energy(rc) == far and energy(rc + 1e-9) == far and energy(rc + 3.0) == far
    # value, slope and curvature go to their far-field values as r -> rc
    h = 1e-3
    e1, e2, e3 = energy(rc - h), energy(rc - 2 * h), energy(rc - 3 * h)
    assert abs(e1 - far) < 1e-6
    assert abs((e1 - e2) / h) < 1e-4
    assert abs((e1 - 2 * e2 + e3) / h ** 2) < 0.5
    # C1 inside: left and right slopes agree at an interior point
    r0 = 3.0
    sl = (energy(r0) - energy(r0 - 1e-5)) / 1e-5
    sr = (energy(r0 + 1e-5) - energy(r0)) / 1e-5
    assert sl == pytest.approx(sr, rel=1e-3, abs=1e-8)


def test_sel_independence(oracle, synth):
    """Padding rows are zero (Algorithm 2): with the unscaled descriptor, a
    larger sel changes nothing when no neighbour is cut."""
    w = synth.workload("water192")
    d1 = dict(w["model"], desc_scale_nm=0)
    d2 = dict(d1, sel=(64, 128))
    P = synth.model_params(d1, 0, fit_in_gain=300.0 / 138 ** 2)
    a = oracle.evaluate(d1, P, w["coords"], w["types"], w["box"])
    b = oracle.evaluate(d2, P, w["coords"], w["types"], w["box"])
    assert a["overflow"] == 0
    assert b["energy"] == pytest.approx(a["energy"], rel=1e-13)
    np.testing.assert_allclose(b["force"], a["force"], atol=1e-12 * np.abs(a["force"]).max())


# ---------------------------------------------------------------------- MD --

def test_md_energy_drift_scales_dt2(oracle, synth):
    w = synth.workload("water192")
    P = synth.model_params(w["model"], 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=2)

    def drift(dt, n):
        _, _, _, th, _ = oracle.md(w["model"], P, w["coords"], v0, w["types"], w["box"], w["masses"], dt, n,
                                   rebuild_every=1, skin=0.0)
        etot = th[:, 0] + th[:, 1]
        return np.abs(etot - etot[0]).max(), th

    # asymptotic regime: halving dt cuts the energy error ~4x (at 0.5 fs the
    # seeded model's stiffest modes are already beyond it)
    d1, th = drift(0.25, 80)
    d2, _ = drift(0.125, 160)
    assert 2.5 < d1 / d2 < 6.0
    assert d1 < 5e-3 * len(m)   # below 5 meV per atom over 20 fs
    assert th[0, 2] == pytest.approx(300.0, rel=0.1)


def test_md_time_reversible(oracle, synth):
    w = synth.workload("water192")
    P = synth.model_params(w["model"], 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=2)
    x1, v1, f1, _, _ = oracle.md(w["model"], P, w["coords"], v0, w["types"], w["box"], w["masses"], 0.5, 20,
                                 rebuild_every=1, skin=0.0)
    x2, v2, _, _, _ = oracle.md(w["model"], P, x1, -v1, w["types"], w["box"], w["masses"], 0.5, 20,
                                rebuild_every=1, skin=0.0, force=f1)
    d = x2 - w["coords"]
    d -= w["box"] * np.round(d / w["box"])
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(-v2, v0, atol=1e-10)


# Unit conversions from the SI definitions (amu, eV, k_B exact in the 2019 SI
# or CODATA 2018), independent of the oracle's own constants.
_AMU_KG = 1.66053906660e-27
_EV_J = 1.602176634e-19
_KB_J = 1.380649e-23
_AMU_A2_FS2_IN_EV = _AMU_KG * 1e10 / _EV_J       # 1 amu (A/fs)^2 in eV
_ACC_A_FS2 = _EV_J / 1e-10 / _AMU_KG * 1e-20     # 1 eV/A/amu in A/fs^2


def test_md_one_step_is_velocity_verlet(oracle, synth):
    """One step from (x0, v0): x1 = x0 + dt v0 + dt^2/2 a0, v1 = v0 + dt/2 (a0 + a1),
    a = F/m in A/fs^2, F from the evaluator at x0 and x1 (Sec. 4)."""
    w = synth.workload("water192")
    P = synth.model_params(w["model"], 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=5)
    dt = 0.5
    x1, v1, f1, _, _ = oracle.md(w["model"], P, w["coords"], v0, w["types"], w["box"], w["masses"], dt, 1,
                                 rebuild_every=1, skin=0.0)
    f0 = oracle.evaluate(w["model"], P, w["coords"], w["types"], w["box"])["force"]
    a0 = f0 / m[:, None] * _ACC_A_FS2
    x1_ref = np.mod(w["coords"] + dt * v0 + 0.5 * dt * dt * a0, w["box"])
    d = x1 - x1_ref
    d -= w["box"] * np.round(d / w["box"])
    assert np.abs(d).max() < 1e-12
    f1_ref = oracle.evaluate(w["model"], P, x1, w["types"], w["box"])["force"]
    np.testing.assert_allclose(f1, f1_ref, rtol=0, atol=1e-13 * np.abs(f1_ref).max())
    v1_ref = v0 + 0.5 * dt * (a0 + f1_ref / m[:, None] * _ACC_A_FS2)
    np.testing.assert_allclose(v1, v1_ref, rtol=0, atol=1e-12 * np.abs(v1_ref).max())


def test_md_thermo_definitions(oracle, synth):
    """thermo = (E_pot, E_kin, T, P) of the configuration after the step:
    E_kin = sum m v^2 / 2, T = 2 E_kin / ((3N - 3) k_B), P = (2 E_kin + tr Xi) / (3V)."""
    w = synth.workload("water192")
    P = synth.model_params(w["model"], 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=6)
    x, v, _, th, _ = oracle.md(w["model"], P, w["coords"], v0, w["types"], w["box"], w["masses"], 0.5, 3,
                               rebuild_every=1, skin=0.0)
    out = oracle.evaluate(w["model"], P, x, w["types"], w["box"])
    n = len(m)
    ke = 0.5 * float((m[:, None] * v * v).sum()) * _AMU_A2_FS2_IN_EV
    temp = 2.0 * ke / ((3 * n - 3) * _KB_J / _EV_J)
    vol = float(np.prod(w["box"]))
    pres = (2.0 * ke + float(np.trace(np.asarray(out["virial"]).reshape(3, 3)))) / (3.0 * vol)
    assert th[-1, 0] == pytest.approx(out["energy"], rel=1e-13)
    assert th[-1, 1] == pytest.approx(ke, rel=1e-9)
    assert th[-1, 2] == pytest.approx(temp, rel=1e-9)
    assert th[-1, 3] == pytest.approx(pres, rel=1e-9)


# ------------------------------------------------------- parameter gradient --

def _phi(oracle, desc, P, w, cE, lam):
    o = oracle.evaluate(desc, P, w["coords"], w["types"], w["box"])
    return cE * o["energy"] + float((lam * o["force"]).sum())


@pytest.mark.parametrize("cE,fw", [(1.0, 0.0), (0.0, 1.0), (0.7, 30.0)])
def test_param_grad_directional_fd(oracle, synth, cE, fw):
    """d/dW of cE E + sum lambda . F against Richardson-extrapolated central
    differences along random directions in parameter space (the force term
    differentiates through F = -grad E: a second derivative)."""
    w = synth.workload("water192")
    desc = w["model"]
    P = synth.model_params(desc, 0)
    rng = np.random.default_rng(31)
    lam = fw * rng.standard_normal((len(w["coords"]), 3))
    g = oracle.param_grad(desc, P, w["coords"], w["types"], w["box"], cE, lam)
    for trial in range(2):
        V = rng.standard_normal(len(P))
        V /= np.linalg.norm(V)
        def fd(h):
            return (_phi(oracle, desc, P + h * V, w, cE, lam) - _phi(oracle, desc, P - h * V, w, cE, lam)) / (2 * h)
        d1, d2 = fd(2e-4), fd(1e-4)
        rich = (4 * d2 - d1) / 3
        assert rich == pytest.approx(float(g @ V), rel=1e-6, abs=1e-9 * (abs(cE) + fw))


def test_param_grad_single_parameters(oracle, synth):
    """Central differences on single parameters of every kind: embedding W0,
    b0, inner W and b of both neighbour types, fitting W1, hidden W, w_out,
    b_out."""
    w = synth.workload("water192")
    desc = w["model"]
    P = synth.model_params(desc, 0)
    rng = np.random.default_rng(32)
    lam = 20.0 * rng.standard_normal((len(w["coords"]), 3))
    cE = 0.3
    g = oracle.param_grad(desc, P, w["coords"], w["types"], w["box"], cE, lam)
    offs, off = {}, 0
    for name, shape in synth.layer_shapes(desc):
        offs[name] = off
        off += int(np.prod(shape))
    picks = [offs["emb00.W0"] + 3, offs["emb01.b0"] + 7, offs["emb10.W1"] + 111, offs["emb11.b2"] + 42,
             offs["emb01.W2"] + 2500, offs["fit0.W1"] + 5000, offs["fit1.W2"] + 777, offs["fit0.wo"] + 5,
             offs["fit1.bo"], offs["fit1.b3"] + 9]
    for p in picks:
        def fd(h):
            Pp, Pm = P.copy(), P.copy()
            Pp[p] += h
            Pm[p] -= h
            return (_phi(oracle, desc, Pp, w, cE, lam) - _phi(oracle, desc, Pm, w, cE, lam)) / (2 * h)
        d1, d2 = fd(2e-4), fd(1e-4)
        rich = (4 * d2 - d1) / 3
        assert rich == pytest.approx(g[p], rel=1e-5, abs=1e-8 * max(1.0, np.abs(g).max()))


def test_eval_local_partition_additivity(oracle, synth):
    """Sub-region evaluation: with every atom a centre it is the whole-system
    evaluation; over a partition of the centres (the rest as ghosts) the
    energies, forces and virials add up to the whole system's."""
    w = synth.workload("water192")
    desc = w["model"]
    P = synth.model_params(desc, 0)
    N = len(w["coords"])
    ref = oracle.evaluate(desc, P, w["coords"], w["types"], w["box"])
    full = oracle.evaluate_local(desc, P, w["coords"], w["types"], w["box"], N)
    assert full["energy"] == ref["energy"]
    assert np.array_equal(full["force"], ref["force"])
    perm = np.random.default_rng(3).permutation(N)
    E, F, V = 0.0, np.zeros((N, 3)), np.zeros((3, 3))
    for part in (perm[:70], perm[70:150], perm[150:]):
        order = np.concatenate([part, np.setdiff1d(np.arange(N), part)])
        r = oracle.evaluate_local(desc, P, w["coords"][order], w["types"][order], w["box"], len(part))
        E += r["energy"]
        F[order] += r["force"]
        V += r["virial"]
    assert E == pytest.approx(ref["energy"], rel=1e-13)
    assert np.abs(F - ref["force"]).max() < 1e-13 * np.abs(ref["force"]).max()
    assert np.abs(V - ref["virial"]).max() < 1e-12 * np.abs(ref["virial"]).max()

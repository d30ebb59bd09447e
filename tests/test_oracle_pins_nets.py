"""Pins of the oracle's embedding and fitting nets with every weight non-zero.

The invariance, finite-difference and strain pins hold for any smooth
function of the descriptor, so they cannot see a transposed weight matrix, a
dropped skip or a concatenation in the wrong order.  Here the atomic energies
of small clusters are recomputed by a plain numpy forward pass written from
the equations of Sec. 2, independently of the oracle:

  environment row   R~_k = s(r)(1, x/r, y/r, z/r)              (Algorithm 2)
  embedding layer 0 h = tanh(s W_0 + b_0)                        (Eq. embedding-first)
  embedding layer l h = skip(h) + tanh(h W_l + b_l)              (Eq. embedding-rest)
                    skip = (h, h) when the width doubles, h when it is equal,
                    none otherwise
  descriptor        T = R~^T G / N_m,  D = T[:, :M2]^T T          (Eq. descrpt)
  fitting           h = tanh(D W_1 + b_1); equal widths add h;  E_i = h w_o + b_o
                                                                 (Eqs. fitting, fitting-detail)

with one embedding net per ordered type pair and one fitting net per centre
type (Remark 1).  Weights are stored input-index first (W[in][out]).  The
cases cover each skip kind of the embedding net (doubling, equal, none) and a
fitting net with two equal-width residual layers after its first layer.
Forces are then tied to this energy by central differences.
"""
import numpy as np
import pytest


def _views(S, desc, P):
    out, off = {}, 0
    for name, shape in S.layer_shapes(desc):
        n = int(np.prod(shape))
        out[name] = P[off:off + n].reshape(shape)
        off += n
    assert off == len(P)
    return out


def _s(r, rs, rc):
    """s(r) = w(r)/r, quintic gate between rs and rc (the reading of Sec. 2's gate)."""
    if r < rs:
        return 1.0 / r
    if r >= rc:
        return 0.0
    u = (r - rs) / (rc - rs)
    return (u ** 3 * (-6 * u * u + 15 * u - 10) + 1) / r


def _layer(h, W, b):
    out = np.tanh(h @ W + b)
    n_in, n_out = W.shape
    if n_out == 2 * n_in:
        return np.concatenate([h, h]) + out
    if n_out == n_in:
        return h + out
    return out


def _atom_energies(desc, V, x, types, box):
    """E_i of every atom of a small system, all pairs within rcut (no sel overflow)."""
    N = len(x)
    nm = sum(desc["sel"])
    M, M2 = desc["emb"][-1], desc["m2"]
    scale = 1.0 / nm if desc.get("desc_scale_nm", 1) else 1.0
    E = np.zeros(N)
    for i in range(N):
        T = np.zeros((4, M))
        for j in range(N):
            if j == i:
                continue
            d = x[j] - x[i]
            d = d - box * np.rint(d / box)
            r = np.sqrt(d @ d)
            s = _s(r, desc["rcut_smth"], desc["rcut"])
            if s == 0.0:
                continue
            R = s * np.array([1.0, d[0] / r, d[1] / r, d[2] / r])
            net = f"emb{types[i]}{types[j]}"
            h = np.tanh(s * V[f"{net}.W0"] + V[f"{net}.b0"])
            for l in range(1, len(desc["emb"])):
                h = _layer(h, V[f"{net}.W{l}"], V[f"{net}.b{l}"])
            T += np.outer(R, h)
        T *= scale
        D = (T[:, :M2].T @ T).ravel()
        fit = f"fit{types[i]}"
        h = np.tanh(D @ V[f"{fit}.W1"] + V[f"{fit}.b1"])
        for l in range(2, len(desc["fit"]) + 1):
            h = _layer(h, V[f"{fit}.W{l}"], V[f"{fit}.b{l}"])
        E[i] = h @ V[f"{fit}.wo"] + V[f"{fit}.bo"][0]
    return E


BASE = dict(ntypes=2, sel=(3, 4), rcut=4.0, rcut_smth=1.0, m2=2, desc_scale_nm=1)
CASES = {
    # widths (input 1) 1-2-4: layer 1 doubles -> (h, h) + tanh
    "emb_2_4": dict(BASE, emb=(2, 4), fit=(5, 5, 5)),
    # 1-2-4-8: two doubling layers (the paper's shape, scaled down)
    "emb_2_4_8": dict(BASE, emb=(2, 4, 8), fit=(6, 6)),
    # 1-3-3-5: an equal-width layer (h + tanh), then a layer without skip
    "emb_3_3_5": dict(BASE, emb=(3, 3, 5), m2=3, fit=(4, 4, 4)),
    # 1-4-6: no skip at all; fitting without residual layers
    "emb_4_6": dict(BASE, emb=(4, 6), fit=(7, 3)),
    # unscaled descriptor with every weight non-zero
    "unscaled": dict(BASE, emb=(2, 4, 8), fit=(5, 5), desc_scale_nm=0),
}


def _cluster(seed, N=6, ntypes=2):
    rng = np.random.default_rng(seed)
    box = np.array([40.0, 41.0, 42.0])
    c = np.array([20.0, 20.0, 20.0])
    x = c + rng.uniform(-1.6, 1.6, (N, 3))
    # keep every pair apart by at least 0.7 A (so r spans all three gate regions)
    for _ in range(200):
        d = np.linalg.norm(x[:, None] - x[None], axis=-1) + np.eye(N) * 9
        if d.min() > 0.7:
            break
        x = c + rng.uniform(-1.6, 1.6, (N, 3))
    t = (np.arange(N) % ntypes).astype(np.int32)
    rng.shuffle(t)
    return x, t, box


def _params(S, desc, seed):
    # a first-layer gain of 3 keeps the fitting pre-activations away from saturation
    P = S.model_params(desc, seed, fit_in_gain=3.0, out_scale=1.0)
    V = _views(S, desc, P)
    for a in range(desc["ntypes"]):      # the seeded output bias is 0: give it a value
        V[f"fit{a}.bo"][0] = 0.3 * (a + 1)
    for name, arr in V.items():          # every weight and bias is non-zero
        assert np.all(arr != 0.0), name
    return P, V


@pytest.mark.parametrize("case", sorted(CASES))
def test_atom_energies_match_equations(oracle, synth, case):
    desc = CASES[case]
    P, V = _params(synth, desc, 11)
    x, t, box = _cluster(21)
    out = oracle.evaluate(desc, P, x, t, box)
    assert out["overflow"] == 0
    assert np.all(out["nreal"].sum(1) > 0)
    exp = _atom_energies(desc, V, x, t, box)
    np.testing.assert_allclose(out["atom_energy"], exp, rtol=1e-12, atol=1e-14)
    assert out["energy"] == pytest.approx(exp.sum(), rel=1e-12)


@pytest.mark.parametrize("case", ["emb_2_4_8", "emb_3_3_5"])
def test_forces_match_equations_gradient(oracle, synth, case):
    """F = -dE/dx of the numpy energy above (Richardson-extrapolated central
    differences), so the oracle's back-propagation through these nets is tied
    to the equations as well."""
    desc = CASES[case]
    P, V = _params(synth, desc, 12)
    x, t, box = _cluster(22)
    out = oracle.evaluate(desc, P, x, t, box)

    def e(xx):
        return _atom_energies(desc, V, xx, t, box).sum()

    fd = np.zeros_like(x)
    for i in range(len(x)):
        for a in range(3):
            def c(h):
                xp, xm = x.copy(), x.copy()
                xp[i, a] += h
                xm[i, a] -= h
                return (e(xp) - e(xm)) / (2 * h)
            h = 1e-4
            fd[i, a] = -(4 * c(h / 2) - c(h)) / 3
    scale = np.abs(out["force"]).max()
    assert scale > 0
    np.testing.assert_allclose(out["force"], fd, rtol=0, atol=1e-8 * scale)


def test_weight_layout_is_input_index_first(oracle, synth):
    """A square embedding layer and its transpose give different energies, and
    the oracle agrees with the input-index-first one only."""
    desc = CASES["emb_3_3_5"]
    P, V = _params(synth, desc, 13)
    x, t, box = _cluster(23)
    out = oracle.evaluate(desc, P, x, t, box)
    VT = {k: v.copy() for k, v in V.items()}
    for net in ("emb00", "emb01", "emb10", "emb11"):
        VT[f"{net}.W1"] = V[f"{net}.W1"].T.copy()
    good = _atom_energies(desc, V, x, t, box)
    bad = _atom_energies(desc, VT, x, t, box)
    assert np.abs(good - bad).max() > 1e-6 * np.abs(good).max()
    np.testing.assert_allclose(out["atom_energy"], good, rtol=1e-12, atol=1e-14)

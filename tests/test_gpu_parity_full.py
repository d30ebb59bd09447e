"""Parity at the paths the kernels take at full size (Algorithm 1 and the
packed keys of Sec. 3.2.2):

* exact ties: perfect lattices (zero jitter) put whole shells of neighbours
  at one distance, so equal (type, floor(|r| 1e8)) keys are ordered by the
  smaller index j on the GPU as in the oracle;
* the 393,216-atom water box: indices j >= 2^15 and N > 2^16 in the packed
  keys; formatted list bit-exact, E/F/virial within 1e-10 of the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11658_gb300 import dp as _dp
    _dp.lib()
    return _dp


def lattice(synth, name):
    if name == "cu_fcc_perfect_864":
        c, t, b = synth.copper_fcc(6, jitter_frac=0.0)
        return dict(coords=c, types=t, box=b, model=synth.CU_MODEL)
    if name == "cu_fcc_perfect_2048":
        c, t, b = synth.copper_fcc(8, jitter_frac=0.0)
        return dict(coords=c, types=t, box=b, model=synth.CU_MODEL)
    if name == "water_lattice_648":
        # O atoms on a perfect simple-cubic lattice (no jitter): every O-O shell ties
        c, t, b = synth.water_box(6, 6 * 49.7 / 16, jitter=0.0)
        return dict(coords=c, types=t, box=b, model=synth.WATER_MODEL)
    raise KeyError(name)


def rel_errors(g, o):
    eE = abs(g["energy"].item() - o["energy"]) / abs(o["energy"])
    F = g["force"].cpu().numpy()
    eF = np.abs(F - o["force"]).max() / np.abs(o["force"]).max()
    V = g["virial"].cpu().numpy().reshape(3, 3)
    eV = np.abs(V - o["virial"]).max() / np.abs(o["virial"]).max()
    return eE, eF, eV


def _ties(nlist, coords, box):
    """Number of adjacent kept pairs with the same distance quantum."""
    x = coords
    n = 0
    for i in range(min(len(x), 64)):
        js = nlist[i][nlist[i] >= 0]
        d = x[js] - x[i]
        d -= box * np.rint(d / box)
        q = np.floor(np.sqrt((d * d).sum(1)) * 1e8)
        n += int((q[1:] == q[:-1]).sum())
    return n


@pytest.mark.parametrize("name", ["cu_fcc_perfect_864", "cu_fcc_perfect_2048", "water_lattice_648"])
@pytest.mark.parametrize("skin", [0.0, 2.0])
def test_format_ties_bit_exact(dp, oracle, synth, name, skin):
    w = lattice(synth, name)
    d = w["model"]
    N = len(w["coords"])
    cap = oracle.default_cap(d, w["box"], N, skin)
    ncand, cand, over = oracle.candidates(w["coords"], w["box"], d["rcut"] + skin, cap)
    assert over == 0
    onl, onr, _ = oracle.format_nlist(w["coords"], w["types"], w["box"], ncand, cand, d["sel"], d["rcut"])
    assert _ties(onl, w["coords"], w["box"]) > 100, "the lattice should produce exact ties"
    model = dp.Model(d, synth.model_params(d, 0))
    ctx = dp.Context(model, N)
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], skin)
    nl, nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"])
    np.testing.assert_array_equal(nl.cpu().numpy(), onl)
    np.testing.assert_array_equal(nr.cpu().numpy(), onr)


@pytest.mark.parametrize("name", ["cu_fcc_perfect_864", "water_lattice_648"])
def test_eval_parity_on_lattices(dp, oracle, synth, name):
    w = lattice(synth, name)
    d = w["model"]
    P = synth.model_params(d, 0)
    o = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
    model = dp.Model(d, P)
    ctx = dp.Context(model, len(w["coords"]))
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 0.0)
    g = dp.dp_eval(ctx, x, t, w["box"])
    eE, eF, eV = rel_errors(g, o)
    # on a perfect lattice forces cancel to rounding: compare against the scale of the terms
    if name.startswith("cu"):
        assert eE < TOL
        fo = np.abs(o["force"]).max()
        assert np.abs(g["force"].cpu().numpy() - o["force"]).max() < 1e-12 + TOL * fo
    else:
        assert eE < TOL and eF < TOL and eV < TOL, (eE, eF, eV)


@pytest.mark.slow
def test_water393216_parity(dp, oracle, synth):
    """The 393,216-atom water box of the benchmark (131,072 H2O, 157.6 A):
    formatted list (2 A skin candidates) bit-exact with the oracle's, energy,
    forces and virial within 1e-10."""
    w = synth.workload("water393216")
    d = w["model"]
    P = synth.model_params(d, 0)
    N = len(w["coords"])
    assert N > 2 ** 16
    o = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
    model = dp.Model(d, P)
    ctx = dp.Context(model, N)
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 2.0)
    nl, nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"])
    nl = nl.cpu().numpy()
    np.testing.assert_array_equal(nl, o["nlist"])
    np.testing.assert_array_equal(nr.cpu().numpy(), o["nreal"])
    assert nl.max() >= 2 ** 18          # neighbour indices use the high bits of the key's j field
    g = dp.dp_eval(ctx, x, t, w["box"], want_atom_energy=True)
    eE, eF, eV = rel_errors(g, o)
    print(f"water393216: E {eE:.2e} F {eF:.2e} V {eV:.2e}")
    assert eE < TOL and eF < TOL and eV < TOL, (eE, eF, eV)
    ea = np.abs(g["atom_energy"].cpu().numpy() - o["atom_energy"]).max() / np.abs(o["atom_energy"]).max()
    assert ea < TOL

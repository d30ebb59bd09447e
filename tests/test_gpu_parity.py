"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: formatted neighbour lists bit-exact (integer work); energy, forces and
virial within 1e-10 relative (norm-wise: |dE|/|E|, max|dF|/max|F|,
max|dXi|/max|Xi|), the paper's own FP64 agreement of 10+ digits (Sec. 6).
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


def system(synth, name):
    if name == "water648":
        return synth.sub_box_water(6, 6 * 49.7 / 16)
    if name == "cu864":
        c, t, b = synth.copper_fcc(6)
        return dict(coords=c, types=t, box=b, model=synth.CU_MODEL, masses=(synth.MASS["Cu"],))
    return synth.workload(name)


_oracle_cache = {}


def oracle_eval(oracle, synth, name, desc=None, seed=0):
    key = (name, repr(desc), seed)
    if key not in _oracle_cache:
        w = system(synth, name)
        d = desc or w["model"]
        P = synth.model_params(d, seed)
        out = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
        _oracle_cache[key] = (w, d, P, out)
    return _oracle_cache[key]


def oracle_nlist(oracle, w, desc, skin):
    """Algorithm 1 by the oracle from candidates built with rcut + skin."""
    cap = oracle.default_cap(desc, w["box"], len(w["coords"]), skin)
    ncand, cand, over = oracle.candidates(w["coords"], w["box"], desc["rcut"] + skin, cap)
    assert over == 0
    nl, nr, _ = oracle.format_nlist(w["coords"], w["types"], w["box"], ncand, cand, desc["sel"], desc["rcut"])
    return nl, nr


def gpu_run(dp, desc, P, w, skin=0.0, cand_cap=0, precision=None):
    N = len(w["coords"])
    model = dp.Model(desc, P)
    ctx = dp.Context(model, N, cand_cap=cand_cap, precision=dp.DP_PREC_FP64 if precision is None else precision)
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], skin)
    return model, ctx, x, t


def rel_errors(g, o):
    eE = abs(g["energy"].item() - o["energy"]) / abs(o["energy"])
    F = g["force"].cpu().numpy()
    eF = np.abs(F - o["force"]).max() / np.abs(o["force"]).max()
    V = g["virial"].cpu().numpy().reshape(3, 3)
    eV = np.abs(V - o["virial"]).max() / np.abs(o["virial"]).max()
    return eE, eF, eV


@pytest.mark.parametrize("name", ["water192", "water648", "cu864"])
def test_format_bit_exact(dp, oracle, synth, name):
    w, d, P, o = oracle_eval(oracle, synth, name)
    model, ctx, x, t = gpu_run(dp, d, P, w)
    nl, nr, s = dp.dp_format_nlist(ctx, x, t, w["box"])
    np.testing.assert_array_equal(nl.cpu().numpy(), o["nlist"])
    np.testing.assert_array_equal(nr.cpu().numpy(), o["nreal"])


@pytest.mark.parametrize("name", ["water192", "water648", "cu864"])
@pytest.mark.parametrize("fit", ["tensor", "simt"])
def test_eval_parity(dp, oracle, synth, name, fit):
    """FP64 modes: the fitting net's GEMMs on the tensor cores by exact
    splitting (DP_PREC_FP64) and on the FP64 units (DP_PREC_FP64_SIMT)."""
    w, d, P, o = oracle_eval(oracle, synth, name)
    prec = dp.DP_PREC_FP64 if fit == "tensor" else dp.DP_PREC_FP64_SIMT
    model, ctx, x, t = gpu_run(dp, d, P, w, precision=prec)
    g = dp.dp_eval(ctx, x, t, w["box"], want_atom_energy=True)
    eE, eF, eV = rel_errors(g, o)
    print(f"{name} {fit}: E {eE:.2e} F {eF:.2e} V {eV:.2e}")
    assert eE < TOL and eF < TOL and eV < TOL, (eE, eF, eV)
    ea = np.abs(g["atom_energy"].cpu().numpy() - o["atom_energy"]).max() / np.abs(o["atom_energy"]).max()
    assert ea < TOL


def test_eval_with_skin_list_matches(dp, oracle, synth):
    """Candidates built with a 2 A skin: Algorithm 1 keeps the candidates
    within rcut only (L(i) of Sec. 2), so the formatted list equals the
    oracle's from the same skin candidates and also its rcut-only list; the
    energy, forces and virial equal those of the rcut-only evaluation."""
    w, d, P, o = oracle_eval(oracle, synth, "water648")
    model, ctx, x, t = gpu_run(dp, d, P, w, skin=2.0)
    nl, nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"])
    onl, onr = oracle_nlist(oracle, w, d, 2.0)
    np.testing.assert_array_equal(nl.cpu().numpy(), onl)
    np.testing.assert_array_equal(nr.cpu().numpy(), onr)
    np.testing.assert_array_equal(nr.cpu().numpy(), o["nreal"])
    g = dp.dp_eval(ctx, x, t, w["box"])
    assert max(rel_errors(g, o)) < TOL


@pytest.mark.parametrize("variant", ["student", "unscaled", "e1_20", "fit_200"])
def test_model_variants(dp, oracle, synth, variant):
    """Other net shapes: the student widths; the unscaled descriptor; an
    embedding net (20, 40, 80) that the tensor-core embedding kernels do not
    take (FP64-unit embedding kernels with the tensor-core fitting net); a
    fitting net of width 200 (column chunks with a ragged last one)."""
    if variant == "student":
        desc = synth.WATER_STUDENT
    elif variant == "e1_20":
        desc = dict(synth.WATER_MODEL, emb=(20, 40, 80))
    elif variant == "fit_200":
        desc = dict(synth.WATER_MODEL, fit=(200, 200))
    else:
        desc = dict(synth.WATER_MODEL, desc_scale_nm=0)
    w, d, P, o = oracle_eval(oracle, synth, "water192", desc=desc)
    if variant == "unscaled":
        P = synth.model_params(d, 0, fit_in_gain=300.0 / 138 ** 2)
        o = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
    model, ctx, x, t = gpu_run(dp, d, P, w)
    g = dp.dp_eval(ctx, x, t, w["box"])
    assert max(rel_errors(g, o)) < TOL


def test_deterministic(dp, oracle, synth):
    w, d, P, o = oracle_eval(oracle, synth, "water648")
    model, ctx, x, t = gpu_run(dp, d, P, w)
    a = dp.dp_eval(ctx, x, t, w["box"])
    b = dp.dp_eval(ctx, x, t, w["box"])
    assert torch.equal(a["force"], b["force"]) and torch.equal(a["energy"], b["energy"])
    assert torch.equal(a["virial"], b["virial"])


def test_sel_overflow_matches_truncated_oracle(dp, oracle, synth):
    w = synth.workload("water192")
    d = dict(w["model"], sel=(20, 40))
    P = synth.model_params(d, 0)
    o = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
    assert o["overflow"] > 0
    model, ctx, x, t = gpu_run(dp, d, P, w)
    g = dp.dp_eval(ctx, x, t, w["box"], check=False)
    assert g["status"] == -3  # DP_ERR_SEL_OVERFLOW, results written
    assert max(rel_errors(g, o)) < TOL


def test_isolated_and_single_atoms(dp, oracle, synth):
    d = synth.WATER_MODEL
    P = synth.model_params(d, 0)
    # a molecule far from a small cluster: atoms with no neighbour at all
    w = synth.workload("water192")
    x = np.concatenate([w["coords"][:30] + 10.0, np.array([[45.0, 45.0, 45.0]])])
    t = np.concatenate([w["types"][:30], np.array([1], np.int32)])
    box = np.array([60.0, 60.0, 60.0])
    o = oracle.evaluate(d, P, x, t, box)
    ws = dict(coords=x, types=t, box=box)
    model, ctx, xg, tg = gpu_run(dp, d, P, ws)
    g = dp.dp_eval(ctx, xg, tg, box, want_atom_energy=True)
    assert max(rel_errors(g, o)) < TOL
    assert np.all(g["force"].cpu().numpy()[-1] == 0.0)
    # N = 1
    ws1 = dict(coords=np.array([[1.0, 2.0, 3.0]]), types=np.array([0], np.int32), box=box)
    o1 = oracle.evaluate(d, P, ws1["coords"], ws1["types"], box)
    model1, ctx1, x1, t1 = gpu_run(dp, d, P, ws1)
    g1 = dp.dp_eval(ctx1, x1, t1, box)
    assert g1["energy"].item() == pytest.approx(o1["energy"], rel=TOL)
    assert torch.all(g1["force"] == 0)


def test_errors_are_reported(dp, synth):
    w = synth.workload("water192")
    d = w["model"]
    P = synth.model_params(d, 0)
    model, ctx, x, t = gpu_run(dp, d, P, w)
    # non-orthorhombic cell
    b = np.diag(w["box"]).copy()
    b[0, 1] = 0.1
    with pytest.raises(dp.DPError) as e:
        dp.dp_eval(ctx, x, t, b)
    assert e.value.status == -2
    # cell too small for rcut + skin
    with pytest.raises(dp.DPError) as e:
        dp.dp_build_nlist(ctx, x, t, w["box"], skin=1.0)
    assert e.value.status == -2
    # type out of range
    tb = t.clone()
    tb[5] = 7
    s = dp.dp_build_nlist(ctx, x, tb, w["box"], 0.0, check=False)
    assert s == -11
    g = dp.dp_eval(ctx, x, tb, w["box"], check=False)
    assert g["status"] == -11
    # wrong parameter count
    with pytest.raises(dp.DPError):
        dp.Model(d, P[:-1])


def test_model_file_round_trip(dp, oracle, synth, tmp_path):
    w, d, P, o = oracle_eval(oracle, synth, "water192")
    m1 = dp.Model(d, P)
    path = str(tmp_path / "water.dpm")
    m1.save(path)
    m2 = dp.Model.load(path, desc=d)
    ctx = dp.Context(m2, len(w["coords"]))
    x = torch.tensor(w["coords"], device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    g = dp.dp_eval(ctx, x, t, w["box"])
    assert max(rel_errors(g, o)) < TOL
    with open(path, "r+b") as f:
        f.truncate(1000)
    with pytest.raises(dp.DPError) as e:
        dp.Model.load(path)
    assert e.value.status == -6


def test_md_parity_small(dp, oracle, synth):
    """dp_md_step against the oracle's velocity Verlet (water192, rebuild every
    step since the 12.42 A cell leaves no room for a skin)."""
    w = synth.workload("water192")
    d = w["model"]
    P = synth.model_params(d, 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=2)
    n = 20
    xo, vo, fo, tho, _ = oracle.md(d, P, w["coords"], v0, w["types"], w["box"], w["masses"], 0.5, n,
                                   rebuild_every=1, skin=0.0)
    model = dp.Model(d, P)
    ctx = dp.Context(model, len(m))
    x = torch.tensor(w["coords"], device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    th = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], 0.5, n, rebuild_every=1, skin=0.0, thermo=th)
    th = th.cpu().numpy()
    np.testing.assert_allclose(th[:, 0], tho[:, 0], rtol=1e-9)
    np.testing.assert_allclose(th[:, 1], tho[:, 1], rtol=1e-9)
    np.testing.assert_allclose(th[:, 3], tho[:, 3], rtol=1e-8, atol=1e-12)
    dx = x.cpu().numpy() - xo
    dx -= w["box"] * np.round(dx / w["box"])
    assert np.abs(dx).max() < 1e-9
    np.testing.assert_allclose(v.cpu().numpy(), vo, atol=1e-10)


def test_md_parity_with_skin(dp, oracle, synth):
    """Skin list rebuilt every 10 steps (water648, 2 A skin), 30 steps."""
    w = system(synth, "water648")
    d = w["model"]
    P = synth.model_params(d, 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=2)
    n = 30
    xo, vo, fo, tho, st = oracle.md(d, P, w["coords"], v0, w["types"], w["box"], w["masses"], 0.5, n,
                                    rebuild_every=10, skin=2.0)
    model = dp.Model(d, P)
    ctx = dp.Context(model, len(m))
    x = torch.tensor(w["coords"], device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    th = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    # two calls of 15 steps: the context keeps the force and the step counter
    dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], 0.5, 15, rebuild_every=10, skin=2.0, thermo=th[:15])
    dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], 0.5, 15, rebuild_every=10, skin=2.0, thermo=th[15:])
    th = th.cpu().numpy()
    np.testing.assert_allclose(th[:, 0], tho[:, 0], rtol=1e-9)
    np.testing.assert_allclose(th[:, 1], tho[:, 1], rtol=1e-9)
    f = dp.dp_md_get_force(ctx, len(m)).cpu().numpy()
    assert np.abs(f - fo).max() < 1e-8 * np.abs(fo).max()


@pytest.mark.slow
@pytest.mark.parametrize("name", ["water12288", "cu32000"])
def test_full_size_parity(dp, oracle, synth, name):
    """Full benchmark sizes (12,288-atom water, 32,000-atom copper): formatted
    list bit-exact, E/F/virial within 1e-10 of the oracle."""
    w, d, P, o = oracle_eval(oracle, synth, name)
    model, ctx, x, t = gpu_run(dp, d, P, w, skin=2.0)
    nl, nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"])
    onl, onr = oracle_nlist(oracle, w, d, 2.0)
    np.testing.assert_array_equal(nl.cpu().numpy(), onl)
    np.testing.assert_array_equal(nr.cpu().numpy(), onr)
    g = dp.dp_eval(ctx, x, t, w["box"])
    eE, eF, eV = rel_errors(g, o)
    assert eE < TOL and eF < TOL and eV < TOL, (eE, eF, eV)


def test_md_parity_early_rebuild(dp, oracle, synth):
    """With a 0.5 A skin and a rebuild period longer than the run, the list is
    rebuilt on the device whenever an atom has moved more than skin/2; the
    oracle applies the same rule."""
    w = system(synth, "water648")
    d = w["model"]
    P = synth.model_params(d, 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 600.0, seed=3)
    n = 40
    xo, vo, fo, tho, st = oracle.md(d, P, w["coords"], v0, w["types"], w["box"], w["masses"], 0.5, n,
                                    rebuild_every=1000, skin=0.5)
    model = dp.Model(d, P)
    ctx = dp.Context(model, len(m))
    x = torch.tensor(w["coords"], device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    th = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    builds0 = ctx.launches
    dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], 0.5, n, rebuild_every=1000, skin=0.5, thermo=th)
    th = th.cpu().numpy()
    np.testing.assert_allclose(th[:, 0], tho[:, 0], rtol=1e-9)
    np.testing.assert_allclose(th[:, 1], tho[:, 1], rtol=1e-9)
    dx = x.cpu().numpy() - xo
    dx -= w["box"] * np.round(dx / w["box"])
    assert np.abs(dx).max() < 1e-9
    assert ctx.launches > builds0


def test_fp64_tanh_accuracy(dp):
    """The FP64 kernels' tanh against CUDA's tanh and the host libm."""
    rng = np.random.default_rng(21)
    x = np.concatenate([np.linspace(-25, 25, 2_000_001), rng.normal(0, 3, 1_000_000),
                        np.array([0.0, -0.0, 1e-300, -1e-300, 1e-12, 0.0125, 0.0124999999, 19.124999, 19.125,
                                  -19.125, 30.0, 1e300, -1e300])])
    xt = torch.tensor(x, device="cuda")
    y = dp.dp_tanh_f64(xt).cpu().numpy()
    ref_cuda = torch.tanh(xt).cpu().numpy()
    ref_host = np.tanh(x)
    assert np.abs(y - ref_host).max() < 4e-16
    assert np.abs(y - ref_cuda).max() < 4e-16
    # relative error: a few 1e-15 where an interval's polynomial cancels
    # (the first intervals away from 0, tanh ~ x), tight in the interval at 0
    # (|x| <= 1/80), where it is the Taylor series at 0
    nz = x != 0
    assert (np.abs(y - ref_host)[nz] / np.abs(ref_host[nz])).max() < 1e-14
    small = (np.abs(x) <= 1.0 / 80) & nz
    assert (np.abs(y - ref_host)[small] / np.abs(ref_host[small])).max() < 1.5e-15
    z = np.where(x == 0.0)[0]
    assert np.all(y[z] == 0.0) and np.array_equal(np.signbit(y[z]), np.signbit(x[z]))
    nan = dp.dp_tanh_f64(torch.tensor([float("nan")], dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.isnan(nan[0])


def test_set_params_refreshes_fp64_contexts(dp, oracle, synth):
    """After dp_model_set_params an existing FP64 context evaluates the new
    parameters (the tensor-core fitting net re-makes its weight digits)."""
    w, d, P, o = oracle_eval(oracle, synth, "water192")
    model, ctx, x, t = gpu_run(dp, d, P, w)
    dp.dp_eval(ctx, x, t, w["box"])
    P2 = synth.model_params(d, 5)
    model.set_params(P2)
    g = dp.dp_eval(ctx, x, t, w["box"])
    o2 = oracle.evaluate(d, P2, w["coords"], w["types"], w["box"])
    assert max(rel_errors(g, o2)) < TOL


def test_model_from_seed_matches_oracle(dp, oracle, synth):
    """A model made in the library from a seed (dp_model_from_seed) is the
    input module's seeded model: parameters equal value for value on this
    machine's libm, and the evaluation matches the oracle's on those weights."""
    w = system(synth, "water648")
    d = w["model"]
    P = synth.model_params(d, 7)
    np.testing.assert_array_equal(dp.dp_model_params_from_seed(d, 7), P)
    o = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
    model = dp.Model.from_seed(d, 7)
    ctx = dp.Context(model, len(w["coords"]))
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 0.0)
    g = dp.dp_eval(ctx, x, t, w["box"])
    eE, eF, eV = rel_errors(g, o)
    assert eE < TOL and eF < TOL and eV < TOL, (eE, eF, eV)

"""dp_eval_local (sub-region evaluation, Sec. 3.1) against the oracle, and
slab decompositions emulated on one GPU against the whole-system dp_eval."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11658_gb300 import dp as _dp
    _dp.lib()
    return _dp


def _water648(synth):
    return synth.sub_box_water(6, 6 * 49.7 / 16)


def _sub_region(domain, w, nslab, q):
    desc = w["model"]
    plan = domain.make_plan(w["coords"], w["box"], nslab, ghost_width=desc["rcut"], pad=desc["rcut"] + 1.0)
    x = torch.tensor(w["coords"])
    t = torch.tensor(w["types"])
    xo = [x[torch.as_tensor(plan.owned[p])] for p in range(nslab)]
    to = [t[torch.as_tensor(plan.owned[p])] for p in range(nslab)]
    ghosts = torch.cat([domain._pack_positions(plan, p, q, xo[p]) for p in range(nslab)], 0)
    tg = torch.cat([to[p][torch.as_tensor(plan.send[p][q][0])] for p in range(nslab)], 0)
    xs = domain._sub_region_coords(plan, q, xo[q], ghosts)
    ts = torch.cat([to[q], tg], 0)
    return xs.numpy(), ts.numpy(), plan.sub_box(), len(plan.owned[q])


@pytest.mark.parametrize("nslab,q", [(2, 0), (3, 1)])
def test_eval_local_matches_oracle(dp, oracle, synth, nslab, q):
    from paper_2004_11658_gb300 import domain
    w = _water648(synth)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    xs, ts, box, nloc = _sub_region(domain, w, nslab, q)
    N = len(xs)
    cap = oracle.default_cap(desc, w["box"], len(w["coords"]), 0.0)
    ref = oracle.evaluate_local(desc, P, xs, ts, box, nloc, cap=cap)
    model = dp.Model(desc, P)
    ctx = dp.Context(model, N, cand_cap=cap)
    x = torch.tensor(xs, device="cuda")
    t = torch.tensor(ts, device="cuda")
    dp.dp_build_nlist(ctx, x, t, box, 0.0)
    ae = torch.empty(nloc, dtype=torch.float64, device="cuda")
    out = dp.dp_eval_local(ctx, x, t, box, nloc, atom_energy=ae)
    F = out["force"].cpu().numpy()
    print(f"slab {q}/{nslab}: nloc {nloc}, ghosts {N - nloc}")
    assert out["energy"].item() == pytest.approx(ref["energy"], rel=1e-10)
    assert np.abs(F - ref["force"]).max() <= 1e-10 * np.abs(ref["force"]).max()
    assert np.abs(out["virial"].cpu().numpy().reshape(3, 3) - ref["virial"]).max() <= \
        1e-10 * np.abs(ref["virial"]).max()
    assert np.abs(ae.cpu().numpy() - ref["atom_energy"]).max() <= 1e-10 * np.abs(ref["atom_energy"]).max()


def test_eval_local_edges(dp, synth):
    """nloc == N is dp_eval bit for bit; nloc == 0 gives zeros; nloc out of
    range is an argument error."""
    w = synth.workload("water192")
    model = dp.Model(w["model"], synth.model_params(w["model"], 0))
    N = len(w["coords"])
    ctx = dp.Context(model, N)
    x = torch.tensor(w["coords"], device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 0.0)
    a = dp.dp_eval(ctx, x, t, w["box"])
    a = {k: v.clone() for k, v in a.items() if torch.is_tensor(v)}
    b = dp.dp_eval_local(ctx, x, t, w["box"], N)
    for k in ("energy", "force", "virial"):
        assert torch.equal(a[k], b[k])
    z = dp.dp_eval_local(ctx, x, t, w["box"], 0)
    assert z["energy"].item() == 0.0
    assert torch.count_nonzero(z["force"]).item() == 0
    assert torch.count_nonzero(z["virial"]).item() == 0
    # a later whole-system call still sees every atom as a centre
    c = dp.dp_eval(ctx, x, t, w["box"])
    assert torch.equal(a["force"], c["force"])
    s = dp.dp_eval_local(ctx, x, t, w["box"], N + 1, check=False)["status"]
    assert s == dp.DP_ERR_ARG


@pytest.mark.parametrize("precision,nslab", [("fp64", 2), ("fp64", 4), ("mixed", 2)])
def test_emulated_slabs_match_whole(dp, synth, precision, nslab):
    from paper_2004_11658_gb300 import domain
    w = synth.workload("water12288")
    desc = w["model"]
    model = dp.Model(desc, synth.model_params(desc, 0))
    N = len(w["coords"])
    prec = dp.DP_PREC_FP64 if precision == "fp64" else dp.DP_PREC_MIXED
    x = torch.tensor(w["coords"], device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    whole = dp.Context(model, N, precision=prec)
    dp.dp_build_nlist(whole, x, t, w["box"], 0.0)
    ref = dp.dp_eval(whole, x, t, w["box"])
    plan = domain.make_plan(w["coords"], w["box"], nslab, ghost_width=desc["rcut"], pad=desc["rcut"] + 1.0)
    nmax = max(len(plan.owned[q]) + len(plan.ghost_src[q]) for q in range(nslab))
    ev = domain.DPLocalEvaluator(model, nmax, N / float(np.prod(w["box"])), precision=prec)
    E, F, V = domain.evaluate_emulated(plan, x, t, ev)
    tol = 1e-10 if precision == "fp64" else 1e-6
    fs = ref["force"].abs().max().item()
    print(f"{precision} {nslab} slabs: |dE|/|E| {abs(E - ref['energy'].item()) / abs(ref['energy'].item()):.2e}, "
          f"max|dF|/max|F| {(F - ref['force']).abs().max().item() / fs:.2e}")
    assert E == pytest.approx(ref["energy"].item(), rel=tol)
    assert (F - ref["force"]).abs().max().item() <= tol * fs
    assert (V.reshape(9) - ref["virial"]).abs().max().item() <= tol * ref["virial"].abs().max().item()


@pytest.mark.parametrize("nslab", [2, 3])
def test_slab_md_matches_single_domain_md(dp, synth, nslab):
    """Velocity-Verlet MD over slabs emulated on one GPU (kicks and drifts by
    dp_md_kick_drift / dp_md_kick, forces by dp_eval_local and the halos,
    re-plans with atom migration every 4 steps) follows the whole-system
    dp_md_step trajectory."""
    from paper_2004_11658_gb300 import domain
    w = _water648(synth)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    N = len(w["coords"])
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=4)
    v0[:, 0] += 0.08          # uniform drift along x: atoms cross slab faces
    model = dp.Model(desc, P)
    n, dt = 16, 1.0
    # whole system
    ctx = dp.Context(model, N)
    x = torch.tensor(w["coords"], device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    th = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], dt, n, rebuild_every=1, skin=0.0, thermo=th)
    # slabs
    rho = N / float(np.prod(w["box"]))
    # a sub-region holds its owned atoms and ghosts, periodic images included: up to ~2 N here
    evs = [domain.DPLocalEvaluator(model, 3 * N, rho) for _ in range(nslab)]
    integ = [domain.GPUIntegrator(e.ctx) for e in evs]
    md = domain.SlabMD(domain.LocalComm(nslab), w["box"], desc["rcut"], 1.0, torch.tensor(w["coords"], device="cuda"),
                       torch.tensor(v0, device="cuda"), torch.tensor(w["types"], device="cuda"), w["masses"], dt,
                       evs, integ, replan_every=4)
    owner0 = {int(g): k for k, s in enumerate(md.s) for g in s["gid"]}
    rows = np.array(md.run(n))
    xs = np.zeros((N, 3))
    vs = np.zeros((N, 3))
    for gid, xx, vv, ff in md.owned():
        xs[gid.cpu().numpy()] = xx.cpu().numpy()
        vs[gid.cpu().numpy()] = vv.cpu().numpy()
    d = xs - x.cpu().numpy()
    d -= w["box"] * np.round(d / w["box"])
    assert np.abs(d).max() < 1e-9
    assert np.abs(vs - v.cpu().numpy()).max() < 1e-10
    th = th.cpu().numpy()
    np.testing.assert_allclose(rows[:, 0], th[:, 0], rtol=1e-11)
    np.testing.assert_allclose(rows[:, 1], th[:, 1], rtol=1e-11)
    owner1 = {int(g): k for k, s in enumerate(md.s) for g in s["gid"]}
    assert sum(owner0[g] != owner1[g] for g in owner0) > 20

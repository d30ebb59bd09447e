"""The FP64 embedding kernels with G and dG/ds kept between the forward and
the backward (k_embed_tan_x + k_embed_bwd_st) and without (k_embed_fwd_x +
k_embed_bwd_x, which recomputes them): both against the oracle (1e-10, the
bar of the other parity tests), against each other, and the context switch.

The back-propagation of Sec. 2 needs, per real neighbour row, G and dG/ds;
keeping or recomputing them changes only the order of the sums over the M
features in the backward, so the atomic energies (forward only) agree to
rounding and the forces and virial to a few ulps of their largest terms.
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


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def evaluate(dp, ctx, x, t, box):
    g = dp.dp_eval(ctx, x, t, box, want_atom_energy=True)
    return {k: v.cpu().numpy() if hasattr(v, "cpu") else v for k, v in g.items()}


# water (e1 = 25, a TMEM quarter of 4 real features), copper (e1 = 32, dense
# quarters), the student widths (e1 = 16, two padding quarters)
@pytest.mark.parametrize("name,student", [("water648", False), ("cu864", False), ("water648", True)])
def test_store_and_recompute_match_oracle(dp, oracle, synth, name, student):
    w = system(synth, name)
    d = synth.WATER_STUDENT if student else w["model"]
    P = synth.model_params(d, 0)
    o = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
    model = dp.Model(d, P)
    ctx = dp.Context(model, len(w["coords"]))
    assert ctx.embed_store, "a small FP64 context keeps G and dG/ds"
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 2.0)
    gs = evaluate(dp, ctx, x, t, w["box"])
    ctx.set_embed_store(False)
    assert not ctx.embed_store
    gr = evaluate(dp, ctx, x, t, w["box"])
    for g in (gs, gr):
        eE = abs(g["energy"].item() - o["energy"]) / abs(o["energy"])
        eF = rel(g["force"], o["force"])
        eV = rel(g["virial"].reshape(3, 3), o["virial"])
        assert eE < TOL and eF < TOL and eV < TOL, (eE, eF, eV)
        assert rel(g["atom_energy"], o["atom_energy"]) < TOL
    # same forward (T, D and the fitting net): atomic energies to rounding
    assert rel(gs["atom_energy"], gr["atom_energy"]) < 1e-14
    assert rel(gs["force"], gr["force"]) < 1e-13
    assert rel(gs["virial"], gr["virial"]) < 1e-13


@pytest.mark.slow
def test_store_and_recompute_agree_at_full_size(dp, synth):
    """The 12,288-atom water box with a 2 A skin (both paths; the store path
    is also the one the full-size oracle parity tests take)."""
    w = synth.workload("water12288")
    d = w["model"]
    model = dp.Model(d, synth.model_params(d, 0))
    ctx = dp.Context(model, len(w["coords"]))
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 2.0)
    ctx.set_embed_store(True)
    gs = evaluate(dp, ctx, x, t, w["box"])
    gs2 = evaluate(dp, ctx, x, t, w["box"])
    ctx.set_embed_store(False)
    gr = evaluate(dp, ctx, x, t, w["box"])
    for k in ("energy", "force", "virial", "atom_energy"):
        np.testing.assert_array_equal(gs[k], gs2[k])  # deterministic
    assert rel(gs["atom_energy"], gr["atom_energy"]) < 1e-14
    assert rel(gs["force"], gr["force"]) < 1e-13
    assert rel(gs["virial"], gr["virial"]) < 1e-13


def test_store_switch(dp, synth):
    """On/off/on on an FP64 context; DP_ERR_UNSUPPORTED for contexts whose
    kernels have no store (split-operand mixed precision, FP64 units only),
    which keep working."""
    w = system(synth, "water648")
    d = w["model"]
    model = dp.Model(d, synth.model_params(d, 0))
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    ctx = dp.Context(model, len(w["coords"]))
    dp.dp_build_nlist(ctx, x, t, w["box"], 0.0)
    ref = evaluate(dp, ctx, x, t, w["box"])
    for on in (False, False, True, True, False):
        ctx.set_embed_store(on)
        assert ctx.embed_store == on
        g = evaluate(dp, ctx, x, t, w["box"])
        assert rel(g["force"], ref["force"]) < 1e-13
    for prec in (dp.DP_PREC_MIXED_SPLIT, dp.DP_PREC_FP64_SIMT):
        c2 = dp.Context(model, len(w["coords"]), precision=prec)
        assert not c2.embed_store
        with pytest.raises(dp.DPError) as ei:
            c2.set_embed_store(True)
        assert ei.value.status == -8
        c2.set_embed_store(False)
        dp.dp_build_nlist(c2, x, t, w["box"], 0.0)
        g = evaluate(dp, c2, x, t, w["box"])
        assert np.isfinite(g["force"]).all()


# mixed precision (plain BF16 operands): G and dG/ds kept in FP32
@pytest.mark.parametrize("name,student", [("water648", False), ("cu864", False), ("water648", True)])
def test_mixed_store_and_recompute(dp, oracle, synth, name, student):
    """k_embed_tan_mx + k_embed_bwd_stmx against k_embed_fwd_mx +
    k_embed_bwd_mx: the same forward (atomic energies to rounding; the same
    FP32 G in both), the backward's double-float sums in another order
    (forces and virial to 1e-11 relative), and both within the mixed bars of
    the FP64 oracle (relative force RMSE in plain BF16: <= 1e-2 for the water
    model, 5e-2 for the student widths, measured 2.4e-2 on this machine, and
    1e-1 for copper)."""
    w = system(synth, name)
    d = synth.WATER_STUDENT if student else w["model"]
    P = synth.model_params(d, 0)
    o = oracle.evaluate(d, P, w["coords"], w["types"], w["box"])
    model = dp.Model(d, P)
    ctx = dp.Context(model, len(w["coords"]), precision=dp.DP_PREC_MIXED)
    assert ctx.embed_store
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 2.0)
    gs = evaluate(dp, ctx, x, t, w["box"])
    gs2 = evaluate(dp, ctx, x, t, w["box"])
    for k in ("energy", "force", "virial", "atom_energy"):
        np.testing.assert_array_equal(gs[k], gs2[k])  # deterministic
    ctx.set_embed_store(False)
    assert not ctx.embed_store
    gr = evaluate(dp, ctx, x, t, w["box"])
    assert rel(gs["atom_energy"], gr["atom_energy"]) < 1e-14
    assert rel(gs["force"], gr["force"]) < 1e-11
    assert rel(gs["virial"], gr["virial"]) < 1e-11
    bar = 1e-1 if name == "cu864" else (5e-2 if student else 1e-2)
    for g in (gs, gr):
        dF = g["force"] - o["force"]
        relrmse = np.sqrt((dF ** 2).mean()) / np.sqrt((o["force"] ** 2).mean())
        assert relrmse < bar, relrmse
    ctx.set_embed_store(True)
    assert ctx.embed_store
    g3 = evaluate(dp, ctx, x, t, w["box"])
    np.testing.assert_array_equal(g3["force"], gs["force"])


def test_store_left_off_when_it_does_not_fit(dp, oracle, synth):
    """dp_ctx_create keeps G and dG/ds only when they take at most half of
    the free device memory: a copper context for 150,000 atoms (sel 512,
    M = 128: 157 GB of rows, more than half of a GB300's memory) is created
    without the store, and evaluates through the recompute kernels."""
    c, t_, b = synth.copper_fcc(6)
    d = synth.CU_MODEL
    P = synth.model_params(d, 0)
    need = 150000 * sum(d["sel"]) * 2 * d["emb"][-1] * 8
    free, _ = torch.cuda.mem_get_info()
    if need <= free // 2:
        pytest.skip("this device holds the rows")
    ctx = dp.Context(dp.Model(d, P), 150000)
    assert not ctx.embed_store
    x = torch.tensor(c, dtype=torch.float64, device="cuda")
    t = torch.tensor(t_, dtype=torch.int32, device="cuda")
    dp.dp_build_nlist(ctx, x, t, b, 0.0)
    g = evaluate(dp, ctx, x, t, b)
    o = oracle.evaluate(d, P, c, t_, b)
    assert rel(g["force"], o["force"]) < TOL
    ctx.close()

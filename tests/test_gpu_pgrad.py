"""Parameter gradients (training path) against the FP64 oracle's gradient
and finite differences; the autograd.Function on top of them."""
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


def system(synth, name):
    if name == "cu864":
        c, t, b = synth.copper_fcc(6)
        return dict(coords=c, types=t, box=b, model=synth.CU_MODEL)
    return synth.workload(name)


@pytest.mark.parametrize("name,variant", [("water192", None), ("water192", "student"), ("cu864", None)])
def test_param_grad_matches_oracle(dp, oracle, synth, name, variant):
    w = system(synth, name)
    desc = synth.WATER_STUDENT if variant == "student" else w["model"]
    P = synth.model_params(desc, 0)
    rng = np.random.default_rng(41)
    N = len(w["coords"])
    lam = 10.0 * rng.standard_normal((N, 3))
    cE = 0.37
    ref = oracle.param_grad(desc, P, w["coords"], w["types"], w["box"], cE, lam)
    model = dp.Model(desc, P)
    ctx = dp.Context(model, N)
    x = torch.tensor(w["coords"], device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 0.0)
    g = dp.dp_param_grad(ctx, x, t, w["box"], cE, torch.tensor(lam, device="cuda")).cpu().numpy()
    err = np.abs(g - ref).max() / np.abs(ref).max()
    print(f"{name} {variant}: max|dgrad|/max|grad| = {err:.2e}")
    assert err < 1e-10
    g2 = dp.dp_param_grad(ctx, x, t, w["box"], cE, torch.tensor(lam, device="cuda")).cpu().numpy()
    assert np.array_equal(g, g2)   # reproducible bit for bit


def test_autograd_loss_gradient(dp, oracle, synth):
    """loss = (E - E0)^2 / N + |F - F0|^2 / N through DPEnergyForces; its
    gradient equals the oracle's parameter gradient with cE = dL/dE and
    lambda = dL/dF, and a directional finite difference of the loss."""
    w = synth.workload("water192")
    desc = w["model"]
    P0 = synth.model_params(desc, 0)
    N = len(w["coords"])
    rng = np.random.default_rng(42)
    E0 = -20.0
    F0 = 0.01 * rng.standard_normal((N, 3))
    model = dp.Model(desc, P0)
    ctx = dp.Context(model, N)
    x = torch.tensor(w["coords"], device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    dp.dp_build_nlist(ctx, x, t, w["box"], 0.0)
    params = torch.tensor(P0, dtype=torch.float64, requires_grad=True)
    F0t = torch.tensor(F0, device="cuda")

    def loss_of(p):
        E, F, V = dp.DPEnergyForces.apply(p, x, t, w["box"], ctx)
        return (E[0] - E0) ** 2 / N + ((F - F0t) ** 2).sum() / N, E, F

    L, E, F = loss_of(params)
    L.backward()
    g = params.grad.numpy()
    cE = 2.0 * (E.item() - E0) / N
    lam = 2.0 * (F.detach().cpu().numpy() - F0) / N
    ref = oracle.param_grad(desc, P0, w["coords"], w["types"], w["box"], cE, lam)
    assert np.abs(g - ref).max() / np.abs(ref).max() < 1e-10
    V = rng.standard_normal(len(P0))
    V /= np.linalg.norm(V)
    with torch.no_grad():
        def Lh(h):
            return float(loss_of(torch.tensor(P0 + h * V))[0])
        d1 = (Lh(2e-4) - Lh(-2e-4)) / 4e-4
        d2 = (Lh(1e-4) - Lh(-1e-4)) / 2e-4
    rich = (4 * d2 - d1) / 3
    assert rich == pytest.approx(float(g @ V), rel=1e-6, abs=1e-12)

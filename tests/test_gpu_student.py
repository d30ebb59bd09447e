"""Student model (embedding net 1-16-32-64): its training loss gradient
through the hand-written kernels against finite differences on 192-atom
frames, and a short training run on teacher-labelled frames."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frames():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11658_gb300 import student, synth
    w = synth.workload("water192")
    return student.generate_frames(w["model"], synth.model_params(w["model"], 0), w, n_traj=4,
                                   frames_per_traj=25)


def test_frames_are_teacher_labels(frames, oracle, synth):
    """Labels are the FP64 teacher's energies and forces (checked against
    the oracle on two frames)."""
    desc = synth.WATER_MODEL
    P = synth.model_params(desc, 0)
    for f in (0, 77):
        x = frames["coords"][f].cpu().numpy()
        ref = oracle.evaluate(desc, P, x, frames["types"].cpu().numpy(), frames["box"])
        assert frames["energy"][f].item() == pytest.approx(ref["energy"], rel=1e-10)
        assert np.abs(frames["force"][f].cpu().numpy() - ref["force"]).max() < 1e-10 * np.abs(ref["force"]).max()


def test_student_loss_gradient_matches_finite_differences(frames, synth):
    from paper_2004_11658_gb300 import dp, student
    S = synth.WATER_STUDENT
    P0 = synth.model_params(S, 7)
    N = frames["coords"].shape[1]
    ctx = dp.Context(dp.Model(S, P0), N)
    sc = float(frames["force"].pow(2).mean().sqrt())
    E_lab, F_lab = frames["energy"] / sc, frames["force"] / sc
    idx = [3, 30, 55, 90]
    p = torch.tensor(P0, dtype=torch.float64, requires_grad=True)
    student.batch_loss(p, ctx, frames, E_lab, F_lab, idx, 1.0, 100.0, backward=True)
    g = p.grad.numpy().copy()
    rng = np.random.default_rng(5)
    checks = []
    for trial in range(2):
        V = rng.standard_normal(len(P0))
        V /= np.linalg.norm(V)

        def L(h):
            with torch.no_grad():
                return student.batch_loss(torch.tensor(P0 + h * V), ctx, frames, E_lab, F_lab, idx, 1.0, 100.0)
        h = 1e-4
        d1 = (L(2 * h) - L(-2 * h)) / (4 * h)
        d2 = (L(h) - L(-h)) / (2 * h)
        fd = (4 * d2 - d1) / 3
        checks.append((fd, float(g @ V)))
    # single parameters: an output weight and a first-layer embedding weight
    for name in ("fit1.wo", "emb01.W0"):
        k = student.param_offset(S, name) + 3
        e = np.zeros(len(P0))
        e[k] = 1.0

        def Lk(h):
            with torch.no_grad():
                return student.batch_loss(torch.tensor(P0 + h * e), ctx, frames, E_lab, F_lab, idx, 1.0, 100.0)
        h = 1e-4 * max(1.0, abs(P0[k]))
        fd = (4 * (Lk(h) - Lk(-h)) / (2 * h) - (Lk(2 * h) - Lk(-2 * h)) / (4 * h)) / 3
        checks.append((fd, float(g[k])))
    for fd, an in checks:
        print(f"fd {fd:.10e} analytic {an:.10e}")
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(g).max())


def test_student_training_reduces_force_error(frames, synth):
    """Adam (lr 1e-3 decaying, batch 4 frames) on three trajectories; the
    force error on the held-out fourth trajectory falls, and the trained
    student in mixed precision stays within 1e-3 eV/A of its FP64 self."""
    from paper_2004_11658_gb300 import dp, student
    S = synth.WATER_STUDENT
    nf = frames["coords"].shape[0]
    train = dict(frames)
    for k in ("coords", "energy", "force"):
        train[k] = frames[k][:75]
    held = list(range(75, nf, 3))
    P0 = synth.model_params(S, 7)
    before = student.force_errors(S, student.shift_energy_bias(S, P0, train, range(0, 75, 10)), frames, held)
    P, hist = student.train(S, train, 300, lr=1e-3, lr_stop=1e-5, batch=4)
    after = student.force_errors(S, P, frames, held)
    mixed = student.force_errors(S, P, frames, held, precision=dp.DP_PREC_MIXED)
    print("before", before)
    print("after", after)
    print("mixed", mixed)
    assert np.isfinite(hist[-1]["loss"])
    assert after["force_rmse"] < 0.7 * before["force_rmse"]
    assert abs(mixed["force_rmse"] - after["force_rmse"]) < 1e-3


def test_fast_path_with_full_model_fallback(synth):
    """The trained student runs MD as the fast path; the FP64 full model
    checks it every 5 steps.  With a loose tolerance the run stays on the
    student; with a tight one it switches at the first check and continues
    exactly as a full-model run started from that configuration."""
    import os
    from paper_2004_11658_gb300 import dp, student
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    path = os.path.join(os.path.dirname(student.__file__), "data", "student_water12288.npy")
    Ps = np.load(path).astype(np.float64)
    w = synth.workload("water192")
    N = len(w["coords"])
    full = dp.Model(w["model"], synth.model_params(w["model"], 0))
    stud = dp.Model(synth.WATER_STUDENT, Ps)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, 300.0, seed=2)
    t = torch.tensor(w["types"], device="cuda")
    kw = dict(rebuild_every=10, skin=0.2)

    x = torch.tensor(w["coords"], device="cuda")
    v = torch.tensor(v0, device="cuda")
    loose = student.FastPathMD(full, stud, N, tol=1.0, check_every=5)
    checks, sw = loose.run(x, v, t, w["box"], w["masses"], 0.5, 20, **kw)
    print("loose:", checks)
    assert sw is None and len(checks) == 4
    assert all(c["model"] == "student" and c["force_rmse"] < 1.0 for c in checks)
    # the checks read the student's MD force and leave its run untouched: the same
    # trajectory as a plain student run, and that force is the student's force of
    # the final coordinates
    xp = torch.tensor(w["coords"], device="cuda")
    vp = torch.tensor(v0, device="cuda")
    plain = dp.Context(stud, N, precision=dp.DP_PREC_MIXED)
    dp.dp_md_step(plain, xp, vp, t, w["box"], w["masses"], 0.5, 20, **kw)
    assert torch.equal(x, xp) and torch.equal(v, vp)
    fresh = dp.Context(stud, N, precision=dp.DP_PREC_MIXED)
    dp.dp_build_nlist(fresh, x, t, w["box"], 0.0)
    f_eval = dp.dp_eval(fresh, x, t, w["box"])["force"]
    f_md = dp.dp_md_get_force(loose.fast, N)
    assert torch.allclose(f_md, f_eval, rtol=0, atol=1e-12 * float(f_eval.abs().max()))

    x = torch.tensor(w["coords"], device="cuda")
    v = torch.tensor(v0, device="cuda")
    tight = student.FastPathMD(full, stud, N, tol=0.0, check_every=5)
    # first 5 steps on the student, then the switch
    checks, sw = tight.run(x, v, t, w["box"], w["masses"], 0.5, 5, **kw)
    assert sw == 5 and checks[-1]["model"] == "full"
    xs, vs = x.clone(), v.clone()
    tight.run(x, v, t, w["box"], w["masses"], 0.5, 10, **kw)
    ref = dp.Context(full, N)
    dp.dp_md_step(ref, xs, vs, t, w["box"], w["masses"], 0.5, 10, **kw)
    assert torch.equal(x, xs) and torch.equal(v, vs)

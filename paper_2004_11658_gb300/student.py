"""Student model: a narrower embedding net (1-16-32-64) trained on energies
and forces that the full model produces on its own MD trajectories.

The teacher runs velocity-Verlet MD (mixed precision: its trajectory only has
to be plausible) and labels the visited frames with FP64 energies and forces.
The student -- same cutoffs and sel, embedding widths (16, 32, 64), its own
fitting net -- is trained with Adam on
    L = pe * ((E - E_ref) / N)^2 + pf * |F - F_ref|^2 / (3 N)
through DPEnergyForces, whose backward runs the library's hand-written
parameter-gradient kernels (dp_param_grad).  Once trained, the student is the
fast path (its mixed-precision throughput is the highest of all modes) and
the FP64 full model stays the reference for its force error.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import dp, synth


def generate_frames(teacher_desc, teacher_params, workload, n_traj=20, frames_per_traj=50, stride=2,
                    T0=300.0, dt=0.5, seed0=100, device="cuda"):
    """Frames from n_traj teacher trajectories (different Maxwell seeds), one
    frame every `stride` MD steps (20 x 50 frames at stride 2: twenty 100-step
    NVE runs of the starting configuration), labelled by the FP64 teacher.
    Returns dict(coords [F,N,3], energy [F], force [F,N,3]) on the device."""
    w = workload
    N = len(w["coords"])
    m = np.array(w["masses"])[w["types"]]
    # the Verlet-list skin: 2 A where the cell allows it (each edge must be at
    # least 2 (rcut + skin)); the device-side displacement check rebuilds early
    b = np.asarray(w["box"], dtype=np.float64)
    Lmin = float(np.min(np.diag(b.reshape(3, 3)) if b.size == 9 else b))
    skin = max(0.0, min(2.0, 0.999 * (0.5 * Lmin - teacher_desc["rcut"])))
    model = dp.Model(teacher_desc, teacher_params)
    md_ctx = dp.Context(model, N, precision=dp.DP_PREC_MIXED)
    lab_ctx = dp.Context(model, N)
    t = torch.tensor(w["types"], dtype=torch.int32, device=device)
    xs, es, fs = [], [], []
    for tr in range(n_traj):
        x = torch.tensor(w["coords"], dtype=torch.float64, device=device)
        v = torch.tensor(synth.maxwell_velocities(m, T0, seed=seed0 + tr), dtype=torch.float64, device=device)
        dp.dp_md_reset(md_ctx)
        for k in range(frames_per_traj):
            dp.dp_md_step(md_ctx, x, v, t, w["box"], w["masses"], dt, stride, rebuild_every=10, skin=skin)
            dp.dp_build_nlist(lab_ctx, x, t, w["box"], 0.0)
            out = dp.dp_eval(lab_ctx, x, t, w["box"])
            xs.append(x.clone())
            es.append(out["energy"].clone())
            fs.append(out["force"].clone())
    return dict(coords=torch.stack(xs), energy=torch.cat(es), force=torch.stack(fs), types=t, box=w["box"])


def param_offset(desc, name):
    """Offset of a named block in the flat parameter vector."""
    off = 0
    for nm, shape in synth.layer_shapes(desc):
        if nm == name:
            return off
        off += int(np.prod(shape))
    raise KeyError(name)


def shift_energy_bias(desc, params, frames, which):
    """Add to every type's output bias the mean per-atom energy residual of
    the model on the frames `which` (the frames share one composition, so
    only this common shift is determined by the energies)."""
    P = np.array(params, dtype=np.float64, copy=True)
    N = frames["coords"].shape[1]
    model = dp.Model(desc, P)
    ctx = dp.Context(model, N)
    res = []
    for f in which:
        x = frames["coords"][f]
        dp.dp_build_nlist(ctx, x, frames["types"], frames["box"], 0.0)
        out = dp.dp_eval(ctx, x, frames["types"], frames["box"])
        res.append((frames["energy"][f].item() - out["energy"].item()) / N)
    delta = float(np.mean(res))
    for a in range(desc["ntypes"]):
        P[param_offset(desc, f"fit{a}.bo")] += delta
    return P


def _output_slices(desc):
    """Flat-vector slices of every type's output weights wo and bias bo."""
    out = []
    for a in range(desc["ntypes"]):
        o = param_offset(desc, f"fit{a}.wo")
        out.append(slice(o, o + desc["fit"][-1] + 1))   # wo then bo
    return out


def batch_loss(params, ctx, frames, E_lab, F_lab, idx, pe, pf, backward=False):
    """Mean over the frames idx of
        pe ((E - E_lab) / N)^2 + pf |F - F_lab|^2 / (3 N)
    with (E, F) from DPEnergyForces (parameters `params`, any float tensor;
    ctx an FP64 context of the model).  backward=True accumulates the
    gradient into params.grad frame by frame (the kernels' parameter
    gradient); returns the loss as a float."""
    N = frames["coords"].shape[1]
    t, box = frames["types"], frames["box"]
    tot = 0.0
    for f in idx:
        x = frames["coords"][f]
        dp.dp_build_nlist(ctx, x, t, box, 0.0)
        E, F, V = dp.DPEnergyForces.apply(params.double(), x, t, box, ctx)
        L = pe * ((E[0] - E_lab[f]) / N) ** 2 + pf * ((F - F_lab[f]) ** 2).sum() / (3 * N)
        if backward:
            (L / len(idx)).backward()
        tot += float(L.detach())
    return tot / len(idx)


def train(student_desc, frames, steps, lr=1e-3, lr_stop=1e-5, batch=4, pe=1.0, pf=100.0, seed=7,
          init_params=None, label_scale=None, time_limit_s=None, log_every=20):
    """Adam (FP32 parameters and state) on the energy + force loss; the
    gradient of every frame comes from the hand-written kernels.  The
    learning rate decays exponentially from lr to lr_stop over `steps` (or
    over time_limit_s of wall time, whichever ends first).  A fresh student
    (init_params None) starts from seeded weights with its output bias
    shifted to the mean energy of the frames.

    Energies and forces are trained in units of `label_scale` (default: the
    RMS force of the frames), i.e. on E / s and F / s with the output layer
    (wo, bo) divided by s.  The model is linear in (wo, bo), so this is the
    same model; it keeps Adam's per-parameter step (~lr) small against the
    output weights when the labels' forces are far from O(1) eV/A.
    Returns (params float64 numpy in the labels' units, history)."""
    N = frames["coords"].shape[1]
    nf = frames["coords"].shape[0]
    if init_params is None:
        P0 = synth.model_params(student_desc, seed)
        P0 = shift_energy_bias(student_desc, P0, frames, range(0, nf, max(1, nf // 8)))
    else:
        P0 = np.array(init_params, dtype=np.float64, copy=True)
    if label_scale is None:
        label_scale = float(frames["force"].pow(2).mean().sqrt())
    sc = float(label_scale)
    outs = _output_slices(student_desc)
    for sl in outs:
        P0[sl] /= sc
    E_lab = frames["energy"] / sc
    F_lab = frames["force"] / sc
    params = torch.tensor(P0, dtype=torch.float32, requires_grad=True)
    opt = torch.optim.Adam([params], lr=lr)
    model = dp.Model(student_desc, P0)
    ctx = dp.Context(model, N)
    t = frames["types"]
    box = frames["box"]
    rng = np.random.default_rng(seed)
    hist = []
    t0 = time.time()
    for step in range(steps):
        frac = step / max(1, steps)
        if time_limit_s is not None:
            frac = max(frac, (time.time() - t0) / time_limit_s)
        if frac >= 1.0:
            break
        for g in opt.param_groups:
            g["lr"] = lr * (lr_stop / lr) ** frac
        idx = rng.choice(nf, size=batch, replace=False)
        opt.zero_grad()
        tot = batch_loss(params, ctx, frames, E_lab, F_lab, idx, pe, pf, backward=True)
        opt.step()
        if step % log_every == 0:
            hist.append(dict(step=step, loss=tot, lr=opt.param_groups[0]["lr"], seconds=time.time() - t0))
    hist.append(dict(step=step, loss=tot, lr=opt.param_groups[0]["lr"], seconds=time.time() - t0))
    P = params.detach().double().numpy().copy()
    for sl in outs:
        P[sl] *= sc
    return P, hist


def force_errors(desc, params, frames, which, precision=dp.DP_PREC_FP64):
    """Force and energy errors of a model against the frames' FP64 teacher
    labels over the frame indices `which`: RMSE per component, the per-atom
    error |F - F_ref| at the 50th / 90th / 99th percentile, and the RMS
    per-atom energy error."""
    N = frames["coords"].shape[1]
    model = dp.Model(desc, params)
    ctx = dp.Context(model, N, precision=precision)
    se, sf, cnt = 0.0, 0.0, 0
    per_atom = []
    for f in which:
        x = frames["coords"][f]
        dp.dp_build_nlist(ctx, x, frames["types"], frames["box"], 0.0)
        out = dp.dp_eval(ctx, x, frames["types"], frames["box"])
        d = out["force"] - frames["force"][f]
        sf += float((d ** 2).mean())
        per_atom.append(d.norm(dim=1).cpu().numpy())
        se += (float(out["energy"].item() - frames["energy"][f].item()) / N) ** 2
        cnt += 1
    pa = np.concatenate(per_atom)
    p50, p90, p99 = np.percentile(pa, [50, 90, 99])
    return dict(force_rmse=float(np.sqrt(sf / cnt)), energy_rmse_per_atom=float(np.sqrt(se / cnt)),
                force_rms_ref=float(frames["force"][list(which)].pow(2).mean().sqrt()),
                atom_err_p50=float(p50), atom_err_p90=float(p90), atom_err_p99=float(p99))


class FastPathMD:
    """Velocity-Verlet MD on the student (the fast path, mixed precision by
    default) with the FP64 full model as its reference and fallback: every
    `check_every` steps the full model evaluates the current configuration;
    when the student's force RMSE against it exceeds `tol` (eV/A) the run
    continues on the full model from that configuration and velocity.

    run() advances coords/vel in place and returns the list of checks
    (step, force RMSE, max per-atom force error, on which model the run goes
    on) and the step at which it switched (None if it never did)."""

    def __init__(self, full_model, student_model, natoms_max, tol=1e-3, check_every=10,
                 precision=dp.DP_PREC_MIXED):
        self.fast = dp.Context(student_model, natoms_max, precision=precision)
        # one FP64 context serves the checks and, after a switch, the MD run (no check follows a
        # switch; dp_md_reset at the switch clears what the checks left in it)
        self.full = dp.Context(full_model, natoms_max)
        self.refc = self.full
        self.tol = float(tol)
        self.check_every = int(check_every)
        self.on_full = False
        self.switched_at = None
        self.done = 0          # MD steps advanced so far (over all calls)
        self.checks = []       # every check so far

    def _check(self, x, t, box):
        dp.dp_build_nlist(self.refc, x, t, box, 0.0)
        ref = dp.dp_eval(self.refc, x, t, box)["force"].clone()
        # the student's force of these coordinates, kept by its last MD step
        f = dp.dp_md_get_force(self.fast, x.shape[0], device=x.device)
        d = (f - ref).double()
        return float(d.pow(2).mean().sqrt()), float(d.norm(dim=1).max()), float(ref.pow(2).mean().sqrt())

    @property
    def context(self):
        """The context the run is currently on."""
        return self.full if self.on_full else self.fast

    def run(self, x, v, t, box, masses, dt, nsteps, rebuild_every=10, skin=2.0):
        """Advance nsteps.  The step count and the check schedule (every
        check_every steps counted from the first call) continue across
        calls, so the run may be advanced one step at a time."""
        new = []
        left = int(nsteps)
        while left > 0:
            n = min(left, self.check_every - self.done % self.check_every)
            dp.dp_md_step(self.context, x, v, t, box, masses, dt, n, rebuild_every=rebuild_every, skin=skin)
            self.done += n
            left -= n
            if not self.on_full and self.done % self.check_every == 0:
                rmse, worst, frms = self._check(x, t, box)
                if rmse > self.tol:
                    self.on_full = True
                    self.switched_at = self.done
                    dp.dp_md_reset(self.full)  # forces of the current configuration on the next step
                new.append(dict(step=self.done, force_rmse=rmse, max_atom_err=worst, force_rms_full=frms,
                                model="full" if self.on_full else "student"))
        self.checks.extend(new)
        return new, self.switched_at


def main(argv=None):
    """Trains the water student on teacher trajectories of the 12,288-atom
    box and writes its parameters (float32 .npy) and a JSON summary."""
    import argparse
    import json
    import os
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--out", required=True, help="parameter file (.npy); the summary goes to <out>.json")
    ap.add_argument("--minutes", type=float, default=40.0, help="training wall time")
    ap.add_argument("--trajectories", type=int, default=20)
    ap.add_argument("--frames", type=int, default=50, help="frames per trajectory")
    ap.add_argument("--stride", type=int, default=2, help="MD steps between frames")
    ap.add_argument("--seed", type=int, default=7)
    a = ap.parse_args(argv)
    w = synth.workload("water12288")
    teacher = w["model"]
    t0 = time.time()
    fr = generate_frames(teacher, synth.model_params(teacher, 0), w, n_traj=a.trajectories,
                         frames_per_traj=a.frames, stride=a.stride)
    t_gen = time.time() - t0
    nf = fr["coords"].shape[0]
    ntrain = nf - a.frames  # the last trajectory is held out
    train_fr = dict(fr)
    for k in ("coords", "energy", "force"):
        train_fr[k] = fr[k][:ntrain]
    held = list(range(ntrain, nf))
    S = WATER_STUDENT_DESC
    P, hist = train(S, train_fr, 10 ** 9, seed=a.seed, time_limit_s=60.0 * a.minutes, log_every=50)
    res = dict(desc={k: list(v) if isinstance(v, tuple) else v for k, v in S.items()},
               frames=nf, train_frames=ntrain, held_out_frames=len(held), stride=a.stride, generate_s=t_gen,
               steps=hist[-1]["step"] + 1, history=hist,
               held_out_fp64=force_errors(S, P, fr, held),
               held_out_mixed=force_errors(S, P, fr, held, precision=dp.DP_PREC_MIXED))
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.save(a.out, P.astype(np.float32))
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({k: v for k, v in res.items() if k != "history"}, indent=1))


WATER_STUDENT_DESC = synth.WATER_STUDENT

if __name__ == "__main__":
    main()

"""Velocity-Verlet MD over slabs (Sec. 3.1, Remark 4, Sec. 4) on the CPU:
kick/drift of the owned atoms, re-planning with atom migration, forward and
reverse halos and the all-reduce, with the oracle's sub-region evaluation,
against the oracle's single-domain velocity Verlet on the whole system;
slabs emulated in one process and one slab per gloo rank."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2004_11658_gb300 import domain  # noqa: E402

ACC = 9.648533212e-3


class TorchIntegrator:
    """The oracle's velocity-Verlet arithmetic (test side only)."""

    def kick_drift(self, x, v, f, t, masses, dt):
        c = (0.5 * dt * ACC / torch.as_tensor(masses, dtype=torch.float64))[t.long()]
        v += c[:, None] * f
        x += dt * v

    def kick(self, v, f, t, masses, dt):
        c = (0.5 * dt * ACC / torch.as_tensor(masses, dtype=torch.float64))[t.long()]
        v += c[:, None] * f


def _oracle_eval(oracle, desc, P, cap):
    def ev(xs, ts, box, nloc):
        r = oracle.evaluate_local(desc, P, xs.numpy(), ts.numpy(), box, nloc, cap=cap)
        return r["energy"], torch.tensor(r["force"]), torch.tensor(r["virial"])
    return ev


def _system(synth):
    w = synth.sub_box_water(6, 6 * 49.7 / 16)        # 648 atoms, 18.64 A
    m = np.array(w["masses"])[w["types"]]
    v = synth.maxwell_velocities(m, 300.0, seed=4)
    v[:, 0] += 0.08        # a uniform drift along x (A/fs): many atoms cross slab faces
    w["vel"] = v
    return w


NSTEPS, DT, SKIN = 16, 1.0, 1.0


def _reference(oracle, synth, w, P):
    return oracle.md(w["model"], P, w["coords"], w["vel"], w["types"], w["box"], w["masses"], DT, NSTEPS,
                     rebuild_every=1, skin=0.0)


def _gather(md, N):
    x = np.zeros((N, 3))
    v = np.zeros((N, 3))
    for gid, xs, vs, fs in md.owned():
        x[gid.numpy()] = xs.numpy()
        v[gid.numpy()] = vs.numpy()
    return x, v


def _check(x, v, th, ref, box):
    xo, vo, fo, tho, _ = ref
    d = x - xo
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(v - vo).max() < 1e-10
    np.testing.assert_allclose(th[:, 0], tho[:, 0], rtol=1e-11)
    np.testing.assert_allclose(th[:, 1], tho[:, 1], rtol=1e-11)


@pytest.mark.parametrize("nslab,replan", [(1, 4), (2, 4), (3, 5), (4, 100)])
def test_emulated_slab_md_matches_single_domain(oracle, synth, nslab, replan):
    w = _system(synth)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    N = len(w["coords"])
    cap = 512
    comm = domain.LocalComm(nslab)
    md = domain.SlabMD(comm, w["box"], desc["rcut"], SKIN, torch.tensor(w["coords"]), torch.tensor(w["vel"]),
                       torch.tensor(w["types"]), w["masses"], DT,
                       [_oracle_eval(oracle, desc, P, cap) for _ in range(nslab)],
                       [TorchIntegrator() for _ in range(nslab)], replan_every=replan)
    owner0 = {int(g): k for k, s in enumerate(md.s) for g in s["gid"]}
    th = np.array(md.run(NSTEPS))
    x, v = _gather(md, N)
    assert sum(len(s["gid"]) for s in md.s) == N
    _check(x, v, th, _reference(oracle, synth, w, P), w["box"])
    if 1 < nslab and replan < NSTEPS:
        # atoms crossed slab faces and were handed over to their new owners
        owner1 = {int(g): k for k, s in enumerate(md.s) for g in s["gid"]}
        assert sum(owner0[g] != owner1[g] for g in owner0) > 20


def _rank_main(rank, world, port, desc, P, w, cap, out_dir):
    import torch.distributed as dist
    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = domain.DistComm(rank, world)
        md = domain.SlabMD(comm, w["box"], desc["rcut"], SKIN, torch.tensor(w["coords"]), torch.tensor(w["vel"]),
                           torch.tensor(w["types"]), w["masses"], DT, [_oracle_eval(oracle, desc, P, cap)],
                           [TorchIntegrator()], replan_every=4)
        th = np.array(md.run(NSTEPS))
        (gid, x, v, f), = md.owned()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), th=th, gid=gid.numpy(), x=x.numpy(), v=v.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_slab_md(oracle, synth, tmp_path, world):
    import torch.multiprocessing as mp
    w = _system(synth)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    N = len(w["coords"])
    port = 29700 + (os.getpid() % 1500) + 10 * world
    mp.start_processes(_rank_main, args=(world, port, desc, P, w, 512, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    x = np.zeros((N, 3))
    v = np.zeros((N, 3))
    seen = np.zeros(N, dtype=int)
    ths = []
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        x[d["gid"]] = d["x"]
        v[d["gid"]] = d["v"]
        seen[d["gid"]] += 1
        ths.append(d["th"])
    assert np.all(seen == 1)                       # every atom owned by exactly one rank
    for th in ths[1:]:
        np.testing.assert_array_equal(th, ths[0])  # every rank saw the same all-reduced thermo
    _check(x, v, ths[0], _reference(oracle, synth, w, P), w["box"])


def test_send_lists_match_global_plan(synth):
    """The send lists a slab computes from its own atoms equal those of the
    global plan (make_plan) for the same positions."""
    w = synth.sub_box_water(6, 6 * 49.7 / 16)
    x, box = w["coords"], w["box"]
    for nslab in (2, 3):
        plan = domain.make_plan(x, box, nslab, ghost_width=7.0, pad=7.0)
        for p in range(nslab):
            own = plan.owned[p]
            mine = domain._send_lists(np.asarray(box), nslab, 7.0, p, own, x[own])
            for q in range(nslab):
                np.testing.assert_array_equal(mine[q][0], plan.send[p][q][0])
                np.testing.assert_array_equal(mine[q][1], plan.send[p][q][1])

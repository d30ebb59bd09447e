"""Spatial domain decomposition (Sec. 3.1, Remark 4) on the CPU: slabs with
ghost shells, forward and reverse halos and the energy/virial all-reduce,
with the oracle's sub-region evaluation, against the oracle on the whole
periodic system; one slab per gloo rank for two and three ranks."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2004_11658_gb300 import domain  # noqa: E402


def _oracle_eval(oracle, desc, P, cap):
    def ev(xs, ts, box, nloc):
        r = oracle.evaluate_local(desc, P, xs.numpy(), ts.numpy(), box, nloc, cap=cap)
        return r["energy"], torch.tensor(r["force"]), torch.tensor(r["virial"])
    return ev


def _case(synth, name):
    if name == "water648":
        return synth.sub_box_water(6, 6 * 49.7 / 16)
    return synth.workload(name)


@pytest.mark.parametrize("name,nslab", [("water192", 1), ("water192", 2), ("water648", 2), ("water648", 3)])
def test_emulated_slabs_match_whole_system(oracle, synth, name, nslab):
    w = _case(synth, name)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    N = len(w["coords"])
    ref = oracle.evaluate(desc, P, w["coords"], w["types"], w["box"])
    cap = oracle.default_cap(desc, w["box"], N, 0.0)
    plan = domain.make_plan(w["coords"], w["box"], nslab, ghost_width=desc["rcut"], pad=desc["rcut"] + 1.0)
    assert sum(len(o) for o in plan.owned) == N
    E, F, V = domain.evaluate_emulated(plan, torch.tensor(w["coords"]), torch.tensor(w["types"]),
                                       _oracle_eval(oracle, desc, P, cap))
    scale = np.abs(ref["force"]).max()
    assert E == pytest.approx(ref["energy"], rel=1e-12, abs=1e-12)
    assert np.abs(F.numpy() - ref["force"]).max() < 1e-12 * scale
    assert np.abs(V.numpy() - ref["virial"]).max() < 1e-11 * np.abs(ref["virial"]).max()


def test_plan_halo_lists(synth):
    """Every atom within the ghost width of a slab face appears as a ghost of
    that slab exactly once per periodic image, and owners send exactly what
    the slab receives."""
    w = _case(synth, "water648")
    L = w["box"][0]
    plan = domain.make_plan(w["coords"], w["box"], 3, ghost_width=6.0, pad=7.0)
    width = L / 3
    xw = np.mod(w["coords"][:, 0], L)
    for q in range(3):
        lo, hi = q * width - 6.0, (q + 1) * width + 6.0
        expect = 0
        for s in (-1, 0, 1):
            xs = xw + s * L
            inside = (xs >= lo) & (xs < hi)
            if s == 0:
                inside &= ~np.isin(np.arange(len(xw)), plan.owned[q])
            expect += int(inside.sum())
        assert len(plan.ghost_src[q]) == expect
        for p in range(3):
            pos, shift = plan.send[p][q]
            gx = xw[plan.owned[p][pos]] + shift * L
            assert np.all((gx >= lo) & (gx < hi))


def _rank_main(rank, world, port, desc, P, coords, types, box, cap, out_dir):
    import torch.distributed as dist
    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = domain.make_plan(coords, box, world, ghost_width=desc["rcut"], pad=desc["rcut"] + 1.0)
        own = plan.owned[rank]
        t = torch.tensor(types)[torch.as_tensor(own)]
        slab = domain.DistributedSlab(plan, rank, t, _oracle_eval(oracle, desc, P, cap))
        E, F, V = slab.forces(torch.tensor(coords)[torch.as_tensor(own)])
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), E=E, F=F.numpy(), V=V.numpy(), own=own)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_slabs(oracle, synth, tmp_path, world):
    """One slab per gloo rank; with three ranks on the 18.6 A box every rank
    exchanges halos with both others."""
    import torch.multiprocessing as mp
    w = _case(synth, "water648")
    desc = w["model"]
    P = synth.model_params(desc, 0)
    N = len(w["coords"])
    ref = oracle.evaluate(desc, P, w["coords"], w["types"], w["box"])
    cap = oracle.default_cap(desc, w["box"], N, 0.0)
    port = 29500 + (os.getpid() % 2000) + 10 * world
    mp.start_processes(_rank_main, args=(world, port, desc, P, w["coords"], w["types"], w["box"], cap,
                                         str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    F = np.zeros((N, 3))
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        assert float(d["E"]) == pytest.approx(ref["energy"], rel=1e-12)
        assert np.abs(d["V"] - ref["virial"]).max() < 1e-11 * np.abs(ref["virial"]).max()
        F[d["own"]] = d["F"]
    assert np.abs(F - ref["force"]).max() < 1e-12 * np.abs(ref["force"]).max()

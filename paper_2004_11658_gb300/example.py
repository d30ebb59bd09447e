"""A minimal use of the library from Python: build the neighbour list,
evaluate energy, forces and virial, and run 100 velocity-Verlet steps of the
12,288-atom water box (device tensors in, device tensors out; the synthetic
water box and seeded weights stand in for a trained model).

    python -m paper_2004_11658_gb300.example
"""
import numpy as np
import torch

from paper_2004_11658_gb300 import dp, synth


def main():
    w = synth.workload("water12288")                   # 4,096 H2O in a 49.7 A box
    model = dp.Model(w["model"], synth.model_params(w["model"], seed=0))
    ctx = dp.Context(model, natoms_max=len(w["types"]), precision=dp.DP_PREC_FP64)

    x = torch.tensor(w["coords"], device="cuda")       # N x 3 float64, A
    t = torch.tensor(w["types"], device="cuda")        # N int32
    dp.dp_build_nlist(ctx, x, t, w["box"], skin=2.0)
    out = dp.dp_eval(ctx, x, t, w["box"])              # energy [1] eV, force [N, 3] eV/A, virial [9] eV

    m = np.array(w["masses"])[w["types"]]
    v = torch.tensor(synth.maxwell_velocities(m, 300.0), device="cuda")
    thermo = torch.empty((100, 4), dtype=torch.float64, device="cuda")   # E_pot, E_kin, T, P per step
    dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], 0.5, 100, rebuild_every=10, skin=2.0, thermo=thermo)
    return out, thermo, ctx


if __name__ == "__main__":
    out, thermo, ctx = main()
    torch.cuda.synchronize()
    print(f"E = {out['energy'].item():.6f} eV, T after 100 steps = {thermo[-1, 2].item():.1f} K")

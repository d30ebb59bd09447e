#!/usr/bin/env python
"""Benchmark: Deep Potential MD throughput (atom-steps/s) on GB300.

Workload (default): 131,072 H2O = 393,216 atoms in a 157.6 A periodic box, the
water model (se_a, rcut 6 A, rcut_smth 0.5 A, sel 46/92, embedding 25-50-100,
M2 = 16, fitting 240-240-240, seeded FP64 weights), velocity Verlet at
dt = 0.5 fs from 300 K, candidates with a 2 A skin rebuilt every 10 steps.
One benchmark step = one MD step of the whole box (every tenth step includes
the candidate rebuild, so any 10 consecutive steps run every row of the path:
candidate build, Algorithm 1, environment matrix, embedding, descriptor,
fitting, backward, ProdForce/ProdVirial, energy sum, integrator).  The
12,288-atom box (--workload water12288) and copper run 10 MD steps per
benchmark step.

Modes beside the FP64 path: mixed precision (full model; plain BF16 and
split-operand embedding GEMMs) and the student model as the fast path with
the FP64 full model as its periodic judge and fallback; each reports its force error against the FP64 full model at the
start and at the end of a 100-step trajectory (200 for copper).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.  Multi-GPU (--gpus N under
torchrun): N independent replicas, one per GPU (the path has no exchange step
on one box); value sums all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "atom-steps/s"
SKIN = 2.0
REBUILD_EVERY = 10
L2_BYTES = 129 * 1024 * 1024
DEFAULT_WORKLOAD = "water393216"

# Per workload: MD steps per benchmark step, dt (fs), T0 (K), length of the
# trajectory on which each mode's accuracy is reported (MD steps), and the
# centres of the oracle's bounded sample per MD step (all cores, one core).
WORKLOADS = {
    "water393216": dict(md_per_step=1, dt=0.5, T0=300.0, traj=100, sample=8192, sample_1core=1024),
    "water12288": dict(md_per_step=10, dt=0.5, T0=300.0, traj=100, sample=12288, sample_1core=1024),
    "cu32000": dict(md_per_step=10, dt=1.0, T0=330.0, traj=200, sample=4096, sample_1core=512),
    "water192": dict(md_per_step=1, dt=0.5, T0=300.0, traj=20, sample=192, sample_1core=192),
}

# FP64 pipe peak of a GB300: 152 SMs x 2 FP64 FMA/clk/SM x 2 FLOP x 2.07 GHz.
# The per-SM rate is the one that reproduces the nominal 1.25 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 pipe peak: 152 SMs x 128 FMA/clk/SM x 2 FLOP x 2.07 GHz (nominal).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP32 instructions per multiply-add of the mixed kernels' double-float
# contractions (mixed.cu df_fma: 2 multiplies/FMAs for the exact product, 6
# adds for the two-sum, 2 for the error terms)
DF_FP32_INST_PER_FMA = 10
FORCE_RMSE_TARGET = 1e-3   # eV/A, against the FP64 full model

# Per-kernel counters from one ncu capture of one evaluation of the 12,288-atom
# water box (bench.py --workload water12288 --profile-eval 1, 1,046,154 real
# neighbour rows), reported only while the kernel source is the one captured
# (hash of the .cu file and the shared header):
#   bytes_per_row     (dram__bytes_read.sum + dram__bytes_write.sum) / rows: the
#                     traffic of a launch grows with its rows (G and dG/ds rows,
#                     per-atom T, D and dE/dD at ~91 rows per atom), so the bench
#                     reports bytes_per_row x the rows of its own launch
#   fp64_flop_per_row 2 x dfma + dadd + dmul thread instructions
#                     (smsp__sass_thread_inst_executed_op_d{fma,add,mul}_pred_on.sum)
#                     per real neighbour row
#   pipe_busy         sm__inst_executed_pipe_fp64 share of the active cycles
PROFILE_ROWS = 1046154
TRAFFIC = {
    "embed_tan<25>": {"bytes_per_row": (10.468352e6 + 1811.331840e6) / PROFILE_ROWS, "file": "embed_x.cu",
                      "src_sha": "c2c89c84fd00c488"},
    "embed_bwd_st<25>": {"bytes_per_row": (1883.360000e6 + 28.511232e6) / PROFILE_ROWS, "file": "embed_x.cu",
                         "src_sha": "c2c89c84fd00c488"},
    "embed_tan_mx<25>": {"bytes_per_row": (49.605120e6 + 1008.945408e6) / PROFILE_ROWS, "file": "mixed.cu",
                         "src_sha": "bd0c7271cc3b2bf4"},
    "embed_bwd_st_mx<25>": {"bytes_per_row": (1043.964160e6 + 26.513920e6) / PROFILE_ROWS, "file": "mixed.cu",
                            "src_sha": "bd0c7271cc3b2bf4"},
    "embed_bwd_mx<25, split>": {"bytes_per_row": (204.796928e6 + 17.978880e6) / PROFILE_ROWS, "file": "mixed.cu",
                                "src_sha": "bd0c7271cc3b2bf4"},
    "embed_tan_mx<16>": {"bytes_per_row": (7.999488e6 + 603.240704e6) / PROFILE_ROWS, "file": "mixed.cu",
                         "src_sha": "bd0c7271cc3b2bf4"},
    "embed_bwd_st_mx<16>": {"bytes_per_row": (669.597440e6 + 25.187072e6) / PROFILE_ROWS, "file": "mixed.cu",
                            "src_sha": "bd0c7271cc3b2bf4"},
}
# Pipe shares of the mixed embedding kernels (ncu, one evaluation of the
# 12,288-atom water box, --profile-precision mixed / split): active-cycle
# busy fractions of the FP64, FP32 (fma), integer (alu) and tensor pipes and
# the schedulers' issue-active share.
MODE_PIPES = {
    "embed_tan_mx<25>": {"fp64": 0.386, "fma": 0.196, "alu": 0.087, "tensor": 0.016, "issue_active": 0.333,
                         "file": "mixed.cu", "src_sha": "bd0c7271cc3b2bf4"},
    "embed_bwd_st_mx<25>": {"fp64": 0.689, "fma": 0.282, "alu": 0.041, "tensor": 0.0, "issue_active": 0.406,
                            "file": "mixed.cu", "src_sha": "bd0c7271cc3b2bf4"},
    "embed_bwd_mx<25, split>": {"fp64": 0.448, "fma": 0.180, "alu": 0.094, "tensor": 0.028, "issue_active": 0.302,
                                "file": "mixed.cu", "src_sha": "bd0c7271cc3b2bf4"},
    "embed_tan_mx<16>": {"fp64": 0.442, "fma": 0.168, "alu": 0.081, "tensor": 0.006, "issue_active": 0.300,
                         "file": "mixed.cu", "src_sha": "bd0c7271cc3b2bf4"},
    "embed_bwd_st_mx<16>": {"fp64": 0.754, "fma": 0.239, "alu": 0.048, "tensor": 0.0, "issue_active": 0.366,
                            "file": "mixed.cu", "src_sha": "bd0c7271cc3b2bf4"},
}
FP64_ISSUED = {
    # k_embed_tan_x<25>: dfma 2.257e9, dadd 0.818e9, dmul 0.106e9 thread
    # instructions; FP64 pipe busy 41.2% (issue active 24.3%)
    "embed_tan<25>": {"fp64_flop_per_row": (2 * 2.257052574e9 + 0.817909986e9 + 0.105703644e9) / PROFILE_ROWS,
                      "pipe_busy": 0.412, "file": "embed_x.cu", "src_sha": "c2c89c84fd00c488"},
    # k_embed_bwd_st<25>: dfma 1.070e9, dadd 0.101e9, dmul 0.044e9; FP64 pipe busy 93.9%
    "embed_bwd_st<25>": {"fp64_flop_per_row": (2 * 1.069532688e9 + 0.100726048e9 + 0.043622898e9) / PROFILE_ROWS,
                         "pipe_busy": 0.939, "file": "embed_x.cu", "src_sha": "c2c89c84fd00c488"},
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision measurement")
    p.add_argument("--no-student", action="store_true", help="skip the student-model measurement")
    p.add_argument("--decomp", choices=["replicas", "slab"], default="replicas",
                   help="replicas: one independent system per GPU; slab: one system cut into one slab per "
                        "GPU (forward/reverse halos over NCCL point-to-point, all-reduce of E and the virial)")
    p.add_argument("--profile-eval", type=int, default=0, metavar="N",
                   help="run N energy/force evaluations of the workload and exit (profiling driver)")
    p.add_argument("--profile-precision", choices=["fp64", "mixed", "split"], default="fp64")
    p.add_argument("--profile-model", choices=["full", "student"], default="full")
    return p.parse_args()


def emb_row_flops(desc):
    """Algorithmic FLOPs per real neighbour row (one embedding net pass)."""
    e = list(desc["emb"])
    g = 2 * e[0]
    for a, b in zip(e[:-1], e[1:]):
        g += 2 * a * b
    return g


def fit_atom_flops(desc):
    M = desc["emb"][-1]
    prev = desc["m2"] * M
    f = 0
    for w in desc["fit"]:
        f += 2 * prev * w
        prev = w
    return f + 2 * prev


def kernel_flops(desc, rows, natoms, store=False):
    """FLOPs per launch of each kernel group, counted from the algorithm
    (multiply-add = 2, tanh not counted):
      embed_fwd: embedding GEMMs per real row + T = R~^T G (8 M per row)
                 + D = T_<^T T (8 M2 M per atom)
      embed_bwd: embedding recomputed + its s-tangent (2x GEMMs) + the two
                 4 x M contractions with gT (16 M per row) + gT (16 M2 M per atom)
      fit:       fitting forward + backward to the descriptor (2x forward).
    store: G and dG/ds kept between the two (k_embed_tan_x, k_embed_bwd_st):
      the forward evaluates the GEMMs with the s-tangent (2x GEMMs) + T + D,
      the backward only the contractions and gT."""
    M, m2 = desc["emb"][-1], desc["m2"]
    g = emb_row_flops(desc)
    if store:
        return {
            "embed_fwd": rows * (2 * g + 8 * M) + natoms * 8 * m2 * M,
            "embed_bwd": rows * 16 * M + natoms * 16 * m2 * M,
            "fit": natoms * 2 * fit_atom_flops(desc),
        }
    return {
        "embed_fwd": rows * (g + 8 * M) + natoms * 8 * m2 * M,
        "embed_bwd": rows * (2 * g + 16 * M) + natoms * 16 * m2 * M,
        "fit": natoms * 2 * fit_atom_flops(desc),
    }


def digit_mma_flops_bwd(desc, nreal):
    """Tensor-core FLOPs the FP64 embedding backward kernel issues per launch
    (k_embed_bwd_x, doubling nets with e1 <= 32): for every chunk of up to 32
    rows of one atom's type block, the last layer's value and tangent
    products, 28 digit pairs x ceil(2 e1 / 16) MMAs of M = 128, N = 32,
    K = 16 each, and layer 1's, 28 x ceil(e1 / 16) MMAs of M = 64 each.
    nreal: [N, ntypes] real rows per type block."""
    e1 = desc["emb"][0]
    k2p, k1p = -(-2 * e1 // 16), -(-e1 // 16)
    chunks = int(np.ceil(np.asarray(nreal, dtype=np.int64) / 32.0).sum())
    per_chunk = 2 * 28 * (k2p * 2 * 128 * 32 * 16 + k1p * 2 * 64 * 32 * 16)
    return chunks * per_chunk


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def source_sha(fn):
    """Hash of a kernel source file together with the shared device header."""
    h = hashlib.sha256()
    for name in (fn, "dp_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2004_11658_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _counter(table, key):
    tr = table.get(key)
    return tr if tr and tr.get("src_sha") == source_sha(tr["file"]) else None


def workload_config(name, w, world):
    """The config block both arms print (same keys, same values)."""
    wl = WORKLOADS[name]
    desc = w["model"]
    return {"workload": name, "atoms": int(len(w["coords"])), "md_steps_per_step": wl["md_per_step"],
            "dt_fs": wl["dt"], "skin": SKIN, "rebuild_every": REBUILD_EVERY, "T0_K": wl["T0"],
            "model": "se_a %s %s / M2 %d / fit %s, seeded FP64 weights" % (
                "copper" if desc["ntypes"] == 1 else "water", "-".join(map(str, desc["emb"])), desc["m2"],
                "x".join(map(str, desc["fit"]))),
            "l2": "inputs larger than L2, and L2 flushed between steps (256 MB write)",
            "parallelism": f"replicas x{world}"}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------------ the oracle --

def oracle_sample_step(O, w, desc, P, S):
    """One MD step's work of the oracle for the first S atoms of the workload
    as centres (the 393,216-atom box lists its molecules in a random order of
    lattice sites, so they are spread over the box): candidates of those
    centres from the cell list (counted 1/10, rebuilt every 10 steps),
    Algorithm 1 and the FP64 evaluation of their energies and pair gradients.
    Returns the seconds per MD step of S atoms."""
    x, t, box = w["coords"], w["types"], w["box"]
    N = len(x)
    S = min(S, N)
    cap = O.default_cap(desc, box, N, SKIN)
    t0 = time.perf_counter()
    ncand, cand, _ = O.candidates(x, box, desc["rcut"] + SKIN, cap, ncentre=S if S < N else None)
    t_cand = time.perf_counter() - t0
    t0 = time.perf_counter()
    nl, _, _ = O.format_nlist(x, t, box, ncand, cand, desc["sel"], desc["rcut"], ncentre=S)
    O.eval_nlist(desc, P, x, t, box, nl, nloc=S)
    return time.perf_counter() - t0 + t_cand / REBUILD_EVERY


def cpu_baseline(w, desc, P, name):
    """The oracle as it stands on this host's cores (all, then one), each on a
    bounded sample of the workload: S centres' MD-step work, best of 2."""
    from oracle import oracle as O
    wl = WORKLOADS[name]
    out = {}
    for key, S, threads in (("all", wl["sample"], None), ("one", wl["sample_1core"], 1)):
        if threads is not None:
            O.set_num_threads(threads)
        cores = O.num_threads()
        per = min(oracle_sample_step(O, w, desc, P, S) for _ in range(2))
        S = min(S, len(w["coords"]))
        out[key] = {"value": S / per, "unit": METRIC, "cores": cores, "kind": "oracle",
                    "sample": f"{S} of the {len(w['coords'])} atoms as centres: candidates (cell list, /"
                              f"{REBUILD_EVERY}), Algorithm 1 and the FP64 evaluation of one MD step, best of 2; "
                              f"{per:.2f} s"}
    O.set_num_threads(os.cpu_count() or 1)
    res = dict(out["all"])
    res["cpu"] = cpu_model()
    res["nproc"] = os.cpu_count()
    res["one_core"] = out["one"]
    return res


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: every benchmark step is a bounded
    sample of one MD step of the workload (the first S atoms as centres on the
    starting configuration), scaled to atom-steps/s."""
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2004_11658_gb300 import synth
    w = synth.workload(args.workload)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    wl = WORKLOADS[args.workload]
    S = min(wl["sample"], len(w["coords"]))
    times = []
    for k in range(args.warmup + args.steps):
        dt = oracle_sample_step(O, w, desc, P, S) * wl["md_per_step"]
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    # atom-steps of the sample per benchmark step
    value = S * wl["md_per_step"] * len(times) / total
    cores = O.num_threads()
    sample = (f"each step: {wl['md_per_step']} MD step(s) of {S} of the {len(w['coords'])} atoms as centres "
              f"(candidates from the cell list counted 1/{REBUILD_EVERY}, Algorithm 1, FP64 evaluation)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.workload, w, world),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours --

def mixed_kernel_flops(desc, rows, natoms, store=False):
    """Per-launch work of the mixed-precision kernels, split by unit:
    tensor-core FLOPs (BF16 GEMMs, unpadded), the per-row contractions with
    R~ and dE/dT (double-float arithmetic on the FP32 pipe) and the per-atom
    FP64 FLOPs (D = T_<^T T forward, dE/dT backward).  store: G and dG/ds
    kept between the two (k_embed_tan_mx evaluates the GEMMs with the
    s-tangent, k_embed_bwd_stmx only the contractions)."""
    M, m2 = desc["emb"][-1], desc["m2"]
    g = emb_row_flops(desc) - 2 * desc["emb"][0]   # layer 0 runs on the CUDA cores
    if store:
        return {
            "embed_fwd": {"tensor": rows * 2 * g, "df": rows * 8 * M, "fp64": natoms * 8 * m2 * M},
            "embed_bwd": {"tensor": 0, "df": rows * 16 * M, "fp64": natoms * 16 * m2 * M},
            "fit": {"tensor": natoms * 2 * fit_atom_flops(desc), "df": 0, "fp64": 0},
        }
    return {
        "embed_fwd": {"tensor": rows * g, "df": rows * 8 * M, "fp64": natoms * 8 * m2 * M},
        "embed_bwd": {"tensor": rows * 2 * g, "df": rows * 16 * M, "fp64": natoms * 16 * m2 * M},
        "fit": {"tensor": natoms * 2 * fit_atom_flops(desc), "df": 0, "fp64": 0},
    }


def _accuracy(dp, ctx, refc, x, t, box):
    """Forces, energy and virial of ctx against the reference context (FP64 full
    model) on the configuration x: RMSE per component, absolute and relative to
    the RMS reference force, per-atom |dF| percentiles, energy error per atom,
    virial error relative to its max."""
    import torch
    N = x.shape[0]
    dp.dp_build_nlist(ctx, x, t, box, SKIN)
    dp.dp_build_nlist(refc, x, t, box, SKIN)
    a = dp.dp_eval(ctx, x, t, box)
    a = {k: v.clone() for k, v in a.items() if torch.is_tensor(v)}
    b = dp.dp_eval(refc, x, t, box)
    dF = (a["force"] - b["force"]).double()
    rmse = float(dF.pow(2).mean().sqrt())
    frms = float(b["force"].pow(2).mean().sqrt())
    pa = dF.norm(dim=1).cpu().numpy()
    p50, p90, p99 = (float(q) for q in np.percentile(pa, [50, 90, 99]))
    fa = b["force"].norm(dim=1).cpu().numpy()
    worst = int(np.argmax(pa))
    return {"force_rmse_eV_per_A": rmse, "force_rms_eV_per_A": frms,
            "rel_force_rmse": rmse / frms if frms > 0 else None,
            "atom_force_err_p50_p90_p99_eV_per_A": [p50, p90, p99],
            "atom_force_err_max_eV_per_A": float(pa[worst]),
            "force_at_worst_atom_eV_per_A": float(fa[worst]), "force_max_eV_per_A": float(fa.max()),
            "atoms_err_above_1e-3": int((pa > 1e-3).sum()),
            "energy_err_eV_per_atom": abs(a["energy"].item() - b["energy"].item()) / N,
            "virial_rel_err": float((a["virial"] - b["virial"]).abs().max() / b["virial"].abs().max()),
            "meets_target": rmse <= FORCE_RMSE_TARGET}


def _mode_roofline(fl, groups, dom, tag, traffic):
    """Roofline of a mode's dominant kernel by unit: BF16 tensor FLOPs, the
    double-float contractions as FP32 instructions issued (an estimate from
    the instruction count per multiply-add) and the per-atom FP64 FLOPs; the
    top-level entry is the busiest of the three."""
    sec = groups[dom]["ms"] / groups[dom]["launches"] / 1000.0
    pk = measured_peaks()
    bf16_peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1720.9))
    ach_t = fl[dom]["tensor"] / sec / 1e12
    ach_c = fl[dom]["df"] / sec / 1e12
    ach_f32 = ach_c / 2 * DF_FP32_INST_PER_FMA * 2   # FP32 FLOP-equivalents (an instruction counts 2)
    ach_d = fl[dom]["fp64"] / sec / 1e12
    units = {
        "tensor_bf16": {"achieved": ach_t, "peak": bf16_peak, "frac": ach_t / bf16_peak,
                        "what": "algorithmic BF16 GEMM FLOPs (unpadded)",
                        "peak_source": "MEASURED_PEAKS bf16_tflops_sustained (of measured)"},
        "fp32_double_float": {"achieved": ach_f32, "peak": FP32_PEAK_TFLOPS, "frac": ach_f32 / FP32_PEAK_TFLOPS,
                              "contraction_tflops": ach_c,
                              "what": "the contractions with R~ and dE/dT (algorithmic contraction_tflops) in "
                                      "double-float arithmetic, as FP32 pipe work: %d FP32 instructions per "
                                      "multiply-add, 2 FLOP each (estimate)" % DF_FP32_INST_PER_FMA,
                              "peak_source": "152 SMs x 128 FMA/clk x 2 x 2.07 GHz (nominal)"},
        "fp64": {"achieved": ach_d, "peak": FP64_PEAK_TFLOPS, "frac": ach_d / FP64_PEAK_TFLOPS,
                 "what": "algorithmic per-atom FP64 FLOPs (D = T_<^T T, dE/dT)"},
    }
    top = max(units, key=lambda u: units[u]["frac"])
    out = {"bound": "tensor" if top == "tensor_bf16" else "alu", "kernel": tag, "unit": "TFLOP/s",
           "achieved": units[top]["achieved"], "peak": units[top]["peak"], "frac": units[top]["frac"],
           "traffic": traffic}
    out.update(units)
    pipes = _counter(MODE_PIPES, tag)
    if pipes:
        out["pipes_ncu"] = {k: v for k, v in pipes.items() if k not in ("file", "src_sha")}
    return out


def measure_mode(args, dp, w, run_desc, run_P, ref_model, v0, dev, world, flush, dtype, fast_path=False,
                 precision=None):
    """MD with another model or precision on the same workload: throughput,
    per-kernel times, roofline of the dominant kernel, and accuracy against
    the FP64 full model at the start and at the end of the mode's trajectory
    (WORKLOADS[...]["traj"] MD steps, continued untimed after the timed steps).
    fast_path: the run goes through student.FastPathMD (the FP64 full model
    checks the force error every 10 MD steps inside the timed region and takes
    over when it exceeds the target)."""
    import torch
    from paper_2004_11658_gb300 import student
    wl = WORKLOADS[args.workload]
    N = len(v0)
    model = dp.Model(run_desc, run_P)
    x = torch.tensor(w["coords"], dtype=torch.float64, device=dev)
    v = torch.tensor(v0, dtype=torch.float64, device=dev)
    t = torch.tensor(w["types"], dtype=torch.int32, device=dev)
    th = torch.empty((wl["md_per_step"], 4), dtype=torch.float64, device=dev)
    prec = dp.DP_PREC_MIXED if precision is None else precision
    if fast_path:
        fp = student.FastPathMD(ref_model, model, N, tol=FORCE_RMSE_TARGET, check_every=REBUILD_EVERY,
                                precision=prec)
        ctx = fp.fast
    else:
        ctx = dp.Context(model, N, precision=prec)
    store = ctx.embed_store
    # after the fast path's FP64 context, which then takes the G store first when device memory
    # holds only one (its checks run inside the timed region)
    refc = dp.Context(ref_model, N)
    acc_first = _accuracy(dp, ctx, refc, x, t, w["box"])
    dp.dp_md_reset(ctx)
    done = 0

    def step():
        nonlocal done
        n = wl["md_per_step"]
        if fast_path:
            fp.run(x, v, t, w["box"], w["masses"], wl["dt"], n, rebuild_every=REBUILD_EVERY, skin=SKIN)
        else:
            dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], wl["dt"], n, rebuild_every=REBUILD_EVERY,
                          skin=SKIN, thermo=th, check=False)
        done += n

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.set_timing(1)
    evs, thermo_all = [], []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        evs.append((e0, e1))
        if not fast_path:
            thermo_all.append(th.clone())
    torch.cuda.synchronize()
    kt = ctx.kernel_times()
    ctx.set_timing(0)
    total_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    total_ms = float(tmax.item())
    nl, nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"], check=False)
    rows = int(nr.sum().item())
    # the rest of the trajectory, untimed
    while done < wl["traj"]:
        n = min(wl["md_per_step"], wl["traj"] - done)
        if fast_path:
            fp.run(x, v, t, w["box"], w["masses"], wl["dt"], n, rebuild_every=REBUILD_EVERY, skin=SKIN)
        else:
            th2 = torch.empty((n, 4), dtype=torch.float64, device=dev)
            dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], wl["dt"], n, rebuild_every=REBUILD_EVERY,
                          skin=SKIN, thermo=th2, check=False)
            thermo_all.append(th2)
        done += n
    last_ctx = fp.context if fast_path else ctx
    acc_last = _accuracy(dp, last_ctx, refc, x, t, w["box"])
    fl = mixed_kernel_flops(run_desc, rows, N, store)
    groups = {g: {"ms": ms, "launches": n} for g, (ms, n) in kt.items() if n > 0}
    dom = max(groups, key=lambda g: groups[g]["ms"])
    roof = None
    if dom in fl:
        kname = fp64_kernel_key(dom, store)   # embed_tan / embed_bwd_st with the store
        tag = f"{kname}_mx<{run_desc['emb'][0]}" + (", split>" if prec == dp.DP_PREC_MIXED_SPLIT else ">")
        tr = _counter(TRAFFIC, tag)
        roof = _mode_roofline(fl, groups, dom, tag, tr["bytes_per_row"] * rows if tr else None)
    out = {"value": world * N * wl["md_per_step"] * args.steps / (total_ms / 1000.0), "unit": METRIC,
           "ms_per_step": total_ms / args.steps, "dtype": dtype,
           "model": "se_a %s / M2 %d / fit %s" % ("-".join(map(str, run_desc["emb"])), run_desc["m2"],
                                                   "x".join(map(str, run_desc["fit"]))),
           "kernels_ms_per_step": {g: d["ms"] / args.steps for g, d in groups.items()},
           "roofline": roof,
           "embed_store": bool(store),
           "accuracy_vs_fp64_full_model": {"target_force_rmse_eV_per_A": FORCE_RMSE_TARGET,
                                           "first_config": acc_first,
                                           "last_config": dict(acc_last, md_step=done)}}
    if fast_path:
        out["fast_path"] = {"check_every_md_steps": fp.check_every, "tol_force_rmse_eV_per_A": fp.tol,
                            "checks": fp.checks, "switched_to_full_model_at_md_step": fp.switched_at,
                            "note": "timed steps include the FP64 full-model checks that fall inside them"}
    else:
        th_all = torch.cat(thermo_all).cpu().numpy().reshape(-1, 4)
        etot = th_all[:, 0] + th_all[:, 1]
        out["nve"] = {"max_abs_drift_eV_per_atom": float(np.abs(etot - etot[0]).max() / N),
                      "T_last_K": float(th_all[-1, 2]), "md_steps": int(len(th_all))}
    return out


STUDENT_PARAMS = os.path.join(ROOT, "paper_2004_11658_gb300", "data", "student_water12288.npy")


def fp64_kernel_key(dom, store):
    """Counter-table key of an FP64 kernel group: with the G store the
    groups run k_embed_tan_x (embed_fwd) and k_embed_bwd_st (embed_bwd)."""
    if store and dom in ("embed_fwd", "embed_bwd"):
        return {"embed_fwd": "embed_tan", "embed_bwd": "embed_bwd_st"}[dom]
    return dom


def fp64_roofline(desc, groups, dom, rows, nreal, N, store=False):
    """Roofline of the FP64 path's dominant kernel, by unit: the FP64 pipe
    (FP64 FLOPs issued, from the kernel's ncu instruction counts per row),
    the tensor cores (digit-MMA FLOPs issued), and the algorithmic FP64
    FLOPs as an FP64-equivalent rate."""
    flops = kernel_flops(desc, rows, N, store)
    per_launch_s = groups[dom]["ms"] / groups[dom]["launches"] / 1000.0
    pk = measured_peaks()
    bf16_peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1720.9))
    # counters are per kernel instantiation (the embedding width e1); other widths report the
    # FP64-equivalent rate only
    key = fp64_kernel_key(dom, store) + f"<{desc['emb'][0]}>"
    tr = _counter(TRAFFIC, key)
    issued = _counter(FP64_ISSUED, key)
    equiv = flops[dom] / per_launch_s / 1e12 if dom in flops else None
    roof = {"bound": "alu", "kernel": key, "unit": "TFLOP/s", "traffic": tr["bytes_per_row"] * rows if tr else None,
            "rows_per_launch": rows,
            "fp64_equivalent": {"achieved": equiv, "peak": FP64_PEAK_TFLOPS,
                                "frac": equiv / FP64_PEAK_TFLOPS if equiv else None,
                                "what": "algorithmic FP64 FLOPs per launch / time; part of them run on the "
                                        "tensor cores as exact digit products, so this may exceed 1"}}
    if dom == ("embed_fwd" if store else "embed_bwd"):
        mma = digit_mma_flops_bwd(desc, nreal)
        roof["tensor_bf16"] = {"achieved": mma / per_launch_s / 1e12, "peak": bf16_peak,
                               "frac": mma / per_launch_s / 1e12 / bf16_peak,
                               "what": "BF16 digit-MMA FLOPs issued (padded shapes)",
                               "peak_source": "MEASURED_PEAKS bf16_tflops_sustained (of measured)"}
    if issued:
        fp = issued["fp64_flop_per_row"] * rows / per_launch_s / 1e12
        roof["fp64_pipe"] = {"achieved": fp, "peak": FP64_PEAK_TFLOPS, "frac": fp / FP64_PEAK_TFLOPS,
                             "busy_ncu": issued["pipe_busy"],
                             "what": "FP64 FLOPs issued on the FP64 units (2 dfma + dadd + dmul, ncu count "
                                     "per row of the 12,288-atom box); busy_ncu: the FP64 pipe's share of "
                                     "issue cycles (conversions, compares and idle lanes included)"}
        roof.update(achieved=fp, peak=FP64_PEAK_TFLOPS, frac=fp / FP64_PEAK_TFLOPS,
                    peak_source="FP64 pipe: 152 SMs x 2 FMA/clk x 2 FLOP x 2.07 GHz (nominal 1.25 TFLOP/s)")
    else:
        roof.update(achieved=equiv, peak=FP64_PEAK_TFLOPS, frac=equiv / FP64_PEAK_TFLOPS if equiv else None,
                    peak_source="FP64 pipe: 152 SMs x 2 FMA/clk x 2 FLOP x 2.07 GHz (nominal 1.25 TFLOP/s)",
                    note="FP64-equivalent rate (no ncu count of the issued FP64 FLOPs for this source)")
    if store and dom == "embed_fwd" and groups.get("embed_bwd", {}).get("launches"):
        # the streaming backward beside it: FP64 work issued, and its G / dG/ds reads against HBM
        bs = groups["embed_bwd"]["ms"] / groups["embed_bwd"]["launches"] / 1000.0
        kb = f"embed_bwd_st<{desc['emb'][0]}>"
        iss = _counter(FP64_ISSUED, kb)
        trb = _counter(TRAFFIC, kb)
        other = {"kernel": kb, "ms_per_launch": bs * 1e3}
        if iss:
            a = iss["fp64_flop_per_row"] * rows / bs / 1e12
            other["fp64_pipe"] = {"achieved": a, "peak": FP64_PEAK_TFLOPS, "frac": a / FP64_PEAK_TFLOPS,
                                  "busy_ncu": iss["pipe_busy"], "unit": "TFLOP/s"}
        if trb:
            gbs = trb["bytes_per_row"] * rows / bs / 1e9
            other["hbm"] = {"achieved": gbs, "peak": measured_peaks().get("hbm_gbs", 6712.6),
                            "frac": gbs / measured_peaks().get("hbm_gbs", 6712.6), "unit": "GB/s",
                            "traffic": trb["bytes_per_row"] * rows}
        roof["backward"] = other
    return roof


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2004_11658_gb300 import dp, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = WORKLOADS[args.workload]
    w = synth.workload(args.workload)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    m = np.array(w["masses"])[w["types"]]
    v0 = synth.maxwell_velocities(m, wl["T0"], seed=2)
    N = len(m)
    model = dp.Model(desc, P)
    ctx = dp.Context(model, N)
    store = ctx.embed_store
    x = torch.tensor(w["coords"], dtype=torch.float64, device=dev)
    v = torch.tensor(v0, dtype=torch.float64, device=dev)
    t = torch.tensor(w["types"], dtype=torch.int32, device=dev)
    th = torch.empty((wl["md_per_step"], 4), dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    statuses = {}

    def step():
        _, s = dp.dp_md_step(ctx, x, v, t, w["box"], w["masses"], wl["dt"], wl["md_per_step"],
                             rebuild_every=REBUILD_EVERY, skin=SKIN, thermo=th, check=False)
        if s not in (0, -3, -4):  # anything but "results written" conditions is fatal
            raise dp.DPError(s, dp.lib().dp_last_error().decode())
        statuses[dp.STATUS_NAMES[s]] = statuses.get(dp.STATUS_NAMES[s], 0) + 1

    for _ in range(args.warmup):
        step()

    def barrier():
        if world > 1:
            dist.barrier()

    barrier()
    torch.cuda.synchronize()
    ctx.set_timing(1)
    launches0 = ctx.launches
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    sampler.start()
    evs = []
    thermo_all = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                       # L2 flush, outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        evs.append((e0, e1))
        thermo_all.append(th.clone())
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = ctx.launches - launches0
    kt = ctx.kernel_times()
    ctx.set_timing(0)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    total_ms = float(tmax.item())
    value = world * N * wl["md_per_step"] * args.steps / (total_ms / 1000.0)

    # rows actually evaluated (real neighbours, Algorithm 1 on the final positions)
    nl, nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"], check=False)
    rows = int(nr.sum().item())
    nreal = nr.cpu().numpy()
    del nl
    groups = {g: {"ms": ms, "launches": n} for g, (ms, n) in kt.items()}
    timed_groups = {g: d for g, d in groups.items() if d["launches"] > 0}
    dom = max(timed_groups, key=lambda g: timed_groups[g]["ms"])
    roof = fp64_roofline(desc, groups, dom, rows, nreal, N, store=store)
    th_all = torch.stack(thermo_all).cpu().numpy().reshape(-1, 4)
    etot = th_all[:, 0] + th_all[:, 1]

    # end to end: host buffers in pinned memory, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        vh = v.cpu().pin_memory()
        thh = torch.empty_like(th, device="cpu").pin_memory()
        th_h_bytes = thh.numel() * 8
        th_dev_t = t.cpu().pin_memory()
        ev = []
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            x.copy_(xh, non_blocking=True)
            v.copy_(vh, non_blocking=True)
            t.copy_(th_dev_t, non_blocking=True)
            step()
            xh.copy_(x, non_blocking=True)
            vh.copy_(v, non_blocking=True)
            thh.copy_(th, non_blocking=True)
            b.record()
            ev.append((a, b))
        torch.cuda.synchronize()
        e_ms = sum(a.elapsed_time(b) for a, b in ev)
        te = torch.tensor([e_ms], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e_ms = float(te.item())
        e2e = {"value": world * N * wl["md_per_step"] * args.steps / (e_ms / 1000.0), "unit": METRIC,
               "h2d_bytes_per_step": int(2 * N * 3 * 8 + N * 4),
               "d2h_bytes_per_step": int(2 * N * 3 * 8 + th_h_bytes)}
    del ctx
    torch.cuda.empty_cache()

    modes = {}
    if not args.no_mixed:
        modes["mixed"] = measure_mode(args, dp, w, desc, P, model, v0, dev, world, flush,
                                      "bf16 GEMMs (fp32 accumulate) + f64")
        torch.cuda.empty_cache()
        modes["mixed_split"] = measure_mode(args, dp, w, desc, P, model, v0, dev, world, flush,
                                            "embedding GEMMs on split bf16 operands (hi + lo, fp32 accumulate), "
                                            "fitting bf16, + f64", precision=dp.DP_PREC_MIXED_SPLIT)
        torch.cuda.empty_cache()
    if not args.no_student and args.workload.startswith("water"):
        if os.path.exists(STUDENT_PARAMS):
            Ps = np.load(STUDENT_PARAMS).astype(np.float64)
            modes["student"] = measure_mode(args, dp, w, synth.WATER_STUDENT, Ps, model, v0, dev, world, flush,
                                            "bf16 GEMMs (fp32 accumulate) + f64", fast_path=True)
            modes["student"]["params"] = os.path.relpath(STUDENT_PARAMS, ROOT)
        else:
            modes["student"] = {"unavailable": "no trained student parameters at "
                                + os.path.relpath(STUDENT_PARAMS, ROOT)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, desc, P, args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, w, world),
            "gpu_launches": launches,
            "roofline": roof,
            "embed_store": {"on": bool(store),
                            "what": "G and dG/ds of every real row kept in HBM between the embedding forward "
                                    "(k_embed_tan_x) and the streaming backward (k_embed_bwd_st)"},
            "kernels_ms_per_step": {g: d["ms"] / args.steps for g, d in timed_groups.items()},
            "nve": {"etot_first": float(etot[0]), "etot_last": float(etot[-1]),
                    "max_abs_drift_eV_per_atom": float(np.abs(etot - etot[0]).max() / N),
                    "T_last_K": float(th_all[-1, 2]), "md_steps": int(len(th_all))},
            "status_counts": statuses,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "modes": modes,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_slab(args, rank, world, local_rank):
    """One system cut into `world` slabs along x, one per rank/GPU (Sec. 3.1):
    every MD step runs the forward halo, dp_eval_local, the reverse halo and
    the all-reduce (NCCL), kicks and drifts through the library; re-plans
    with atom migration every 10 steps.  value = atoms x steps / max time."""
    import torch
    import torch.distributed as dist
    from paper_2004_11658_gb300 import domain, dp, synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = WORKLOADS[args.workload]
    w = synth.workload(args.workload)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    m = np.array(w["masses"])[w["types"]]
    N = len(m)
    v0 = synth.maxwell_velocities(m, wl["T0"], seed=2)
    model = dp.Model(desc, P)
    rho = N / float(np.prod(w["box"]))
    # owned atoms plus ghosts (a slab's own periodic images included), with room for density swings
    cap_atoms = int(N / world * (1.0 + 2.0 * (desc["rcut"] + SKIN) * world / w["box"][0]) * 1.3 + 1024)
    ev = domain.DPLocalEvaluator(model, cap_atoms, rho)
    comm = domain.LocalComm(1) if world == 1 else domain.DistComm(rank, world)
    md = domain.SlabMD(comm, w["box"], desc["rcut"], SKIN, torch.tensor(w["coords"], device=dev),
                       torch.tensor(v0, device=dev), torch.tensor(w["types"], device=dev), w["masses"], wl["dt"],
                       [ev], [domain.GPUIntegrator(ev.ctx)], replan_every=REBUILD_EVERY)

    def step():
        for _ in range(wl["md_per_step"]):
            md.step()

    for _ in range(args.warmup):
        step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev.ctx.set_timing(1)
    l0 = ev.ctx.launches
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    tm = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    ms = float(tm.item())
    kt = ev.ctx.kernel_times()
    if rank == 0:
        cfg = workload_config(args.workload, w, world)
        cfg["parallelism"] = f"slab x{world}"
        print(json.dumps({
            "metric": METRIC, "value": N * wl["md_per_step"] * args.steps / (ms / 1000.0), "unit": METRIC,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "gpu_launches": ev.ctx.launches - l0,
            "kernels_ms_per_step_rank0": {g: v[0] / args.steps for g, v in kt.items() if v[1]},
            "wall_s": time.perf_counter() - t0, "e2e": None, "cpu_baseline": None}), flush=True)
    return 0


def profile_eval(args):
    """Small profiling driver: N x (candidate build + dp_eval) of the workload."""
    import torch
    from paper_2004_11658_gb300 import dp, synth
    w = synth.workload(args.workload)
    desc = w["model"]
    P = synth.model_params(desc, 0)
    if args.profile_model == "student":
        desc, P = synth.WATER_STUDENT, np.load(STUDENT_PARAMS).astype(np.float64)
    model = dp.Model(desc, P)
    prec = {"fp64": dp.DP_PREC_FP64, "mixed": dp.DP_PREC_MIXED,
            "split": dp.DP_PREC_MIXED_SPLIT}[args.profile_precision]
    ctx = dp.Context(model, len(w["coords"]), precision=prec)
    x = torch.tensor(w["coords"], device="cuda")
    t = torch.tensor(w["types"], device="cuda")
    for _ in range(args.profile_eval):
        dp.dp_build_nlist(ctx, x, t, w["box"], SKIN)
        out = dp.dp_eval(ctx, x, t, w["box"])
    torch.cuda.synchronize()
    print(f"profile-eval {args.workload}: {args.profile_eval} evaluations, E = {out['energy'].item():.10f}, "
          f"{ctx.launches} launches")
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.profile_eval:
        return profile_eval(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.decomp == "slab":
            return run_slab(args, rank, world, local_rank)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

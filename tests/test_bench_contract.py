"""bench.py's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys the benchmark contract requires."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "water192", "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "atom-steps/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "water192"


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_flop_counts_per_unit():
    """The roofline's algorithmic FLOPs per unit, worked out by hand from the
    nets of Sec. 4 (water: embedding 25-50-100, M2 = 16, fitting 240 x 3;
    copper: embedding 32-64-128): multiply-add = 2, tanh not counted."""
    from paper_2004_11658_gb300 import synth
    b = _bench_module()
    w = synth.WATER_MODEL
    # one embedding pass per row: 2 (25 + 25*50 + 50*100)
    assert b.emb_row_flops(w) == 12550
    # fitting per atom: 2 (1600*240 + 240*240 + 240*240 + 240)
    assert b.fit_atom_flops(w) == 998880
    one_row = b.kernel_flops(w, rows=1, natoms=0)
    one_atom = b.kernel_flops(w, rows=0, natoms=1)
    assert one_row["embed_fwd"] == 12550 + 8 * 100          # + T = R~^T G
    assert one_row["embed_bwd"] == 26700                    # G and dG/ds, two 4 x M contractions
    assert one_atom["embed_fwd"] == 8 * 16 * 100            # D = T_<^T T
    assert one_atom["embed_bwd"] == 25600                   # gT
    assert one_atom["fit"] == 2 * 998880                    # forward and backward to D
    cu = synth.CU_MODEL
    assert b.kernel_flops(cu, rows=1, natoms=0)["embed_bwd"] == 43136


def test_store_flop_counts_and_counter_keys():
    """With G and dG/ds kept between the two embedding kernels the forward
    does the net with its s-tangent (two passes of the GEMMs) and T, the
    backward only the contractions with dE/dT; the sum over both equals the
    recompute path's minus one embedding pass.  The ncu counter tables are
    looked up per kernel instantiation (embedding width)."""
    from paper_2004_11658_gb300 import synth
    b = _bench_module()
    w = synth.WATER_MODEL
    st = b.kernel_flops(w, rows=1, natoms=0, store=True)
    rc = b.kernel_flops(w, rows=1, natoms=0, store=False)
    assert st["embed_fwd"] == 2 * 12550 + 8 * 100
    assert st["embed_bwd"] == 16 * 100
    assert st["embed_fwd"] + st["embed_bwd"] == rc["embed_fwd"] + rc["embed_bwd"] - 12550
    assert b.kernel_flops(w, rows=0, natoms=1, store=True) == b.kernel_flops(w, rows=0, natoms=1)
    mx = b.mixed_kernel_flops(w, rows=1, natoms=0, store=True)
    assert mx["embed_bwd"]["tensor"] == 0 and mx["embed_fwd"]["tensor"] == 2 * (12550 - 50)
    assert b.fp64_kernel_key("embed_fwd", True) == "embed_tan"
    assert b.fp64_kernel_key("embed_bwd", True) == "embed_bwd_st"
    assert b.fp64_kernel_key("embed_bwd", False) == "embed_bwd"
    assert b.fp64_kernel_key("fit", True) == "fit"
    for table in (b.TRAFFIC, b.FP64_ISSUED, b.MODE_PIPES):
        for key, entry in table.items():
            assert key.endswith(">"), key  # one entry per instantiation
            assert entry["file"] in ("embed_x.cu", "mixed.cu")


def test_reference_arm_under_torchrun_two_ranks():
    """Launched as the multi-GPU bench is (torchrun, two ranks): rank 0 alone
    prints the reference line, the other rank exits 0 without work."""
    port = 29600 + (os.getpid() % 1000)
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--workload", "water192", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0

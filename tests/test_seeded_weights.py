"""The seeded model generator (no trained model exists, so weights are drawn
from a seed): splitmix64 -> 53-bit uniforms -> Box-Muller normals, scaled per
layer.  Pinned to the generator's published definition (known first outputs
of splitmix64), to the normal distribution, and to the C ABI's
dp_model_params_from_seed value for value (host code; no GPU needed)."""
import math

import numpy as np
import pytest


def test_splitmix64_known_outputs(synth):
    # first three outputs of splitmix64 from seed 0 (Steele, Lea and Flood,
    # 2014; the reference implementation's well-known start of the sequence)
    z = synth.splitmix64(0, np.arange(1, 4, dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_is_a_sequence(synth):
    """Output i of the counter form equals the i-th step of the sequential
    generator (state += gamma, then the mix) in plain Python integers."""
    seed, mask = 987654321, (1 << 64) - 1
    state, seq = seed, []
    for _ in range(50):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        seq.append(z ^ (z >> 31))
    got = synth.splitmix64(seed, np.arange(1, 51, dtype=np.uint64))
    assert [int(v) for v in got] == seq


def test_normals_are_standard_normal(synth):
    stats = pytest.importorskip("scipy.stats")
    n = 1 << 20
    z = synth.seeded_normals(3, n)
    assert abs(z.mean()) < 5e-3 and abs(z.std() - 1) < 5e-3
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two branches of each Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5e-3
    # and so are neighbouring pairs
    assert abs(np.corrcoef(z[0:-2:2], z[2::2])[0, 1]) < 5e-3
    # prefix property: the first k normals do not depend on n
    np.testing.assert_array_equal(synth.seeded_normals(3, 1001), z[:1001])


def test_layer_scales(synth):
    desc = synth.WATER_MODEL
    P = synth.model_params(desc, 0)
    off = 0
    for name, shape in synth.layer_shapes(desc):
        n = int(np.prod(shape))
        blk = P[off:off + n]
        off += n
        kind = name.split(".")[1]
        if kind == "bo":
            assert np.all(blk == 0.0)
            continue
        if n < 1000:
            continue
        if kind.startswith("W"):
            fan_in = shape[0] if len(shape) == 2 else 1
            exp = 1.0 / math.sqrt(fan_in + shape[-1])
            if name.startswith("fit") and kind == "W1":
                exp *= desc["fit_in_gain"]
        else:
            exp = 1.0
        assert blk.std() == pytest.approx(exp, rel=0.05), name
    assert off == len(P)


@pytest.mark.parametrize("which", ["water", "copper", "student"])
def test_c_abi_generator_matches_value_for_value(synth, which):
    from paper_2004_11658_gb300 import dp
    desc = {"water": synth.WATER_MODEL, "copper": synth.CU_MODEL, "student": synth.WATER_STUDENT}[which]
    for seed in (0, 1, 2 ** 64 - 1):
        a = dp.dp_model_params_from_seed(desc, seed)
        b = synth.model_params(desc, seed)
        np.testing.assert_array_equal(a, b)
    a = dp.dp_model_params_from_seed(desc, 5, fit_in_gain=1.0, out_scale=3.0)
    np.testing.assert_array_equal(a, synth.model_params(desc, 5, fit_in_gain=1.0, out_scale=3.0))


def test_c_abi_generator_errors(synth):
    import ctypes
    from paper_2004_11658_gb300 import dp
    c = dp.make_desc(synth.WATER_MODEL)
    n = dp.dp_model_nparams(c)
    buf = np.empty(n + 1)
    st = dp.lib().dp_model_params_from_seed(ctypes.byref(c), 0, 300.0, 0.02, buf.ctypes.data_as(ctypes.c_void_p),
                                            n + 1)
    assert st == dp.DP_ERR_ARG
    st = dp.lib().dp_model_params_from_seed(ctypes.byref(c), 0, float("nan"), 0.02,
                                            buf.ctypes.data_as(ctypes.c_void_p), n)
    assert st == dp.DP_ERR_ARG

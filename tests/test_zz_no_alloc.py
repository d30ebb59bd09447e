"""The no-allocation entry point dp_format_nlist_noalloc.

It serves callers that cannot allocate device memory when they need the
formatted neighbour list (a host MD engine with a fixed device budget, code
where cudaMalloc is not allowed): its scratch is a fixed file-scope device
array.  Its output must equal dp_format_nlist's, bit for bit, on two calls in
a row (the second call reuses the array the first one left behind).  This
file is collected last on purpose.
"""
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


def _systems(synth):
    w1 = synth.workload("water192")
    w2 = synth.sub_box_water(6, 6 * 49.7 / 16)   # 648 atoms, cell-list path in the context
    c, t, b = synth.copper_fcc(6)
    w3 = dict(coords=c, types=t, box=b, model=synth.CU_MODEL)
    return [(w1, 0.0), (w2, 2.0), (w3, 0.0)]


def test_noalloc_matches_dp_format_nlist_twice(dp, synth):
    for w, skin in _systems(synth):
        desc = w["model"]
        N = len(w["coords"])
        x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
        t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
        model = dp.Model(desc, synth.model_params(desc, 0))
        ctx = dp.Context(model, N)
        dp.dp_build_nlist(ctx, x, t, w["box"], skin)
        ref_nl, ref_nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"])
        for _ in range(2):
            nl = torch.full_like(ref_nl, -7)
            nr = torch.full_like(ref_nr, -7)
            dp.dp_format_nlist_noalloc(desc, x, t, w["box"], skin, nl, nr)
            assert torch.equal(nl, ref_nl)
            assert torch.equal(nr, ref_nr)


def test_noalloc_rejects_sizes_beyond_its_scratch(dp, synth):
    w = synth.workload("water192")
    desc = w["model"]
    n = 2049
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    nl = torch.empty((n, sum(desc["sel"])), dtype=torch.int32, device="cuda")
    nr = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(dp.DPError) as e:
        dp.dp_format_nlist_noalloc(desc, x, t, np.array([60.0, 60.0, 60.0]), 0.0, nl, nr)
    assert e.value.status == -9


def _reference(dp, synth, w, skin):
    desc = w["model"]
    N = len(w["coords"])
    x = torch.tensor(w["coords"], dtype=torch.float64, device="cuda")
    t = torch.tensor(w["types"], dtype=torch.int32, device="cuda")
    model = dp.Model(desc, synth.model_params(desc, 0))
    ctx = dp.Context(model, N)
    dp.dp_build_nlist(ctx, x, t, w["box"], skin)
    nl, nr, _ = dp.dp_format_nlist(ctx, x, t, w["box"])
    return x, t, nl, nr


def test_noalloc_allocates_nothing_on_a_second_call(dp, synth):
    """Device memory is unchanged across a call once the first call has been
    made (the first one may load the array's module)."""
    w = synth.workload("water192")
    x, t, ref_nl, ref_nr = _reference(dp, synth, w, 0.0)
    nl = torch.empty_like(ref_nl)
    nr = torch.empty_like(ref_nr)
    dp.dp_format_nlist_noalloc(w["model"], x, t, w["box"], 0.0, nl, nr)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    dp.dp_format_nlist_noalloc(w["model"], x, t, w["box"], 0.0, nl, nr)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(nl, ref_nl) and torch.equal(nr, ref_nr)


def test_noalloc_errors_after_the_kernels_then_recovers(dp, synth):
    """More candidates than the scratch holds (600 atoms in a 3 A cube, all
    within rcut of each other) gives DP_ERR_CAPACITY, a type id >= ntypes
    DP_ERR_TYPE; a valid call after each still equals dp_format_nlist."""
    w = synth.workload("water192")
    desc = w["model"]
    x, t, ref_nl, ref_nr = _reference(dp, synth, w, 0.0)
    rng = np.random.default_rng(9)
    n = 600
    xc = torch.tensor(6.0 + rng.uniform(0.0, 3.0, (n, 3)), dtype=torch.float64, device="cuda")
    tc = torch.zeros(n, dtype=torch.int32, device="cuda")
    nlc = torch.empty((n, sum(desc["sel"])), dtype=torch.int32, device="cuda")
    nrc = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    bad_t = t.clone()
    bad_t[17] = 2
    cases = [((desc, xc, tc, np.array([13.0, 13.0, 13.0]), 0.0, nlc, nrc), -9),
             ((desc, x, bad_t, w["box"], 0.0, torch.empty_like(ref_nl), torch.empty_like(ref_nr)), -11)]
    for args, code in cases:
        with pytest.raises(dp.DPError) as e:
            dp.dp_format_nlist_noalloc(*args)
        assert e.value.status == code
        nl = torch.full_like(ref_nl, -7)
        nr = torch.full_like(ref_nr, -7)
        dp.dp_format_nlist_noalloc(desc, x, t, w["box"], 0.0, nl, nr)
        assert torch.equal(nl, ref_nl) and torch.equal(nr, ref_nr)

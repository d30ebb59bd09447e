"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dp.h declares (host-only calls; no kernel runs here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dp_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("dp_build_nlist", "dp_eval", "dp_md_step", "dp_model_create", "dp_ctx_create"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2004_11658_gb300 import dp
    L = dp.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_host_calls(synth):
    from paper_2004_11658_gb300 import dp
    for desc in (synth.WATER_MODEL, synth.CU_MODEL, synth.WATER_STUDENT):
        assert dp.dp_model_nparams(desc) == synth.n_params(desc)
    bad = dict(synth.WATER_MODEL, emb=(25, 50, 200))
    assert dp.dp_model_nparams(bad) == -1
    bad = dict(synth.WATER_MODEL, rcut_smth=7.0)
    assert dp.dp_model_nparams(bad) == -1
    L = dp.lib()
    for code in range(-11, 1):
        assert L.dp_status_string(code)
    # a NULL descriptor is an argument error with a message, not a crash
    h = ctypes.c_void_p()
    assert L.dp_model_create(None, None, 0, ctypes.byref(h)) == -1
    assert L.dp_last_error()
    # the G-store switch on a NULL context: an argument error, and -1 from the query
    assert L.dp_ctx_set_embed_store(None, 1) == -1
    assert L.dp_ctx_set_embed_store(None, 0) == -1
    assert L.dp_ctx_embed_store(None) == -1

"""ctypes wrapper of the plain C FP64 oracle (dp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and
the benchmark's CPU-baseline leg, never by the library.  It builds the C
file with gcc on first use (no FMA contraction, OpenMP over atoms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdp_oracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force=False):
    """Compile the oracle shared library (gcc, -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_switch.argtypes = [ctypes.c_double] * 3 + [_d, _d]
            L.orc_nparams.argtypes = [_i32, _d]
            L.orc_nparams.restype = ctypes.c_long
            L.orc_candidates.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_double, ctypes.c_int32, _i32, _i32]
            L.orc_candidates.restype = ctypes.c_int64
            L.orc_candidates_cells.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _d, ctypes.c_double,
                                               ctypes.c_int32, _i32, _i32]
            L.orc_candidates_cells.restype = ctypes.c_int64
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_format.argtypes = [ctypes.c_int64, _d, _i32, _d, _i32, _i32, ctypes.c_int32,
                                     ctypes.c_int32, _i32, ctypes.c_double, _i32, _i32, _i64]
            L.orc_eval.argtypes = [_i32, _d, _d, ctypes.c_int64, _d, _i32, _d, _i32, _d, _d, _d, _d, _d]
            L.orc_eval_local.argtypes = [_i32, _d, _d, ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, _i32,
                                         _d, _d, _d, _d, _d]
            L.orc_md.argtypes = [_i32, _d, _d, ctypes.c_int64, _d, _d, _i32, _d, _d, ctypes.c_double,
                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                 _d, _i32, _d]
            L.orc_md.restype = ctypes.c_int64
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_param_grad.argtypes = [_i32, _d, _d, ctypes.c_int64, _d, _i32, _d, _i32, ctypes.c_double, _d, _d]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _desc_arrays(desc):
    sel = list(desc["sel"]) + [0] * (8 - len(desc["sel"]))
    emb = list(desc["emb"]) + [0] * (4 - len(desc["emb"]))
    fit = list(desc["fit"]) + [0] * (4 - len(desc["fit"]))
    idesc = np.array([desc["ntypes"], *sel, len(desc["emb"]), *emb, desc["m2"], len(desc["fit"]),
                      *fit, int(desc.get("desc_scale_nm", 1))], dtype=np.int32)
    ddesc = np.array([desc["rcut"], desc["rcut_smth"]], dtype=np.float64)
    return idesc, ddesc


def num_threads():
    return int(lib().orc_num_threads())


def nparams(desc):
    i, d = _desc_arrays(desc)
    return int(lib().orc_nparams(_p(i, _i32), _p(d, _d)))


def switch(r, rs, rc):
    s = ctypes.c_double()
    ds = ctypes.c_double()
    lib().orc_switch(float(r), float(rs), float(rc), ctypes.byref(s), ctypes.byref(ds))
    return s.value, ds.value


def set_num_threads(n):
    """OpenMP threads of every later oracle call."""
    lib().orc_set_num_threads(int(n))


def candidates(coords, box, rlist, cap, method="auto", ncentre=None):
    """Neighbour candidates within rlist, increasing j per centre.

    method: "brute" (O(N^2)), "cells" (cell list; needs >= 3 cells per axis),
    "auto" (cells where possible).  ncentre: only centres [0, ncentre) are
    built (cell list only); the other rows are left empty."""
    x = np.ascontiguousarray(coords, dtype=np.float64)
    N = len(x)
    nc = N if ncentre is None else int(ncentre)
    ncand = np.zeros(N, dtype=np.int32)
    cand = np.full((N, cap), -1, dtype=np.int32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    if method in ("auto", "cells"):
        over = lib().orc_candidates_cells(N, nc, _p(x, _d), _p(b, _d), float(rlist), int(cap), _p(ncand, _i32),
                                          _p(cand, _i32))
        if over >= 0:
            return ncand, cand, int(over)
        if method == "cells" or nc != N:
            raise ValueError("cell list needs at least 3 cells per axis (box edge >= 3 rlist)")
    over = lib().orc_candidates(N, _p(x, _d), _p(b, _d), float(rlist), int(cap), _p(ncand, _i32), _p(cand, _i32))
    return ncand, cand, int(over)


def format_nlist(coords, types, box, ncand, cand, sel, rcut, ncentre=None):
    """Algorithm 1 for the centres [0, ncentre) (all atoms by default); the
    neighbours may be any of the atoms."""
    x = np.ascontiguousarray(coords, dtype=np.float64)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    N = len(x) if ncentre is None else int(ncentre)
    cap = cand.shape[1]
    sel_a = np.ascontiguousarray(sel, dtype=np.int32)
    nm = int(sel_a.sum())
    nlist = np.empty((N, nm), dtype=np.int32)
    nreal = np.empty((N, len(sel_a)), dtype=np.int32)
    ovf = np.empty(N, dtype=np.int64)
    lib().orc_format(N, _p(x, _d), _p(t, _i32), _p(b, _d), _p(np.ascontiguousarray(ncand, dtype=np.int32), _i32),
                     _p(np.ascontiguousarray(cand, dtype=np.int32), _i32), int(cap), len(sel_a),
                     _p(sel_a, _i32), float(rcut), _p(nlist, _i32), _p(nreal, _i32), _p(ovf, _i64))
    return nlist, nreal, ovf


def eval_nlist(desc, params, coords, types, box, nlist, want_descriptor=False, nloc=None):
    """Evaluation on a formatted list.  With nloc, only the centres [0, nloc)
    are evaluated (nlist holds their rows): E and the virial of those
    centres, and their force increments on all atoms."""
    if nloc is not None:
        return _eval_centres(desc, params, coords, types, box, nlist, int(nloc))
    i, d = _desc_arrays(desc)
    x = np.ascontiguousarray(coords, dtype=np.float64)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    P = np.ascontiguousarray(params, dtype=np.float64)
    nl = np.ascontiguousarray(nlist, dtype=np.int32)
    N = len(x)
    E = np.zeros(1)
    F = np.zeros((N, 3))
    V = np.zeros(9)
    Ei = np.zeros(N)
    M = desc["emb"][-1]
    D = np.zeros((N, desc["m2"] * M)) if want_descriptor else None
    rc = lib().orc_eval(_p(i, _i32), _p(d, _d), _p(P, _d), N, _p(x, _d), _p(t, _i32), _p(b, _d),
                        _p(nl, _i32), _p(E, _d), _p(F, _d), _p(V, _d), _p(Ei, _d), _p(D, _d))
    if rc != 0:
        raise RuntimeError(f"orc_eval failed: {rc}")
    out = dict(energy=float(E[0]), force=F, virial=V.reshape(3, 3), atom_energy=Ei)
    if want_descriptor:
        out["descriptor"] = D
    return out


def _eval_centres(desc, params, coords, types, box, nlist, nloc):
    i, d = _desc_arrays(desc)
    x = np.ascontiguousarray(coords, dtype=np.float64)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    P = np.ascontiguousarray(params, dtype=np.float64)
    nl = np.ascontiguousarray(nlist[:nloc], dtype=np.int32)
    N = len(x)
    E = np.zeros(1)
    F = np.zeros((N, 3))
    V = np.zeros(9)
    Ei = np.zeros(max(nloc, 1))
    rc = lib().orc_eval_local(_p(i, _i32), _p(d, _d), _p(P, _d), N, nloc, _p(x, _d), _p(t, _i32), _p(b, _d),
                              _p(nl, _i32), _p(E, _d), _p(F, _d), _p(V, _d), _p(Ei, _d), None)
    if rc != 0:
        raise RuntimeError(f"orc_eval_local failed: {rc}")
    return dict(energy=float(E[0]), force=F, virial=V.reshape(3, 3), atom_energy=Ei[:nloc])


def evaluate_local(desc, params, coords, types, box, nloc, cap=None):
    """Sub-region evaluation (Sec. 3.1): atoms [0, nloc) are the centres,
    [nloc, N) ghost atoms that only appear as neighbours.  Returns E and the
    virial of the centres and the force increments on all N atoms."""
    N = len(coords)
    if cap is None:
        cap = default_cap(desc, box, N, 0.0)
    i, d = _desc_arrays(desc)
    x = np.ascontiguousarray(coords, dtype=np.float64)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    P = np.ascontiguousarray(params, dtype=np.float64)
    ncand, cand, over = candidates(x, b, desc["rcut"], cap)
    if over:
        raise RuntimeError("candidate capacity exceeded")
    nlist, _, _ = format_nlist(x, t, b, ncand, cand, desc["sel"], desc["rcut"])
    E = np.zeros(1)
    F = np.zeros((N, 3))
    V = np.zeros(9)
    Ei = np.zeros(max(nloc, 1))
    rc = lib().orc_eval_local(_p(i, _i32), _p(d, _d), _p(P, _d), N, int(nloc), _p(x, _d), _p(t, _i32), _p(b, _d),
                              _p(nlist, _i32), _p(E, _d), _p(F, _d), _p(V, _d), _p(Ei, _d), None)
    if rc != 0:
        raise RuntimeError(f"orc_eval_local failed: {rc}")
    return dict(energy=float(E[0]), force=F, virial=V.reshape(3, 3), atom_energy=Ei[:nloc])


def default_cap(desc, box, N, skin):
    rho = N / float(np.prod(box))
    rl = desc["rcut"] + skin
    expect = rho * 4.0 / 3.0 * np.pi * rl ** 3
    return int(np.ceil((1.5 * expect + 64) / 32.0) * 32)


def evaluate(desc, params, coords, types, box, skin=0.0, cap=None, want_descriptor=False):
    """Full evaluation: candidates (rcut+skin) -> Algorithm 1 -> E, F, virial."""
    N = len(coords)
    if cap is None:
        cap = default_cap(desc, box, N, skin)
    ncand, cand, over = candidates(coords, box, desc["rcut"] + skin, cap)
    if over:
        raise RuntimeError("candidate capacity exceeded")
    nlist, nreal, ovf = format_nlist(coords, types, box, ncand, cand, desc["sel"], desc["rcut"])
    out = eval_nlist(desc, params, coords, types, box, nlist, want_descriptor)
    out["nlist"] = nlist
    out["nreal"] = nreal
    out["overflow"] = int(ovf.sum())
    return out


def md(desc, params, coords, vel, types, box, masses, dt, nsteps, rebuild_every=10, skin=2.0,
       cap=None, force=None):
    """Velocity-Verlet run; returns (coords, vel, force, thermo[nsteps,4], overflow_count)."""
    i, d = _desc_arrays(desc)
    x = np.array(coords, dtype=np.float64, copy=True)
    v = np.array(vel, dtype=np.float64, copy=True)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    P = np.ascontiguousarray(params, dtype=np.float64)
    m = np.ascontiguousarray(masses, dtype=np.float64)
    N = len(x)
    if cap is None:
        cap = default_cap(desc, box, N, skin)
    F = np.zeros((N, 3)) if force is None else np.array(force, dtype=np.float64, copy=True)
    have = np.array([0 if force is None else 1], dtype=np.int32)
    thermo = np.zeros((nsteps, 4))
    st = lib().orc_md(_p(i, _i32), _p(d, _d), _p(P, _d), N, _p(x, _d), _p(v, _d), _p(t, _i32), _p(b, _d),
                      _p(m, _d), float(dt), int(nsteps), int(rebuild_every), float(skin), int(cap),
                      _p(F, _d), _p(have, _i32), _p(thermo, _d))
    if st < 0:
        raise RuntimeError(f"orc_md failed: {st}")
    return x, v, F, thermo, int(st)


def param_grad(desc, params, coords, types, box, cE, lam, skin=0.0, cap=None):
    """d/dW of cE * E + sum_i lam_i . F_i (the parameter gradient of any loss
    on E and F with dLoss/dE = cE, dLoss/dF = lam), on the formatted list."""
    i, d = _desc_arrays(desc)
    x = np.ascontiguousarray(coords, dtype=np.float64)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    P = np.ascontiguousarray(params, dtype=np.float64)
    N = len(x)
    if cap is None:
        cap = default_cap(desc, box, N, skin)
    ncand, cand, over = candidates(x, b, desc["rcut"] + skin, cap)
    nlist, _, _ = format_nlist(x, t, b, ncand, cand, desc["sel"], desc["rcut"])
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    g = np.zeros(len(P))
    rc = lib().orc_param_grad(_p(i, _i32), _p(d, _d), _p(P, _d), N, _p(x, _d), _p(t, _i32), _p(b, _d),
                              _p(nlist, _i32), float(cE), _p(lam, _d), _p(g, _d))
    if rc != 0:
        raise RuntimeError(f"orc_param_grad failed: {rc}")
    return g

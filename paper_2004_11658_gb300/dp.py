"""Thin Python binding of the C ABI in include/dp.h (ctypes).

Argument marshalling only: every step of the path runs in the CUDA library
libdp_gb300.so.  PyTorch supplies device memory and streams.  If the library
cannot be built or loaded this module raises; there is no CPU fallback.

The functions keep the C names (dp_build_nlist, dp_eval, dp_md_step, ...);
``Model`` and ``Context`` wrap the handles.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

DP_OK = 0
STATUS_NAMES = {
    0: "DP_OK", -1: "DP_ERR_ARG", -2: "DP_ERR_BOX", -3: "DP_ERR_SEL_OVERFLOW",
    -4: "DP_ERR_NLIST_STALE", -5: "DP_ERR_NONFINITE", -6: "DP_ERR_FILE", -7: "DP_ERR_CUDA",
    -8: "DP_ERR_UNSUPPORTED", -9: "DP_ERR_CAPACITY", -10: "DP_ERR_NOMEM", -11: "DP_ERR_TYPE",
}
globals().update({name: code for code, name in STATUS_NAMES.items()})
DP_PREC_FP64 = 0
DP_PREC_MIXED = 1
DP_PREC_FP64_SIMT = 2
DP_PREC_MIXED_SPLIT = 3


class DPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class dp_model_desc(ctypes.Structure):
    _fields_ = [("ntypes", ctypes.c_int32), ("sel", ctypes.c_int32 * 8), ("n_emb", ctypes.c_int32),
                ("emb", ctypes.c_int32 * 4), ("m2", ctypes.c_int32), ("n_fit", ctypes.c_int32),
                ("fit", ctypes.c_int32 * 4), ("desc_scale_nm", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rcut", ctypes.c_double), ("rcut_smth", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double


def lib():
    """Load (building first if needed) libdp_gb300.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB if _build.up_to_date() else _build.build()
            L = ctypes.CDLL(path)
            L.dp_last_error.restype = ctypes.c_char_p
            L.dp_status_string.restype = ctypes.c_char_p
            L.dp_status_string.argtypes = [_i32]
            L.dp_model_nparams.restype = _i64
            L.dp_model_nparams.argtypes = [ctypes.POINTER(dp_model_desc)]
            L.dp_model_create.restype = _i32
            L.dp_model_create.argtypes = [ctypes.POINTER(dp_model_desc), _vp, _i64, ctypes.POINTER(_vp)]
            L.dp_model_load.restype = _i32
            L.dp_model_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(_vp)]
            L.dp_model_save.restype = _i32
            L.dp_model_save.argtypes = [_vp, ctypes.c_char_p]
            L.dp_model_free.argtypes = [_vp]
            L.dp_ctx_create.restype = _i32
            L.dp_ctx_create.argtypes = [_vp, _i64, _i32, _i32, _vp, ctypes.POINTER(_vp)]
            L.dp_ctx_free.argtypes = [_vp]
            L.dp_ctx_set_sync.restype = _i32
            L.dp_ctx_set_sync.argtypes = [_vp, _i32]
            L.dp_ctx_status.restype = _i32
            L.dp_ctx_status.argtypes = [_vp]
            L.dp_ctx_launches.restype = _i64
            L.dp_ctx_launches.argtypes = [_vp]
            L.dp_ctx_set_embed_store.restype = _i32
            L.dp_ctx_set_embed_store.argtypes = [_vp, _i32]
            L.dp_ctx_embed_store.restype = _i32
            L.dp_ctx_embed_store.argtypes = [_vp]
            L.dp_build_nlist.restype = _i32
            L.dp_build_nlist.argtypes = [_vp, _vp, _vp, _vp, _i64, _dbl]
            L.dp_format_nlist.restype = _i32
            L.dp_format_nlist.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _vp]
            L.dp_eval.restype = _i32
            L.dp_eval.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp]
            L.dp_eval_local.restype = _i32
            L.dp_eval_local.argtypes = [_vp, _vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]
            L.dp_md_step.restype = _i32
            L.dp_md_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _dbl, _i32, _i32, _dbl, _vp]
            L.dp_md_kick_drift.restype = _i32
            L.dp_md_kick_drift.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _dbl]
            L.dp_md_kick.restype = _i32
            L.dp_md_kick.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _dbl]
            L.dp_md_get_force.restype = _i32
            L.dp_md_get_force.argtypes = [_vp, _vp, _i64]
            L.dp_md_reset.restype = _i32
            L.dp_md_reset.argtypes = [_vp]
            L.dp_ctx_set_timing.restype = _i32
            L.dp_ctx_set_timing.argtypes = [_vp, _i32]
            L.dp_ctx_kernel_times.restype = _i32
            L.dp_ctx_kernel_times.argtypes = [_vp, _vp, _vp]
            L.dp_kernel_group_name.restype = ctypes.c_char_p
            L.dp_kernel_group_name.argtypes = [_i32]
            L.dp_param_grad.restype = _i32
            L.dp_param_grad.argtypes = [_vp, _vp, _vp, _vp, _i64, _dbl, _vp, _vp]
            L.dp_model_set_params.restype = _i32
            L.dp_model_set_params.argtypes = [_vp, _vp, _i64]
            L.dp_tanh_f64.restype = _i32
            L.dp_tanh_f64.argtypes = [_vp, _vp, _i64, _vp]
            L.dp_model_params_from_seed.restype = _i32
            L.dp_model_params_from_seed.argtypes = [ctypes.POINTER(dp_model_desc), ctypes.c_uint64, _dbl, _dbl,
                                                    _vp, _i64]
            L.dp_model_from_seed.restype = _i32
            L.dp_model_from_seed.argtypes = [ctypes.POINTER(dp_model_desc), ctypes.c_uint64, _dbl, _dbl,
                                             ctypes.POINTER(_vp)]
            L.dp_format_nlist_noalloc.restype = _i32
            L.dp_format_nlist_noalloc.argtypes = [ctypes.POINTER(dp_model_desc), _vp, _vp, _vp, _i64, _dbl,
                                                  _vp, _vp, _vp]
            _lib = L
    return _lib


def lib_path():
    return _build.LIB


def _check(status, ok=(DP_OK,)):
    if status not in ok:
        raise DPError(status, lib().dp_last_error().decode())
    return status


def make_desc(d):
    """dp_model_desc from a dict (keys as in synth.WATER_MODEL)."""
    c = dp_model_desc()
    c.ntypes = d["ntypes"]
    for a, s in enumerate(d["sel"]):
        c.sel[a] = s
    c.n_emb = len(d["emb"])
    for l, w in enumerate(d["emb"]):
        c.emb[l] = w
    c.m2 = d["m2"]
    c.n_fit = len(d["fit"])
    for l, w in enumerate(d["fit"]):
        c.fit[l] = w
    c.desc_scale_nm = int(d.get("desc_scale_nm", 1))
    c.rcut = float(d["rcut"])
    c.rcut_smth = float(d["rcut_smth"])
    return c


def dp_model_nparams(desc):
    c = make_desc(desc) if isinstance(desc, dict) else desc
    return int(lib().dp_model_nparams(ctypes.byref(c)))


def _box9(box):
    b = np.asarray(box, dtype=np.float64)
    if b.shape == (3,):
        b = np.diag(b)
    b = np.ascontiguousarray(b.reshape(9), dtype=np.float64)
    return b


def _dev(t, dtype, shape=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _seed_gains(desc, fit_in_gain, out_scale):
    g = float(desc.get("fit_in_gain", 300.0) if fit_in_gain is None else fit_in_gain)
    o = float(desc.get("out_scale", 0.02) if out_scale is None else out_scale)
    return g, o


def dp_model_params_from_seed(desc, seed, fit_in_gain=None, out_scale=None):
    """Seeded flat parameter vector (host float64 numpy) of dp_model_params_from_seed."""
    g, o = _seed_gains(desc, fit_in_gain, out_scale)
    c = make_desc(desc)
    n = dp_model_nparams(c)
    if n < 0:
        raise DPError(DP_ERR_ARG, "invalid descriptor")
    P = np.empty(n, dtype=np.float64)
    _check(lib().dp_model_params_from_seed(ctypes.byref(c), int(seed), g, o, P.ctypes.data_as(_vp), n))
    return P


class Model:
    """dp_model handle (parameters live on the current CUDA device)."""

    def __init__(self, desc=None, params=None, _handle=None):
        self._h = _vp()
        if _handle is not None:
            self._h = _handle
        else:
            self.desc_c = make_desc(desc)
            p = np.ascontiguousarray(params, dtype=np.float64)
            _check(lib().dp_model_create(ctypes.byref(self.desc_c), p.ctypes.data_as(_vp), len(p),
                                         ctypes.byref(self._h)))
        self.desc = desc

    @classmethod
    def from_seed(cls, desc, seed, fit_in_gain=None, out_scale=None):
        """dp_model_from_seed; the gains default to desc's own (as synth.model_params)."""
        g, o = _seed_gains(desc, fit_in_gain, out_scale)
        c = make_desc(desc)
        h = _vp()
        _check(lib().dp_model_from_seed(ctypes.byref(c), int(seed), g, o, ctypes.byref(h)))
        m = cls(desc=desc, _handle=h)
        m.desc_c = c
        return m

    @classmethod
    def load(cls, path, desc=None):
        h = _vp()
        _check(lib().dp_model_load(os.fsencode(path), ctypes.byref(h)))
        return cls(desc=desc, _handle=h)

    def save(self, path):
        _check(lib().dp_model_save(self._h, os.fsencode(path)))

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        _check(lib().dp_model_set_params(self._h, p.ctypes.data_as(_vp), len(p)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().dp_model_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """dp_ctx handle: scratch memory and stream for one system size."""

    def __init__(self, model, natoms_max, cand_cap=0, precision=DP_PREC_FP64, stream=None):
        self.model = model
        self.natoms_max = int(natoms_max)
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        self._h = _vp()
        _check(lib().dp_ctx_create(model.handle, self.natoms_max, int(cand_cap), int(precision),
                                   ctypes.c_void_p(st.cuda_stream), ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def set_sync(self, sync):
        _check(lib().dp_ctx_set_sync(self._h, int(bool(sync))))

    def status(self):
        return lib().dp_ctx_status(self._h)

    @property
    def launches(self):
        return int(lib().dp_ctx_launches(self._h))

    def set_embed_store(self, on):
        """dp_ctx_set_embed_store: keep G and dG/ds of every row between the
        forward and the backward (on) or recompute them (off)."""
        _check(lib().dp_ctx_set_embed_store(self._h, int(bool(on))))

    @property
    def embed_store(self):
        return bool(lib().dp_ctx_embed_store(self._h) == 1)

    def set_timing(self, on):
        _check(lib().dp_ctx_set_timing(self._h, int(bool(on))))

    def kernel_times(self):
        """{group name: (milliseconds, launches)} accumulated while timing was on."""
        ms = np.zeros(8, dtype=np.float64)
        n = np.zeros(8, dtype=np.int64)
        _check(lib().dp_ctx_kernel_times(self._h, ms.ctypes.data_as(_vp), n.ctypes.data_as(_vp)))
        return {lib().dp_kernel_group_name(g).decode(): (float(ms[g]), int(n[g])) for g in range(8)}

    def close(self):
        if self._h:
            lib().dp_ctx_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ C-ABI names --

def dp_build_nlist(ctx, coords, types, box, skin=0.0, check=True):
    N = coords.shape[0]
    b = _box9(box)
    s = lib().dp_build_nlist(ctx.handle, _dev(coords, torch.float64, (N, 3), "coords"),
                             _dev(types, torch.int32, (N,), "types"), b.ctypes.data_as(_vp), N, float(skin))
    return _check(s) if check else s


def dp_format_nlist(ctx, coords, types, box, check=True):
    """Returns (nlist [N, N_m] int32, nreal [N, ntypes] int32, status)."""
    N = coords.shape[0]
    d = ctx.model.desc
    nm = int(sum(d["sel"]))
    nlist = torch.empty((N, nm), dtype=torch.int32, device=coords.device)
    nreal = torch.empty((N, d["ntypes"]), dtype=torch.int32, device=coords.device)
    b = _box9(box)
    s = lib().dp_format_nlist(ctx.handle, _dev(coords, torch.float64, (N, 3), "coords"),
                              _dev(types, torch.int32, (N,), "types"), b.ctypes.data_as(_vp), N,
                              _dev(nlist, torch.int32), _dev(nreal, torch.int32))
    if check:
        _check(s)
    return nlist, nreal, s


def dp_param_grad(ctx, coords, types, box, cE, lam, grad=None):
    """d/dW of cE * E + sum_i lam_i . F_i (device tensor [nparams])."""
    N = coords.shape[0]
    if grad is None:
        grad = torch.empty(dp_model_nparams(ctx.model.desc), dtype=torch.float64, device=coords.device)
    b = _box9(box)
    lam = lam.contiguous()
    _check(lib().dp_param_grad(ctx.handle, _dev(coords, torch.float64, (N, 3), "coords"),
                               _dev(types, torch.int32, (N,), "types"), b.ctypes.data_as(_vp), N, float(cE),
                               _dev(lam, torch.float64, (N, 3), "lambda"), _dev(grad, torch.float64, None, "grad")))
    return grad


def dp_tanh_f64(x, stream=None):
    """The library's FP64 tanh (used by the FP64 kernels) on a CUDA tensor."""
    y = torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().dp_tanh_f64(_dev(x, torch.float64), _dev(y, torch.float64), x.numel(),
                             ctypes.c_void_p(st.cuda_stream)))
    return y


def dp_format_nlist_noalloc(desc, coords, types, box, skin=0.0, nlist=None, nreal=None, stream=None,
                            check=True):
    """Algorithm 1 with no device allocation inside the library (see
    include/dp.h); returns (nlist [N, N_m], nreal [N, ntypes], status).  The
    output tensors are the caller's (allocated here only when not given)."""
    N = coords.shape[0]
    c = make_desc(desc)
    nm = int(sum(desc["sel"]))
    if nlist is None:
        nlist = torch.empty((N, nm), dtype=torch.int32, device=coords.device)
    if nreal is None:
        nreal = torch.empty((N, desc["ntypes"]), dtype=torch.int32, device=coords.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    b = _box9(box)
    s = lib().dp_format_nlist_noalloc(ctypes.byref(c), _dev(coords, torch.float64, (N, 3), "coords"),
                                      _dev(types, torch.int32, (N,), "types"), b.ctypes.data_as(_vp), N,
                                      float(skin), _dev(nlist, torch.int32, (N, nm), "nlist"),
                                      _dev(nreal, torch.int32, (N, desc["ntypes"]), "nreal"),
                                      ctypes.c_void_p(st.cuda_stream))
    if check:
        _check(s)
    return nlist, nreal, s


def dp_eval(ctx, coords, types, box, energy=None, force=None, virial=None, atom_energy=None,
            want_atom_energy=False, check=True):
    """Energy, forces and virial; returns dict of device tensors and the status."""
    N = coords.shape[0]
    dev = coords.device
    if energy is None:
        energy = torch.empty(1, dtype=torch.float64, device=dev)
    if force is None:
        force = torch.empty((N, 3), dtype=torch.float64, device=dev)
    if virial is None:
        virial = torch.empty(9, dtype=torch.float64, device=dev)
    if atom_energy is None and want_atom_energy:
        atom_energy = torch.empty(N, dtype=torch.float64, device=dev)
    b = _box9(box)
    s = lib().dp_eval(ctx.handle, _dev(coords, torch.float64, (N, 3), "coords"),
                      _dev(types, torch.int32, (N,), "types"), b.ctypes.data_as(_vp), N,
                      _dev(energy, torch.float64, (1,), "energy"), _dev(force, torch.float64, (N, 3), "force"),
                      _dev(virial, torch.float64, (9,), "virial"),
                      _dev(atom_energy, torch.float64, (N,), "atom_energy") if atom_energy is not None else None)
    if check:
        _check(s)
    return dict(energy=energy, force=force, virial=virial, atom_energy=atom_energy, status=s)


def dp_eval_local(ctx, coords, types, box, nloc, energy=None, force=None, virial=None, atom_energy=None,
                  check=True):
    """Sub-region evaluation: atoms [0, nloc) are centres, [nloc, N) ghosts.
    Returns dict(energy [1], force [N, 3], virial [9], atom_energy, status)."""
    N = coords.shape[0]
    dev = coords.device
    if energy is None:
        energy = torch.empty(1, dtype=torch.float64, device=dev)
    if force is None:
        force = torch.empty((N, 3), dtype=torch.float64, device=dev)
    if virial is None:
        virial = torch.empty(9, dtype=torch.float64, device=dev)
    b = _box9(box)
    s = lib().dp_eval_local(ctx.handle, _dev(coords, torch.float64, (N, 3), "coords"),
                            _dev(types, torch.int32, (N,), "types"), b.ctypes.data_as(_vp), N, int(nloc),
                            _dev(energy, torch.float64, (1,), "energy"), _dev(force, torch.float64, (N, 3), "force"),
                            _dev(virial, torch.float64, (9,), "virial"),
                            _dev(atom_energy, torch.float64, (int(nloc),), "atom_energy")
                            if atom_energy is not None else None)
    if check:
        _check(s)
    return dict(energy=energy, force=force, virial=virial, atom_energy=atom_energy, status=s)


def dp_md_step(ctx, coords, vel, types, box, masses, dt, nsteps, rebuild_every=10, skin=2.0,
               thermo=None, check=True):
    """Advance coords/vel in place; returns (thermo [nsteps, 4] device tensor or None, status)."""
    N = coords.shape[0]
    m = np.ascontiguousarray(masses, dtype=np.float64)
    b = _box9(box)
    s = lib().dp_md_step(ctx.handle, _dev(coords, torch.float64, (N, 3), "coords"),
                         _dev(vel, torch.float64, (N, 3), "vel"), _dev(types, torch.int32, (N,), "types"),
                         b.ctypes.data_as(_vp), m.ctypes.data_as(_vp), N, float(dt), int(nsteps),
                         int(rebuild_every), float(skin),
                         _dev(thermo, torch.float64, (nsteps, 4), "thermo") if thermo is not None else None)
    if check:
        _check(s)
    return thermo, s


def dp_md_kick_drift(ctx, coords, vel, force, types, box, masses, dt):
    """First half of a velocity-Verlet step: v += F/m dt/2, x += v dt, and
    x wrapped into the cell (box None: no wrapping)."""
    N = coords.shape[0]
    b = _box9(box) if box is not None else None
    m = np.ascontiguousarray(masses, dtype=np.float64)
    _check(lib().dp_md_kick_drift(ctx.handle, _dev(coords, torch.float64, (N, 3), "coords"),
                                  _dev(vel, torch.float64, (N, 3), "vel"), _dev(force, torch.float64, (N, 3), "force"),
                                  _dev(types, torch.int32, (N,), "types"),
                                  b.ctypes.data_as(_vp) if b is not None else None,
                                  m.ctypes.data_as(_vp), N, float(dt)))


def dp_md_kick(ctx, vel, force, types, masses, dt):
    """Second half of a velocity-Verlet step: v += F/m dt/2."""
    N = vel.shape[0]
    m = np.ascontiguousarray(masses, dtype=np.float64)
    _check(lib().dp_md_kick(ctx.handle, _dev(vel, torch.float64, (N, 3), "vel"),
                            _dev(force, torch.float64, (N, 3), "force"), _dev(types, torch.int32, (N,), "types"),
                            m.ctypes.data_as(_vp), N, float(dt)))


def dp_md_get_force(ctx, N, device="cuda"):
    f = torch.empty((N, 3), dtype=torch.float64, device=device)
    _check(lib().dp_md_get_force(ctx.handle, _dev(f, torch.float64), N))
    return f


def dp_md_reset(ctx):
    _check(lib().dp_md_reset(ctx.handle))


class DPEnergyForces(torch.autograd.Function):
    """(E, F, virial) of a model as a differentiable function of its flat
    parameter vector.  Forward: dp_eval.  Backward: dp_param_grad with
    cE = dL/dE and lambda = dL/dF, so any loss on the energy and forces
    trains the model through the hand-written kernels.  A gradient flowing
    into the virial output is not supported (raises).

    Usage:  E, F, V = DPEnergyForces.apply(params, coords, types, box, ctx)
    where params is a float64 tensor (any device) of dp_model_nparams values
    and ctx a FP64 Context of the model whose parameters are trained."""

    @staticmethod
    def forward(fctx, params, coords, types, box, dpctx):
        dpctx.model.set_params(params.detach().to("cpu", torch.float64).numpy())
        out = dp_eval(dpctx, coords, types, box)
        fctx.dpctx = dpctx
        fctx.box = box
        fctx.save_for_backward(coords, types)
        fctx.params_device = params.device
        return out["energy"].clone(), out["force"].clone(), out["virial"].clone()

    @staticmethod
    def backward(fctx, gE, gF, gV):
        coords, types = fctx.saved_tensors
        if gV is not None and bool(torch.any(gV != 0)):
            raise NotImplementedError("gradients through the virial are not supported")
        cE = float(gE.sum().item()) if gE is not None else 0.0
        lam = gF.contiguous().to(torch.float64) if gF is not None else torch.zeros_like(coords)
        grad = dp_param_grad(fctx.dpctx, coords, types, fctx.box, cE, lam)
        return grad.to(fctx.params_device), None, None, None, None

"""Seeded synthetic inputs: systems, model weights, initial velocities.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It holds no arithmetic of the Deep Potential method itself: it
draws random numbers and places atoms.  Everything it returns is plain numpy
data (float64 / int32) that both sides receive as inputs.

Workloads follow the paper's benchmark systems (Sec. 4): liquid water made of
rigid H2O molecules and FCC copper with lattice constant 3.634 A.  No
equilibrated configuration or trained model is available, so:

* water: molecules on a simple-cubic lattice (spacing L/n), the O atom jittered
  uniformly by +-0.2 A per axis, the molecule rigid (O-H 0.96 A, H-O-H 104.5
  deg) with a uniformly random orientation (unit quaternion from 4 normals);
  atoms ordered O,H,H per molecule, types O=0, H=1;
* copper: FCC cells with Gaussian jitter of 1% of the lattice constant;
* weights: every linear layer W ~ N(0, 1/(fan_in+fan_out)), b ~ N(0, 1), drawn
  from one seeded splitmix64 / Box-Muller stream; the first fitting layer is
  multiplied by a gain, the output layer by a scale (zero bias), both per model;
* velocities: Maxwell-Boltzmann at T0, centre-of-mass momentum removed, then
  rescaled to exactly T0 with 3N-3 degrees of freedom.

Model parameter layout (flat float64 vector, the one format both sides read):

  embedding nets, for centre type a = 0..T-1, for neighbour type b = 0..T-1:
      layer 0 : W0[e1], b0[e1]
      layer l : W[e_l][e_{l+1}] (row-major, input index first), b[e_{l+1}]
  fitting nets, for centre type a = 0..T-1:
      layer 1 : W[M2*M][f1], b[f1]
      layer l : W[f_{l-1}][f_l], b[f_l]
      output  : w[f_last], b_out[1]
"""
from __future__ import annotations

import math

import numpy as np

# Physical constants for the velocity draw (units: A, fs, eV, amu, K).
KB_EV = 8.617333262e-5            # Boltzmann constant, eV/K
ACC_CONV = 9.648533212e-3         # (eV/A/amu) -> A/fs^2
MASS = {"O": 15.999, "H": 1.008, "Cu": 63.546}

# ---------------------------------------------------------------- models ----

# fit_in_gain / out_scale: the seeded weights' first-fitting-layer gain and
# output scale (model_params).  Water: RMS force ~4e-3 eV/A at the start; the
# random landscape has no repulsion, and at this scale a 300 K NVE run of the
# water boxes reaches ~320 K and RMS forces of ~1.4e-2 eV/A (largest ~0.4 eV/A)
# after 100 steps of 0.5 fs, while twice the scale gives ~350 K and ~4e-2
# (largest ~1.4 eV/A, close contacts).  Copper: RMS force ~7e-3 eV/A (the
# nearly symmetric FCC environments cancel most of an atom's force, so its
# output scale is larger).
WATER_MODEL = dict(ntypes=2, sel=(46, 92), rcut=6.0, rcut_smth=0.5,
                   emb=(25, 50, 100), m2=16, fit=(240, 240, 240),
                   desc_scale_nm=1, fit_in_gain=300.0, out_scale=0.02)
CU_MODEL = dict(ntypes=1, sel=(512,), rcut=8.0, rcut_smth=2.0,
                emb=(32, 64, 128), m2=16, fit=(240, 240, 240),
                desc_scale_nm=1, fit_in_gain=300.0, out_scale=8.0)
WATER_STUDENT = dict(WATER_MODEL, emb=(16, 32, 64))


def layer_shapes(desc):
    """List of (name, shape) in the flat parameter order documented above."""
    T = desc["ntypes"]
    emb = list(desc["emb"])
    fit = list(desc["fit"])
    M = emb[-1]
    out = []
    for a in range(T):
        for b in range(T):
            out.append((f"emb{a}{b}.W0", (emb[0],)))
            out.append((f"emb{a}{b}.b0", (emb[0],)))
            for l in range(1, len(emb)):
                out.append((f"emb{a}{b}.W{l}", (emb[l - 1], emb[l])))
                out.append((f"emb{a}{b}.b{l}", (emb[l],)))
    for a in range(T):
        prev = desc["m2"] * M
        for l, f in enumerate(fit):
            out.append((f"fit{a}.W{l + 1}", (prev, f)))
            out.append((f"fit{a}.b{l + 1}", (f,)))
            prev = f
        out.append((f"fit{a}.wo", (prev,)))
        out.append((f"fit{a}.bo", (1,)))
    return out


def n_params(desc):
    return int(sum(int(np.prod(s)) for _, s in layer_shapes(desc)))


_SM64_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SM64_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM64_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, i):
    """Outputs i (uint64 array, i >= 1) of splitmix64 seeded with `seed`
    (Steele, Lea and Flood, 2014): mix(seed + i * gamma), arithmetic mod 2^64."""
    z = np.uint64(seed) + np.asarray(i, dtype=np.uint64) * _SM64_GAMMA
    z = (z ^ (z >> np.uint64(30))) * _SM64_M1
    z = (z ^ (z >> np.uint64(27))) * _SM64_M2
    return z ^ (z >> np.uint64(31))


def seeded_normals(seed, n):
    """The first n standard normals of the seeded stream: outputs (2p+1, 2p+2)
    of splitmix64 give u1 = ((z >> 11) + 1) 2^-53 in (0, 1] and
    u2 = (z >> 11) 2^-53 in [0, 1); Box-Muller gives normal 2p =
    sqrt(-2 ln u1) cos(2 pi u2) and normal 2p+1 = sqrt(-2 ln u1) sin(2 pi u2).
    The transcendental functions are the C library's (math module), element by
    element, so that the values equal those of a C implementation using the
    same libm bit for bit."""
    npair = (int(n) + 1) // 2
    with np.errstate(over="ignore"):
        z = splitmix64(seed, np.arange(1, 2 * npair + 1, dtype=np.uint64))
    u1 = ((z[0::2] >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    out = np.empty(2 * npair)
    two_pi = 6.283185307179586
    log, sqrt, cos, sin = math.log, math.sqrt, math.cos, math.sin
    for p, (a, b) in enumerate(zip(u1.tolist(), u2.tolist())):
        r = sqrt(-2.0 * log(a))
        th = two_pi * b
        out[2 * p] = r * cos(th)
        out[2 * p + 1] = r * sin(th)
    return out[:n]


def model_params(desc, seed=0, fit_in_gain=None, out_scale=None):
    """Seeded weights in the flat layout.  No trained model exists; these
    stand in for one (same architecture as the paper's models, Sec. 4).

    Element k of the flat vector is scale_k * n_k with n_k the k-th normal of
    ``seeded_normals(seed, .)`` (the generator of the C ABI's
    dp_model_params_from_seed, value for value): weight matrices
    n / sqrt(fan_in + fan_out), the first fitting layer's then times
    ``fit_in_gain``; hidden biases n; output weights
    (out_scale * n) / sqrt(f_last + 1); output bias 0.

    The gains default to the model's own (``desc["fit_in_gain"]``,
    ``desc["out_scale"]``).  The first fitting layer's gain brings its
    pre-activations to O(1) (with the 1/N_m scale the descriptor entries are
    ~1e-3).  The output scale sets the force scale (RMS forces of ~4e-3 eV/A
    on the water boxes, ~7e-3 on copper).  The random landscape has no
    physical repulsion and slowly draws atoms together, so much larger forces
    heat an NVE run quickly."""
    if fit_in_gain is None:
        fit_in_gain = desc.get("fit_in_gain", 300.0)
    if out_scale is None:
        out_scale = desc.get("out_scale", 0.02)
    shapes = layer_shapes(desc)
    n = sum(int(np.prod(s)) for _, s in shapes)
    z = seeded_normals(seed, n)
    P = np.empty(n)
    k = 0
    for name, shape in shapes:
        m = int(np.prod(shape))
        kind = name.split(".")[1]
        seg = z[k:k + m]
        if kind == "wo":
            P[k:k + m] = (out_scale * seg) / math.sqrt(shape[0] + 1)
        elif kind == "bo":
            P[k:k + m] = 0.0
        elif kind.startswith("W"):
            fan_in = shape[0] if len(shape) == 2 else 1
            w = seg / math.sqrt(fan_in + shape[-1])
            if name.startswith("fit") and kind == "W1" and fit_in_gain != 1.0:
                w = w * fit_in_gain
            P[k:k + m] = w
        else:
            P[k:k + m] = seg
        k += m
    return np.ascontiguousarray(P, dtype=np.float64)


# --------------------------------------------------------------- systems ----

def _random_rotations(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water_box(n_side, L, seed=1, nmol=None, jitter=0.2, roh=0.96, angle_deg=104.5):
    """Rigid water molecules on an n_side^3 lattice in a cubic box of edge L.

    With ``nmol`` < n_side^3 the first ``nmol`` sites of a seeded random
    permutation are used (the 131,072-molecule box on 51^3 sites).
    Returns (coords [N,3] float64, types [N] int32, box [3] float64)."""
    rng = np.random.default_rng(seed)
    g = np.arange(n_side)
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    if nmol is None:
        nmol = n_side ** 3
    else:
        sites = sites[rng.permutation(len(sites))[:nmol]]
    spacing = L / n_side
    O = (sites + 0.5) * spacing + rng.uniform(-jitter, jitter, size=(nmol, 3))
    half = np.deg2rad(angle_deg) / 2
    body = np.array([[roh * np.sin(half), 0.0, roh * np.cos(half)],
                     [-roh * np.sin(half), 0.0, roh * np.cos(half)]])
    R = _random_rotations(rng, nmol)
    H = O[:, None, :] + np.einsum("nij,kj->nki", R, body)
    coords = np.concatenate([O[:, None, :], H], axis=1).reshape(-1, 3)
    coords = np.mod(coords, L)
    types = np.tile(np.array([0, 1, 1], dtype=np.int32), nmol)
    return np.ascontiguousarray(coords), types, np.array([L, L, L], dtype=np.float64)


def copper_fcc(n_cell, a=3.634, seed=1, jitter_frac=0.01):
    """FCC copper, n_cell^3 cells of edge a, Gaussian jitter of jitter_frac*a."""
    rng = np.random.default_rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
    g = np.arange(n_cell)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 1, 3).astype(np.float64)
    coords = ((cells + basis[None]) * a).reshape(-1, 3)
    coords = coords + rng.normal(0.0, jitter_frac * a, size=coords.shape)
    L = n_cell * a
    coords = np.mod(coords, L)
    types = np.zeros(len(coords), dtype=np.int32)
    return np.ascontiguousarray(coords), types, np.array([L, L, L], dtype=np.float64)


def maxwell_velocities(masses, T0, seed=2):
    """Velocities (A/fs) at exactly T0 (3N-3 degrees of freedom)."""
    rng = np.random.default_rng(seed)
    m = np.asarray(masses, dtype=np.float64)
    sigma = np.sqrt(KB_EV * T0 / m * ACC_CONV)
    v = rng.standard_normal((len(m), 3)) * sigma[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    ke = 0.5 * (m[:, None] * v * v).sum() / ACC_CONV
    dof = 3 * len(m) - 3
    v *= np.sqrt(T0 * dof * KB_EV / (2.0 * ke))
    return np.ascontiguousarray(v)


# --------------------------------------------------------- named workloads --

def workload(name, seed_geom=1):
    """Named synthetic systems with the sizes of the paper's benchmarks.

    water192   : 64 H2O, L = 12.42 A
    water12288 : 4,096 H2O, L = 49.7 A
    cu32000    : 20^3 FCC cells, a = 3.634 A
    water393216: 131,072 H2O on 51^3 sites, L = 157.6 A
    Returns dict(coords, types, box, model, masses_per_type)."""
    if name == "water192":
        c, t, b = water_box(4, 12.42, seed_geom)
        return dict(coords=c, types=t, box=b, model=WATER_MODEL, masses=(MASS["O"], MASS["H"]))
    if name == "water12288":
        c, t, b = water_box(16, 49.7, seed_geom)
        return dict(coords=c, types=t, box=b, model=WATER_MODEL, masses=(MASS["O"], MASS["H"]))
    if name == "cu32000":
        c, t, b = copper_fcc(20, 3.634, seed_geom)
        return dict(coords=c, types=t, box=b, model=CU_MODEL, masses=(MASS["Cu"],))
    if name == "water393216":
        c, t, b = water_box(51, 157.6, seed_geom, nmol=131072)
        return dict(coords=c, types=t, box=b, model=WATER_MODEL, masses=(MASS["O"], MASS["H"]))
    raise KeyError(name)


def sub_box_water(n_side, L, seed=1):
    """A smaller water box at the same density (for multi-tile parity cases)."""
    c, t, b = water_box(n_side, L, seed)
    return dict(coords=c, types=t, box=b, model=WATER_MODEL, masses=(MASS["O"], MASS["H"]))

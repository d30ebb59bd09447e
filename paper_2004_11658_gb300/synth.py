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
* weights: every linear layer W ~ N(0, 1/(fan_in+fan_out)), b ~ N(0, 1); the
  first fitting layer is multiplied by 300, the output layer by 0.02 (zero bias);
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

import numpy as np

# Physical constants for the velocity draw (units: A, fs, eV, amu, K).
KB_EV = 8.617333262e-5            # Boltzmann constant, eV/K
ACC_CONV = 9.648533212e-3         # (eV/A/amu) -> A/fs^2
MASS = {"O": 15.999, "H": 1.008, "Cu": 63.546}

# ---------------------------------------------------------------- models ----

WATER_MODEL = dict(ntypes=2, sel=(46, 92), rcut=6.0, rcut_smth=0.5,
                   emb=(25, 50, 100), m2=16, fit=(240, 240, 240),
                   desc_scale_nm=1)
CU_MODEL = dict(ntypes=1, sel=(512,), rcut=8.0, rcut_smth=2.0,
                emb=(32, 64, 128), m2=16, fit=(240, 240, 240),
                desc_scale_nm=1)
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


def model_params(desc, seed=0, fit_in_gain=300.0, out_scale=0.02):
    """Seeded weights in the flat layout.  No trained model exists; these
    stand in for one (same architecture as the paper's models, Sec. 4).

    The first fitting layer is multiplied by ``fit_in_gain``: with the 1/N_m
    descriptor scale the descriptor entries are ~1e-3, and the gain brings
    that layer's pre-activations to O(1).  The output layer is scaled by
    ``out_scale`` (0.02), which gives RMS forces of ~0.01 eV/A on the water
    boxes.  The random landscape has no physical repulsion and slowly draws
    atoms together; at this scale a 300 K NVE run of the 12,288-atom box
    stays below ~330 K and within sel for 300 steps of 0.5 fs, while 5x
    larger forces heat it past 700 K and overflow sel in ~230 steps."""

    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in layer_shapes(desc):
        kind = name.split(".")[1]
        if kind.startswith("W"):
            fan_in = shape[0] if len(shape) == 2 else 1
            fan_out = shape[-1]
            w = rng.standard_normal(shape).ravel() / np.sqrt(fan_in + fan_out)
            if name.startswith("fit") and kind == "W1":
                w = w * fit_in_gain
            parts.append(w)
        elif kind == "wo":
            parts.append(out_scale * rng.standard_normal(shape) / np.sqrt(shape[0] + 1))
        elif kind == "bo":
            parts.append(np.zeros(shape))
        else:
            parts.append(rng.standard_normal(shape))
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float64)


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

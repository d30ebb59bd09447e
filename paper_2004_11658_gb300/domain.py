"""Spatial domain decomposition of the evaluation (Sec. 3.1, Remark 4).

The periodic orthorhombic cell is cut into P slabs along x; slab p owns the
atoms with p L/P <= x < (p+1) L/P.  Every slab also holds ghost atoms: the
copies (periodic images included) of other atoms within the ghost width w of
its faces (w >= rcut).  One evaluation then takes four steps:

1. forward halo: every owner sends the current positions of the atoms other
   slabs hold as ghosts (shifted by the periodic image they stand for);
2. sub-region evaluation (dp_eval_local): energies of the owned atoms, their
   force increments on owned and ghost atoms, and their virial;
3. reverse halo: the force increments on ghosts go back to the owners, which
   add them (the j-side terms of Remark 4 have no Newton-3 shortcut);
4. the energy and the virial are summed over the slabs (an all-reduce).

A slab is evaluated in its own frame: x is shifted so that the slab with its
ghost shells starts at 0, and the cell edge along x is padded to
slab + 2 w + pad with pad >= rcut + skin, so that no atom meets an image of
another through the padded edge.  The edges along y and z stay periodic.

Two drivers share the plan: `evaluate_emulated` runs all slabs one after
another in one process (all sub-region evaluations on one device, halos by
index), and `DistributedSlab` runs one slab per process with
torch.distributed point-to-point messages and an all-reduce.  The plan is made
from the positions at decomposition time (every rank makes the same plan);
between decompositions atoms may move by up to (w - rcut) / 2 before the
ghost lists are stale, as with the Verlet skin.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch


def _box3(box):
    b = np.asarray(box, dtype=np.float64)
    if b.size == 9:
        b9 = b.reshape(3, 3)
        if np.any(b9 - np.diag(np.diag(b9))):
            raise ValueError("only orthorhombic cells are supported")
        b = np.diag(b9)
    return b.astype(np.float64).copy()


@dataclass
class SlabPlan:
    """Ownership and halo lists of a P-slab decomposition.

    For slab p:
      owned[p]           global indices of the owned atoms (ascending);
      ghost_src[p]       owning slab of each ghost;
      ghost_pos[p]       position of the ghost's atom in the owner's owned list;
      ghost_shift[p]     periodic image along x (-1, 0, +1) the ghost stands for;
    and for every ordered pair (p -> q): send[p][q] = (owner positions, shifts)
    of the atoms that slab q holds as ghosts from p, in q's ghost order.
    """
    nslab: int
    box: np.ndarray
    ghost_width: float
    pad: float
    owned: list = field(default_factory=list)
    ghost_src: list = field(default_factory=list)
    ghost_pos: list = field(default_factory=list)
    ghost_shift: list = field(default_factory=list)
    send: list = field(default_factory=list)

    def slab_lo(self, p):
        return p * self.box[0] / self.nslab

    def origin(self, p):
        """x of the sub-region frame's origin (slab start minus the ghost width)."""
        return self.slab_lo(p) - self.ghost_width

    def sub_box(self):
        """Cell of every sub-region: x padded, y and z periodic as the cell."""
        w = self.box[0] / self.nslab
        return np.array([w + 2.0 * self.ghost_width + self.pad, self.box[1], self.box[2]])


def make_plan(coords, box, nslab, ghost_width, pad):
    """Slab decomposition of the positions `coords` [N, 3] (host array)."""
    x = np.asarray(coords, dtype=np.float64)
    L = _box3(box)
    N = len(x)
    if nslab < 1:
        raise ValueError("nslab must be >= 1")
    width = L[0] / nslab
    if ghost_width > width * nslab:
        raise ValueError("ghost width larger than the cell")
    xw = x[:, 0] - L[0] * np.floor(x[:, 0] / L[0])
    owner = np.minimum((xw / width).astype(np.int64), nslab - 1)
    plan = SlabPlan(nslab=nslab, box=L, ghost_width=float(ghost_width), pad=float(pad))
    pos_in_owner = np.empty(N, dtype=np.int64)
    for p in range(nslab):
        own = np.nonzero(owner == p)[0]
        plan.owned.append(own)
        pos_in_owner[own] = np.arange(len(own))
    for q in range(nslab):
        lo = q * width - ghost_width
        hi = (q + 1) * width + ghost_width
        src, pos, shift = [], [], []
        for s in (-1, 0, 1):
            xs = xw + s * L[0]
            inside = (xs >= lo) & (xs < hi)
            if s == 0:
                inside &= owner != q
            idx = np.nonzero(inside)[0]
            src.append(owner[idx])
            pos.append(pos_in_owner[idx])
            shift.append(np.full(len(idx), s, dtype=np.int64))
        src = np.concatenate(src)
        pos = np.concatenate(pos)
        shift = np.concatenate(shift)
        # ghosts grouped by owning slab (stable within a group)
        order = np.argsort(src, kind="stable")
        plan.ghost_src.append(src[order])
        plan.ghost_pos.append(pos[order])
        plan.ghost_shift.append(shift[order])
    for p in range(nslab):
        row = []
        for q in range(nslab):
            sel = plan.ghost_src[q] == p
            row.append((plan.ghost_pos[q][sel], plan.ghost_shift[q][sel]))
        plan.send.append(row)
    return plan


def _pack_positions(plan, p, q, x_owned):
    """Forward-halo message p -> q: positions of q's ghosts owned by p, in
    q's frame."""
    pos, shift = plan.send[p][q]
    idx = torch.as_tensor(pos, device=x_owned.device)
    out = x_owned.index_select(0, idx).clone()
    out[:, 0] += torch.as_tensor(shift, dtype=out.dtype, device=out.device) * plan.box[0]
    return out


def _ghost_ranges(plan, q):
    """Slices of q's ghost list per owning slab."""
    counts = np.bincount(plan.ghost_src[q], minlength=plan.nslab)
    starts = np.concatenate([[0], np.cumsum(counts)])
    return [(int(starts[p]), int(starts[p + 1])) for p in range(plan.nslab)]


def _sub_region_coords(plan, q, x_owned, ghosts):
    """Owned then ghost positions, shifted into q's frame."""
    xs = torch.cat([x_owned, ghosts], 0) if ghosts.numel() else x_owned.clone()
    xs[:, 0] -= plan.origin(q)
    return xs.contiguous()


def evaluate_emulated(plan, coords, types, evaluate_local):
    """All slabs one after another in this process.

    coords: [N, 3] float64 tensor (global order), types: [N] int32 tensor;
    evaluate_local(x_sub, t_sub, sub_box, nloc) -> (E (float), F [n, 3]
    tensor, virial [3, 3] or [9] tensor) evaluates one sub-region.
    Returns (E, F [N, 3], virial [3, 3]) of the whole system, assembled from
    the sub-regions through the halo lists only."""
    P = plan.nslab
    dev = coords.device
    x_owned = [coords.index_select(0, torch.as_tensor(plan.owned[p], device=dev)) for p in range(P)]
    t_owned = [types.index_select(0, torch.as_tensor(plan.owned[p], device=dev)) for p in range(P)]
    # forward halo
    inbox = [[_pack_positions(plan, p, q, x_owned[p]) for p in range(P)] for q in range(P)]
    E = 0.0
    V = torch.zeros(9, dtype=torch.float64, device=dev)
    f_owned = [None] * P
    back = [[None] * P for _ in range(P)]   # back[q][p]: increments q computed on p's atoms
    for q in range(P):
        ghosts = torch.cat(inbox[q], 0)
        t_ghost = torch.cat([t_owned[p].index_select(0, torch.as_tensor(plan.send[p][q][0], device=dev))
                             for p in range(P)], 0)
        xs = _sub_region_coords(plan, q, x_owned[q], ghosts)
        ts = torch.cat([t_owned[q], t_ghost], 0).contiguous()
        nloc = len(plan.owned[q])
        e, f, v = evaluate_local(xs, ts, plan.sub_box(), nloc)
        E += float(e)
        V += torch.as_tensor(v, dtype=torch.float64, device=dev).reshape(9)
        f_owned[q] = f[:nloc].clone()
        for p, (a, b) in enumerate(_ghost_ranges(plan, q)):
            back[q][p] = f[nloc + a: nloc + b]
    # reverse halo: owners add the increments computed on their ghosts
    for p in range(P):
        for q in range(P):
            pos = plan.send[p][q][0]
            if len(pos):
                f_owned[p].index_add_(0, torch.as_tensor(pos, device=dev), back[q][p])
    F = torch.empty_like(coords)
    for p in range(P):
        F.index_copy_(0, torch.as_tensor(plan.owned[p], device=dev), f_owned[p])
    return E, F, V.reshape(3, 3)


class DistributedSlab:
    """One slab per process (torch.distributed; rank = slab).

    forces(x_owned) runs the four steps of one evaluation with point-to-point
    messages to the other ranks (a slab exchanges with its two neighbours,
    and with more when the ghost width exceeds a slab) and one all-reduce of
    the energy and virial."""

    def __init__(self, plan, rank, types_owned, evaluate_local, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.plan = plan
        self.rank = rank
        self.group = group
        self.t_owned = types_owned
        self.evaluate_local = evaluate_local
        self.ranges = _ghost_ranges(plan, rank)
        self.t_ghost = None   # ghost types arrive once, by the same route as positions
        self.nloc = len(plan.owned[rank])
        self.peers = [p for p in range(plan.nslab) if p != rank]

    def _exchange(self, send, recv_shapes, dtype):
        """send[q] -> rank q, receive from every peer into buffers of recv_shapes[p]."""
        dist = self.dist
        dev = next(iter(send.values())).device if send else torch.device("cpu")
        recv = {p: torch.empty(recv_shapes[p], dtype=dtype, device=dev) for p in self.peers}
        ops = []
        for q in self.peers:
            if send[q].shape[0]:
                ops.append(dist.P2POp(dist.isend, send[q].contiguous(), q, self.group))
        for p in self.peers:
            if recv[p].shape[0]:
                ops.append(dist.P2POp(dist.irecv, recv[p], p, self.group))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        return recv

    def _own_ghosts(self, x_owned):
        """Ghosts this rank holds of its own atoms (periodic images when the
        ghost shell wraps onto its own slab)."""
        return _pack_positions(self.plan, self.rank, self.rank, x_owned)

    def forces(self, x_owned):
        plan, me = self.plan, self.rank
        dev = x_owned.device
        send = {q: _pack_positions(plan, me, q, x_owned) for q in self.peers}
        shapes = {p: (self.ranges[p][1] - self.ranges[p][0], 3) for p in self.peers}
        recv = self._exchange(send, shapes, torch.float64)
        if self.t_ghost is None:
            tsend = {q: self.t_owned.index_select(0, torch.as_tensor(plan.send[me][q][0], device=dev))
                     for q in self.peers}
            tshapes = {p: (self.ranges[p][1] - self.ranges[p][0],) for p in self.peers}
            trecv = self._exchange(tsend, tshapes, torch.int32)
            parts = []
            for p in range(plan.nslab):
                if p == me:
                    parts.append(self.t_owned.index_select(0, torch.as_tensor(plan.send[me][me][0], device=dev)))
                else:
                    parts.append(trecv[p])
            self.t_ghost = torch.cat(parts, 0)
        parts = [self._own_ghosts(x_owned) if p == me else recv[p] for p in range(plan.nslab)]
        ghosts = torch.cat(parts, 0)
        xs = _sub_region_coords(plan, me, x_owned, ghosts)
        ts = torch.cat([self.t_owned, self.t_ghost], 0).contiguous()
        e, f, v = self.evaluate_local(xs, ts, plan.sub_box(), self.nloc)
        f_own = f[: self.nloc].clone()
        # reverse halo
        back = {p: f[self.nloc + a: self.nloc + b].contiguous() for p, (a, b) in enumerate(self.ranges)
                if p != me}
        rshapes = {q: (len(plan.send[me][q][0]), 3) for q in self.peers}
        got = self._exchange(back, rshapes, torch.float64)
        a, b = self.ranges[me]
        pieces = [(plan.send[me][me][0], f[self.nloc + a: self.nloc + b])]
        pieces += [(plan.send[me][q][0], got[q]) for q in self.peers]
        for pos, inc in pieces:
            if len(pos):
                f_own.index_add_(0, torch.as_tensor(pos, device=dev), inc)
        red = torch.cat([torch.as_tensor([float(e)], dtype=torch.float64, device=dev),
                         torch.as_tensor(v, dtype=torch.float64, device=dev).reshape(9)])
        self.dist.all_reduce(red, group=self.group)
        return float(red[0]), f_own, red[1:].reshape(3, 3)


class DPLocalEvaluator:
    """evaluate_local on the GPU: dp_build_nlist + dp_eval_local of one
    sub-region.  The candidate capacity is set from the density of the whole
    system (the padded sub-region cell has vacuum, which would make the
    density-based default too small)."""

    def __init__(self, model, natoms_max, density, precision=None, stream=None):
        from . import dp
        self.dp = dp
        rc = model.desc["rcut"]
        expect = density * 4.0 / 3.0 * np.pi * rc ** 3
        cap = int(min(1024, np.ceil((1.5 * expect + 64.0) / 32.0) * 32))
        prec = dp.DP_PREC_FP64 if precision is None else precision
        self.ctx = dp.Context(model, natoms_max, cand_cap=cap, precision=prec, stream=stream)

    def __call__(self, xs, ts, sub_box, nloc):
        self.dp.dp_build_nlist(self.ctx, xs, ts, sub_box, 0.0)
        out = self.dp.dp_eval_local(self.ctx, xs, ts, sub_box, nloc)
        return out["energy"].item(), out["force"], out["virial"]

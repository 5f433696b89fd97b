"""Domain decomposition of one lattice into x slabs, one per rank, with a
halo exchange per time step (the multi-GPU form of the step).

The node update reads the streamed populations of its own node, which come
from the neighbours one column away, and the gradient inputs (u, Pi, Y_a)
of the neighbouring nodes, which are moments of their streamed populations.
A node's new state therefore depends on the post-collision populations of
the previous step up to two columns away.  Each rank keeps its owned
columns plus two ghost columns on every side that borders another rank
(HALO = 2) and runs the ordinary single-lattice step on that local lattice.
After the step the two outermost ghost columns on a side hold values
computed from incomplete data, but every owned column is exact, and the
exchange then overwrites the ghosts with the neighbours' owned columns of
the same step.  The local lattices are plain contexts of the library: a
side that borders another rank is given the kind of the global x faces
(periodic wrap when the global lattice is periodic in x, else the global
face's reservoir or bounce-back rule), which only ever touches the ghost
columns.

Results equal the undivided lattice node for node (the same arithmetic on
the same inputs).  The exchange moves 2 columns x (L Q ny nz) populations
per side and step.

Two transports: ``DistExchange`` (torch.distributed point-to-point, one rank
per process: NCCL between GPUs, gloo on CPU) and ``LocalExchange`` (every
slab in one process, copies).  A stepper is any object with ``step(n)``,
``get_columns(lo, hi)`` returning the populations of its local columns
[lo, hi) as a contiguous tensor [L, Q, nz, ny, hi - lo], and
``set_columns(lo, data)``; only the halo columns move.  ``LatticeStepper``
wraps a library context (lbm_get_columns / lbm_set_columns, asynchronous
on the context's stream).
"""
from __future__ import annotations

import copy
import dataclasses
from typing import List, Optional

import numpy as np

HALO = 2


@dataclasses.dataclass
class Slab:
    rank: int
    x0: int            # first owned global column
    x1: int            # one past the last owned global column
    glo: int           # ghost columns on the low side
    ghi: int           # ghost columns on the high side
    left: Optional[int]    # rank across the low side (None: a global face)
    right: Optional[int]   # rank across the high side

    @property
    def nx_local(self) -> int:
        return self.x1 - self.x0 + self.glo + self.ghi


def plan(nx: int, world: int, periodic: bool) -> List[Slab]:
    """Contiguous x ranges of nearly equal width, one per rank."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    bounds = np.linspace(0, nx, world + 1).round().astype(int)
    slabs = []
    for r in range(world):
        x0, x1 = int(bounds[r]), int(bounds[r + 1])
        if world > 1 and x1 - x0 < HALO:
            raise ValueError("each slab must own at least two columns")
        left = (r - 1) % world if (r > 0 or periodic) else None
        right = (r + 1) % world if (r < world - 1 or periodic) else None
        if world == 1:
            left = right = None
        slabs.append(Slab(r, x0, x1, HALO if left is not None else 0, HALO if right is not None else 0,
                          left, right))
    return slabs


def local_workload(wl, s: Slab):
    """The workload of one slab: the global per-node fields over its owned
    and ghost columns (wrapping periodically), the global faces where the
    slab meets them and the global face kind on its artificial sides."""
    periodic = wl.bc_lo == "periodic"
    cols = np.arange(s.x0 - s.glo, s.x1 + s.ghi)
    if periodic:
        cols = cols % wl.nx
    out = copy.copy(wl)
    out.nx = len(cols)

    def take(a):
        a = np.asarray(a)
        lead = a.shape[:-1]
        g = a.reshape(lead + (wl.nz, wl.ny, wl.nx))[..., cols]
        return np.ascontiguousarray(g.reshape(lead + (-1,)))

    out.porosity = take(wl.porosity)
    out.X_init = take(wl.X_init)
    out.T_init = take(wl.T_init)
    out.P_init = take(wl.P_init)
    if getattr(wl, "U_init", None) is not None:
        out.U_init = take(wl.U_init)
    if not periodic:
        # artificial sides take the global faces' kind; only ghosts see them
        out.bc_lo = wl.bc_lo if s.left is None else (wl.bc_lo if wl.bc_lo != "periodic" else wl.bc_hi)
        out.bc_hi = wl.bc_hi if s.right is None else (wl.bc_hi if wl.bc_hi != "periodic" else wl.bc_lo)
    out.name = f"{wl.name}_slab{s.rank}"
    return out


def owned_range(wl_local, s: Slab, side: str):
    """Local column range of the HALO owned columns next to a side."""
    if side == "lo":
        return s.glo, s.glo + HALO
    n = wl_local.nx - s.ghi
    return n - HALO, n


def ghost_start(wl_local, s: Slab, side: str) -> int:
    """First local column of the ghosts on a side."""
    return 0 if side == "lo" else wl_local.nx - s.ghi


class LocalExchange:
    """Every slab in this process: the ghosts are copied from the neighbours'
    owned columns of the same step."""

    def exchange(self, steppers, wls, slabs):
        edges = [{side: g.get_columns(*owned_range(w, s, side)) for side in ("lo", "hi")}
                 for g, w, s in zip(steppers, wls, slabs)]
        for g, w, s in zip(steppers, wls, slabs):
            if s.left is not None:
                g.set_columns(ghost_start(w, s, "lo"), edges[s.left]["hi"])
            if s.right is not None:
                g.set_columns(ghost_start(w, s, "hi"), edges[s.right]["lo"])


class DistExchange:
    """One slab per rank; point-to-point sends of the owned edge columns to
    the neighbouring ranks (torch.distributed: NCCL or gloo)."""

    def __init__(self, group=None):
        self.group = group

    def exchange(self, steppers, wls, slabs):
        import torch
        import torch.distributed as dist
        (g,), (w,), (s,) = steppers, wls, slabs
        # the owned edge columns next to each side with a neighbour (every
        # edge and ghost block has the same shape: HALO columns)
        edge = {side: g.get_columns(*owned_range(w, s, side))
                for side, nb in (("lo", s.left), ("hi", s.right)) if nb is not None}
        recv = {}
        # two rounds, each with at most one send and one receive per rank, so
        # that messages pair up by order even when both neighbours are the
        # same rank (two slabs on a periodic lattice) and the backend has no
        # tags: first the high edges move right, then the low edges move left
        for send_side, to, recv_side, frm in (("hi", s.right, "lo", s.left), ("lo", s.left, "hi", s.right)):
            ops = []
            if frm is not None:
                recv[recv_side] = torch.empty_like(edge[recv_side])
                ops.append(dist.P2POp(dist.irecv, recv[recv_side], frm, self.group))
            if to is not None:
                ops.append(dist.P2POp(dist.isend, edge[send_side], to, self.group))
            if ops:
                for req in dist.batch_isend_irecv(ops):
                    req.wait()
        for side, data in recv.items():
            g.set_columns(ghost_start(w, s, side), data)


class SlabRun:
    """Steps the slabs of this process (all of them with LocalExchange, its
    own with DistExchange) and exchanges the halos after every step."""

    def __init__(self, wl, world: int, ranks, make_stepper, exchange):
        periodic = wl.bc_lo == "periodic"
        self.all_slabs = plan(wl.nx, world, periodic)
        self.slabs = [self.all_slabs[r] for r in ranks]
        self.wls = [local_workload(wl, s) for s in self.slabs]
        self.steppers = [make_stepper(w) for w in self.wls]
        self.exchange = exchange

    def step(self, n: int = 1):
        for _ in range(n):
            for g in self.steppers:
                g.step(1)
            self.exchange.exchange(self.steppers, self.wls, self.slabs)

    def owned(self, state, k: int):
        """Owned columns of a per-node field [..., N_local] of local slab k,
        as [..., nz, ny, owned columns]."""
        w, s = self.wls[k], self.slabs[k]
        a = np.asarray(state)
        lead = a.shape[:-1]
        return a.reshape(lead + (w.nz, w.ny, w.nx))[..., s.glo:w.nx - s.ghi]


class LatticeStepper:
    """A library context as a slab stepper.  The context runs on the torch
    stream current at construction, so its steps, its column copies and the
    exchange's tensor operations are ordered on one stream."""

    def __init__(self, wl, precision, device=None):
        import ctypes

        import torch

        from . import lbm
        self.torch = torch
        st = torch.cuda.current_stream(device)
        self.g = lbm.Lattice(wl, precision=precision, stream=ctypes.c_void_p(st.cuda_stream))
        self.dtype = torch.float64 if precision == lbm.LBM_FP64 else torch.float32
        self.device = st.device
        self.shape = (self.g.L, self.g.Q, wl.nz, wl.ny)

    def step(self, n: int):
        self.g.step(n)

    def get_columns(self, lo: int, hi: int):
        out = self.torch.empty(self.shape + (hi - lo,), dtype=self.dtype, device=self.device)
        return self.g.get_columns(lo, hi - lo, out)

    def set_columns(self, lo: int, data):
        self.g.set_columns(lo, data.contiguous())

"""x-slab domain decomposition with a halo exchange per step
(paper_2409_02930_gb300/slabs.py), on CPU: the slabs are stepped by the FP64
oracle (the checker stands in for the per-rank stepper here) and the
decomposed run must equal the undivided lattice node for node.  In one
process (every slab, copies) and as two gloo ranks on 127.0.0.1
(point-to-point sends)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_2409_02930_gb300 import slabs as S  # noqa: E402
from paper_2409_02930_gb300 import workloads as W  # noqa: E402


class OracleStepper:
    def __init__(self, wl):
        self.wl = wl
        self.o = oracle.Oracle(wl)

    def _grid(self, p):
        return p.reshape(self.o.nl, self.o.Q, self.wl.nz, self.wl.ny, self.wl.nx)

    def step(self, n):
        self.o.step(n)

    def get_columns(self, lo, hi):
        return torch.from_numpy(np.ascontiguousarray(self._grid(self.o.pops())[..., lo:hi]))

    def set_columns(self, lo, data):
        p = self.o.pops().copy()
        self._grid(p)[..., lo:lo + data.shape[-1]] = data.numpy()
        self.o.set_pops(p)


def cases():
    periodic = W.slab(nx=23, ny=6, steps=30, name="periodic_slab")
    reservoir = W.adjoint_slab(nx=26, ny=5, steps=30)
    closed = W.slab(nx=20, ny=4, steps=30, name="closed_slab")
    closed.bc_lo = closed.bc_hi = W.BC_BOUNCEBACK
    return {"periodic": periodic, "reservoir": reservoir, "bounceback": closed}


def global_owned(o, wl, s):
    p = o.pops().reshape(o.nl, o.Q, wl.nz, wl.ny, wl.nx)
    return p[..., s.x0:s.x1]


@pytest.mark.parametrize("name", ["periodic", "reservoir", "bounceback"])
@pytest.mark.parametrize("world", [2, 3])
def test_slabs_in_one_process_equal_the_whole_lattice(name, world):
    wl = cases()[name]
    run = S.SlabRun(wl, world, range(world), OracleStepper, S.LocalExchange())
    run.step(wl.steps)
    whole = oracle.Oracle(wl)
    whole.step(wl.steps)
    for k, s in enumerate(run.slabs):
        mine = run.owned(run.steppers[k].o.pops(), k)
        ref = global_owned(whole, wl, s)
        np.testing.assert_allclose(mine, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_exchange_moves_only_the_halo_columns():
    """The in-process exchange reads the two owned columns next to each
    inner side and writes the two ghost columns there; every other column of
    every slab is left as it was."""
    wl = cases()["periodic"]
    run = S.SlabRun(wl, 3, range(3), OracleStepper, S.LocalExchange())
    for g in run.steppers:
        g.step(3)
    before = [g.o.pops().copy() for g in run.steppers]
    run.exchange.exchange(run.steppers, run.wls, run.slabs)
    for g, w, s, b in zip(run.steppers, run.wls, run.slabs, before):
        a = g.o.pops().reshape(g.o.nl, g.o.Q, w.nz, w.ny, w.nx)
        b = b.reshape(a.shape)
        changed = np.where(np.any(a != b, axis=(0, 1, 2, 3)))[0]
        ghosts = set(range(s.glo)) | set(range(w.nx - s.ghi, w.nx))
        assert set(changed.tolist()) <= ghosts
        nb = run.steppers[s.left]
        wl_l, s_l = run.wls[s.left], run.slabs[s.left]
        left_edge = nb.o.pops().reshape(a.shape[:4] + (wl_l.nx,))[..., wl_l.nx - s_l.ghi - S.HALO:wl_l.nx - s_l.ghi]
        np.testing.assert_array_equal(a[..., :s.glo], left_edge)


def test_plan_splits_and_links_the_slabs():
    sl = S.plan(10, 3, periodic=False)
    assert [(s.x0, s.x1) for s in sl] == [(0, 3), (3, 7), (7, 10)]
    assert (sl[0].left, sl[0].right, sl[2].right) == (None, 1, None)
    assert (sl[0].glo, sl[0].ghi, sl[1].glo, sl[2].ghi) == (0, 2, 2, 0)
    sp = S.plan(10, 2, periodic=True)
    assert (sp[0].left, sp[1].right) == (1, 0)
    with pytest.raises(ValueError):
        S.plan(3, 2, periodic=True)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wl = cases()[name]
        run = S.SlabRun(wl, ws, [rank], OracleStepper, S.DistExchange())
        run.step(wl.steps)
        out[rank] = run.owned(run.steppers[0].o.pops(), 0)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["periodic", "reservoir"])
def test_two_gloo_ranks_equal_the_whole_lattice(name):
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(ws, port, name, out), nprocs=ws, join=True)
    wl = cases()[name]
    whole = oracle.Oracle(wl)
    whole.step(wl.steps)
    for s in S.plan(wl.nx, ws, wl.bc_lo == W.BC_PERIODIC):
        ref = global_owned(whole, wl, s)
        np.testing.assert_allclose(out[s.rank], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())

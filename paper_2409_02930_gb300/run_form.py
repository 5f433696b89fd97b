"""Run one kernel form for a few steps on a small case (for profilers).

    python -m paper_2409_02930_gb300.run_form anode|anode_gather|react|batch|adjoint|slab_fp64

anode:   D3Q27 anode 64x32x32, six species, FP32, the default form (staged with
         a gradient pass, variant 5), 3 steps
anode_gather: the same with the staged form that gathers the gradient
         inputs itself (variant 3)
react:   the same lattice with the seeded surface mechanism, FP32, 3 steps
batch:   the 64-capillary sweep, FP32, staged persistent form (variant 7), 5 steps
         launched one by one (timing on, so no graph replay)
adjoint: 64x64 adjoint slab, FP32, 10 steps with checkpoints every 5
slab_fp64: the 512x512 slab in FP64, the default form, 3 steps
"""
from __future__ import annotations

import sys

from . import lbm
from . import workloads as W


def main(which: str) -> None:
    if which in ("anode", "anode_gather"):
        g = lbm.Lattice(W.anode3d(nx=64, ny=32, nz=32, steps=3), precision=lbm.LBM_FP32)
        g.set_variant(5 if which == "anode" else 3)
        g.step(3)
        g.sync()
    elif which == "react":
        g = lbm.Lattice(W.anode3d_reactive(nx=64, ny=32, nz=32, steps=3), precision=lbm.LBM_FP32)
        g.step(3)
        g.sync()
    elif which == "batch":
        b = lbm.Batch(W.capillary_batch(), precision=lbm.LBM_FP32)
        b.set_variant(7)
        lbm.load().lbm_set_timing(b._h, 1)
        b.step(5)
        b.sync()
    elif which == "slab_fp64":
        g = lbm.Lattice(W.slab(512, 512, steps=3), precision=lbm.LBM_FP64)
        g.step(3)
        g.sync()
    elif which == "adjoint":
        g = lbm.Lattice(W.adjoint_slab(nx=64, ny=64, steps=10), precision=lbm.LBM_FP32)
        g.adjoint(10, 5)
    else:
        raise SystemExit(f"unknown form {which!r}")
    print("ok")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "anode")

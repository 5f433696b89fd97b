"""torch.autograd.Function over the adjoint of the C library.

``outlet_flux(phi, pore_radius, tortuosity, workload, ...)`` returns the
species flux through a plane after n steps from the workload's initial
state as a differentiable function of the porosity field, the pore radius
and the tortuosity.  The forward pass runs ``lbm_adjoint`` (forward run with
checkpoints, then the reverse sweep); backward scales the stored gradients
by the incoming gradient.  PyTorch only carries the tensors: every step and
every adjoint step runs in the library's kernels.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import lbm


class OutletFlux(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, pore_radius, tortuosity, wl, precision, steps, ckpt_every, species, plane):
        w = copy.copy(wl)
        w.porosity = phi.detach().to("cpu", torch.float64).numpy().reshape(-1).copy()
        w.pore_radius = float(pore_radius)
        w.tortuosity = float(tortuosity)
        g = lbm.Lattice(w, precision=precision)
        try:
            J, dphi, dpore, dtort = g.adjoint(steps, ckpt_every, species=species, plane=plane)
        finally:
            g.close()
        ctx.save_for_backward(torch.from_numpy(dphi).to(phi.device, phi.dtype),
                              torch.tensor(dpore, dtype=torch.float64), torch.tensor(dtort, dtype=torch.float64))
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, gJ):
        dphi, dpore, dtort = ctx.saved_tensors
        gJ = gJ.to(torch.float64)
        return (gJ.to(dphi.dtype) * dphi, (gJ.cpu() * dpore).to(torch.float64), (gJ.cpu() * dtort).to(torch.float64),
                None, None, None, None, None, None)


def outlet_flux(phi: torch.Tensor, pore_radius: torch.Tensor, tortuosity: torch.Tensor, wl,
                precision: int = lbm.LBM_FP32, steps: int = 1000, ckpt_every: int = 50, species: int = 0,
                plane=None) -> torch.Tensor:
    """Differentiable outlet flux of `species` (see ``lbm.Lattice.adjoint``)."""
    plane = wl.nx - 2 if plane is None else int(plane)
    return OutletFlux.apply(phi, pore_radius, tortuosity, wl, precision, int(steps), int(ckpt_every), int(species),
                            plane)

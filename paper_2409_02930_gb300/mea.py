"""One-dimensional charge transport of a porous electrode around the fused
step (Sec. 4.1): the serial outer loops of the membrane-electrode assembly.

Along the cell direction x the electrode phase has one potential
(Eq. 75), the volumetric current of the triple-phase
boundary I_v(x) integrates to the current density I_a(x)
(Eq. 76), and Ohm's law in the electrolyte phase integrates
I_a Omega to the electrolyte potential (Eq. 77), zero at
the start of the active section (x = 0 here, the gas side).  The TPB steps
see Phi_electrode - Phi_electrolyte(x).  The integrals are taken over the
lattice's cells (reading R30): I_a on the face after column i is the sum of
I_v dx over columns 0..i, and the electrolyte potential of column i is the
sum of I_a Omega dx over the faces before it; I_v of a column is its mean
over y and z.

``relax`` alternates blocks of lattice steps with updates of the potential
field until the electrolyte potential settles; ``potential_for_current``
finds by the secant method the electrode potential that carries a target
current density (the paper does this for the cathode potential, Sec. 4.1;
here it is applied to the one electrode the lattice holds), and
``polarisation_curve`` relaxes the cell at a list of electrode potentials.
Both take an optional ``restore`` that puts the stepper back into one
saved state before every relaxation (``lbm.Lattice.load_state`` of an image
from ``save``), so that every point starts from the same state and the
current is a function of the potential alone; without it each relaxation
continues from where the previous one stopped.

A stepper has ``step(n)``, ``current()`` (I_v per node, [N], A/m^3) and
``set_potential(field)`` (Phi_electrode - Phi_electrolyte per node, [N], V);
``lbm.Lattice`` has all three (``current`` through LBM_MOM_CURRENT).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def current_density(Iv_x: np.ndarray, dx: float) -> np.ndarray:
    """I_a on the face after each column [A/m^2] (Eq. 76)."""
    return np.cumsum(np.asarray(Iv_x, float)) * dx


def electrolyte_potential(Ia_faces: np.ndarray, omega_x, dx: float) -> np.ndarray:
    """Electrolyte potential of each column [V], zero at column 0
    (Eq. 77): the ohmic drops I_a Omega dx over the faces
    before it."""
    Ia = np.asarray(Ia_faces, float)
    om = np.broadcast_to(np.asarray(omega_x, float), Ia.shape)
    drop = Ia * om * dx
    return np.concatenate([[0.0], np.cumsum(drop[:-1])])


@dataclasses.dataclass
class CellState:
    phi_electrode: float
    Iv_x: np.ndarray          # column means of the volumetric current [A/m^3]
    Ia_x: np.ndarray          # current density on the faces [A/m^2]
    phi_electrolyte: np.ndarray   # [V] per column
    updates: int

    @property
    def current_density(self) -> float:
        """Current density leaving the electrode at its far face [A/m^2]."""
        return float(self.Ia_x[-1])


class HalfCell:
    """A porous electrode lattice (x the cell direction) with the potential
    field of Sec. 4.1 fed back into its TPB steps."""

    def __init__(self, stepper, nx: int, ny: int, nz: int, dx: float, omega):
        self.g = stepper
        self.nx, self.ny, self.nz, self.dx = nx, ny, nz, dx
        self.omega = omega                       # electrolyte resistivity [Ohm m], scalar or per column
        self.phi_el = np.zeros(nx)

    def _column_mean(self, field: np.ndarray) -> np.ndarray:
        return np.asarray(field).reshape(self.nz, self.ny, self.nx).mean(axis=(0, 1))

    def _apply(self, phi_electrode: float):
        dphi = phi_electrode - self.phi_el
        self.g.set_potential(np.broadcast_to(dphi, (self.nz, self.ny, self.nx)).reshape(-1).copy())

    def reset(self, restore=None):
        """Electrolyte potential back to zero and, with restore, the stepper
        back to its saved state."""
        self.phi_el = np.zeros(self.nx)
        if restore is not None:
            restore()

    def relax(self, phi_electrode: float, steps_per_update: int = 200, max_updates: int = 50,
              tol: float = 1e-6) -> CellState:
        """Steps the lattice in blocks, updating the electrolyte potential from
        the current after each block, until it changes by less than tol [V]."""
        for it in range(1, max_updates + 1):
            self._apply(phi_electrode)
            self.g.step(steps_per_update)
            Iv = self._column_mean(self.g.current())
            Ia = current_density(Iv, self.dx)
            new = electrolyte_potential(Ia, self.omega, self.dx)
            change = float(np.max(np.abs(new - self.phi_el)))
            self.phi_el = new
            if change < tol:
                break
        return CellState(phi_electrode, Iv, Ia, self.phi_el.copy(), it)

    def _point(self, phi_electrode: float, restore, relax_kw) -> CellState:
        if restore is not None:
            self.reset(restore)
        return self.relax(phi_electrode, **relax_kw)

    def potential_for_current(self, target: float, phi0: float, phi1: float, rtol: float = 1e-3,
                              max_iter: int = 20, restore=None, **relax_kw) -> CellState:
        """Secant iteration on the electrode potential until the relaxed cell
        carries the target current density [A/m^2] within rtol."""
        s0 = self._point(phi0, restore, relax_kw)
        s1 = self._point(phi1, restore, relax_kw)
        f0, f1 = s0.current_density - target, s1.current_density - target
        for _ in range(max_iter):
            if abs(f1) <= rtol * max(abs(target), 1e-300):
                return s1
            if f1 == f0:
                break
            phi2 = phi1 - f1 * (phi1 - phi0) / (f1 - f0)
            phi0, f0 = phi1, f1
            s1 = self._point(phi2, restore, relax_kw)
            phi1, f1 = phi2, s1.current_density - target
        if abs(f1) <= rtol * max(abs(target), 1e-300):
            return s1
        raise RuntimeError("secant iteration on the electrode potential did not reach the target current")

    def polarisation_curve(self, potentials, restore=None, **relax_kw):
        """Relaxed cell states at each electrode potential [V] (one point of
        the polarisation curve each)."""
        return [self._point(float(v), restore, relax_kw) for v in potentials]

"""The outer loops of the membrane-electrode assembly (Sec. 4.1,
paper_2409_02930_gb300/mea.py): the charge-transport integrals against
their closed forms, the secant iteration on a stepper with a known
current-potential law, and the loop around the oracle's reactive anode."""
import numpy as np
import pytest

import oracle
from paper_2409_02930_gb300 import mea
from paper_2409_02930_gb300 import workloads as W

F_C = 96485.33212


def test_uniform_current_gives_linear_current_density_and_quadratic_potential():
    """I_v uniform: I_a after column i is (i+1) I_v dx, and the electrolyte
    potential of column i is I_v Omega dx^2 i (i+1)/2 (Eq. 76,
    Eq. 77 summed over the cells, reading R30)."""
    n, dx, Iv, om = 7, 2.5e-6, 3.0e9, 0.3
    Ia = mea.current_density(np.full(n, Iv), dx)
    np.testing.assert_allclose(Ia, (np.arange(n) + 1) * Iv * dx, rtol=1e-14)
    phi = mea.electrolyte_potential(Ia, om, dx)
    i = np.arange(n)
    np.testing.assert_allclose(phi, Iv * om * dx * dx * i * (i + 1) / 2, rtol=1e-14, atol=0)


class TafelStepper:
    """A stepper whose current follows I_v = i0 (exp(a dphi) - exp(-a dphi))
    of the potential it was last given (no lattice: the outer loops alone)."""

    def __init__(self, n, i0=2e9, a=10.0):
        self.n, self.i0, self.a = n, i0, a
        self.dphi = np.zeros(n)

    def set_potential(self, field):
        self.dphi = np.asarray(field, float)

    def step(self, k):
        pass

    def current(self):
        return self.i0 * (np.exp(self.a * self.dphi) - np.exp(-self.a * self.dphi))


def test_relaxation_and_secant_on_a_known_current_law():
    """The potential field converges to the fixed point of the ohmic feedback
    (each column's current computed from Phi_electrode minus its own
    electrolyte potential), and the secant finds the electrode potential of a
    target current density."""
    nx, dx, om = 10, 2e-6, 0.3
    st = TafelStepper(nx)
    cell = mea.HalfCell(st, nx, 1, 1, dx, om)
    s = cell.relax(0.05, steps_per_update=1, max_updates=200, tol=1e-12)
    Iv = st.i0 * (np.exp(st.a * (0.05 - s.phi_electrolyte)) - np.exp(-st.a * (0.05 - s.phi_electrolyte)))
    np.testing.assert_allclose(s.Iv_x, Iv, rtol=1e-9)
    assert s.phi_electrolyte[-1] > 0 and s.current_density > 0
    target = 50.0                                          # A/m^2
    t = cell.potential_for_current(target, 0.01, 0.05, rtol=1e-8, steps_per_update=1, max_updates=200,
                                   tol=1e-13)
    assert abs(t.current_density / target - 1) < 1e-8


class AgingTafelStepper(TafelStepper):
    """A Tafel stepper whose exchange current grows with the steps taken
    since its state was saved: without a restore, the current at a given
    potential depends on the points taken before it."""

    def __init__(self, n, growth=1e-3, **kw):
        super().__init__(n, **kw)
        self.growth, self.steps = growth, 0

    def step(self, k):
        self.steps += k

    def current(self):
        return (1 + self.growth * self.steps) * super().current()

    def restore(self):
        self.steps = 0


def test_polarisation_curve_points_start_from_the_saved_state():
    """With restore every point of the curve equals the point taken alone
    on a fresh stepper (the same schedule from the same state); without it
    the later points carry the steps of the earlier ones."""
    nx, dx, om = 8, 2e-6, 0.3
    pots = [0.01, 0.02, 0.04]
    kw = dict(steps_per_update=5, max_updates=6, tol=0.0)
    st = AgingTafelStepper(nx)
    curve = mea.HalfCell(st, nx, 1, 1, dx, om).polarisation_curve(pots, restore=st.restore, **kw)
    for v, c in zip(pots, curve):
        alone = mea.HalfCell(AgingTafelStepper(nx), nx, 1, 1, dx, om).relax(v, **kw)
        assert c.current_density == alone.current_density
        np.testing.assert_array_equal(c.phi_electrolyte, alone.phi_electrolyte)
    assert all(b.current_density > a.current_density for a, b in zip(curve, curve[1:]))
    st2 = AgingTafelStepper(nx)
    drift = mea.HalfCell(st2, nx, 1, 1, dx, om).polarisation_curve(pots, **kw)
    assert drift[0].current_density == curve[0].current_density
    assert drift[2].current_density > curve[2].current_density
    # the secant with restore: a function of the potential alone
    st3 = AgingTafelStepper(nx)
    target = curve[1].current_density
    t = mea.HalfCell(st3, nx, 1, 1, dx, om).potential_for_current(target, 0.01, 0.04, rtol=1e-10,
                                                                  restore=st3.restore, **kw)
    assert abs(t.phi_electrode - 0.02) < 1e-6


class OracleStepper:
    def __init__(self, wl):
        self.o = oracle.Oracle(wl)

    def set_potential(self, field):
        self.o.set_potential(field)

    def step(self, n):
        self.o.step(n)

    def current(self):
        return self.o.moments(oracle.MOM_CURRENT)


def test_oracle_anode_half_cell():
    """The reactive anode with its TPB steps (a thin 12 x 2 x 2 slice, fuel
    reservoir at x = 0, electrolyte wall at x = nx - 1) inside the loop: the
    current density at the far face equals the sum of the column currents
    times dx, a higher electrode potential carries more current, and the
    secant reaches a target current density."""
    wl = W.anode3d_electro(nx=12, ny=2, nz=2, steps=1)
    om = wl.mechanism.resistivity
    cell = mea.HalfCell(OracleStepper(wl), wl.nx, wl.ny, wl.nz, wl.dx, om)
    lo = cell.relax(0.3, steps_per_update=20, max_updates=30, tol=1e-9)
    np.testing.assert_allclose(lo.current_density, lo.Iv_x.sum() * wl.dx, rtol=1e-12)
    cell2 = mea.HalfCell(OracleStepper(wl), wl.nx, wl.ny, wl.nz, wl.dx, om)
    hi = cell2.relax(0.45, steps_per_update=20, max_updates=30, tol=1e-9)
    assert hi.current_density > lo.current_density
    target = 0.5 * (lo.current_density + hi.current_density)
    cell3 = mea.HalfCell(OracleStepper(wl), wl.nx, wl.ny, wl.nz, wl.dx, om)
    t = cell3.potential_for_current(target, 0.3, 0.45, rtol=1e-3, steps_per_update=20, max_updates=30, tol=1e-9)
    assert abs(t.current_density / target - 1) < 1e-3
    assert 0.3 < t.phi_electrode < 0.45

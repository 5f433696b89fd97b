"""The half-cell loop of Sec. 4.1 (paper_2409_02930_gb300/mea.py) around the
FP64 GPU step against the same loop around the oracle: with the same
schedule of steps and potential updates, the current densities, column
currents and electrolyte potentials agree within the FP64 bound."""
import numpy as np
import pytest

import oracle
from paper_2409_02930_gb300 import mea
from paper_2409_02930_gb300 import workloads as W

pytestmark = pytest.mark.gpu


class OracleStepper:
    def __init__(self, wl):
        self.o = oracle.Oracle(wl)

    def set_potential(self, field):
        self.o.set_potential(field)

    def step(self, n):
        self.o.step(n)

    def current(self):
        return self.o.moments(oracle.MOM_CURRENT)


def test_gpu_half_cell_matches_oracle_half_cell():
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    wl = W.anode3d_electro(nx=12, ny=2, nz=2, steps=1)
    om = wl.mechanism.resistivity
    g = lbm.Lattice(wl, precision=lbm.LBM_FP64)
    a = mea.HalfCell(g, wl.nx, wl.ny, wl.nz, wl.dx, om).relax(0.4, steps_per_update=20, max_updates=8, tol=0.0)
    b = mea.HalfCell(OracleStepper(wl), wl.nx, wl.ny, wl.nz, wl.dx, om).relax(0.4, steps_per_update=20,
                                                                               max_updates=8, tol=0.0)
    assert a.updates == b.updates == 8
    assert abs(a.current_density / b.current_density - 1) < 1e-10
    np.testing.assert_allclose(a.Iv_x, b.Iv_x, rtol=0, atol=1e-10 * np.abs(b.Iv_x).max())
    np.testing.assert_allclose(a.phi_electrolyte, b.phi_electrolyte, rtol=0,
                               atol=1e-10 * np.abs(b.phi_electrolyte).max())
    g.close()


class FreshOracleStepper(OracleStepper):
    def __init__(self, wl):
        self.wl = wl
        super().__init__(wl)

    def restore(self):
        self.o = oracle.Oracle(self.wl)


def test_gpu_polarisation_curve():
    """A synthetic polarisation curve of the anode half-cell on the FP64 GPU
    step: every point starts from the saved initial state (lbm_save /
    lbm_load), so it equals the oracle's point started from a fresh state;
    the current density rises with the electrode potential; the secant with
    the same restore recovers the potential of a point on the curve."""
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    wl = W.anode3d_electro(nx=12, ny=2, nz=2, steps=1)
    om = wl.mechanism.resistivity
    kw = dict(steps_per_update=20, max_updates=6, tol=0.0)
    pots = [0.2, 0.3, 0.4, 0.5]
    g = lbm.Lattice(wl, precision=lbm.LBM_FP64)
    image = g.save()
    cell = mea.HalfCell(g, wl.nx, wl.ny, wl.nz, wl.dx, om)
    curve = cell.polarisation_curve(pots, restore=lambda: g.load_state(image), **kw)
    ost = FreshOracleStepper(wl)
    ref = mea.HalfCell(ost, wl.nx, wl.ny, wl.nz, wl.dx, om).polarisation_curve(pots, restore=ost.restore, **kw)
    for a, b in zip(curve, ref):
        assert abs(a.current_density / b.current_density - 1) < 1e-10, (a.phi_electrode, a.current_density,
                                                                         b.current_density)
    dens = [c.current_density for c in curve]
    print("polarisation curve (V, A/m^2):", list(zip(pots, dens)))
    assert all(b > a for a, b in zip(dens, dens[1:]))
    t = cell.potential_for_current(dens[2], 0.25, 0.45, rtol=1e-7, restore=lambda: g.load_state(image), **kw)
    assert abs(t.phi_electrode - pots[2]) < 1e-4
    g.close()

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

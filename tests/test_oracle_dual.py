"""Pins of the oracle's forward-mode dual-number build (exact directional
derivatives of the time loop), which the adjoint form is checked against.

* the value parts equal the plain FP64 build bit for bit;
* the initial populations are linear in the porosity when the fluid starts
  at rest, so their derivative along e_n is f^0(n) / phi(n) at node n;
* derivatives of an outlet flux after many steps equal central differences
  of the plain build (porosity field, pore radius, tortuosity);
* the Knudsen diffusivity depends on pore radius and tortuosity only
  through their ratio, so r_p dJ/dr_p = -tau dJ/dtau exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2409_02930_gb300 import workloads as W


def slab(steps=40):
    return W.adjoint_slab(nx=14, ny=10, steps=steps, name="adjoint_slab_14x10")


def outlet_flux(o, wl, lane=None):
    """Species-0 x-flux summed over the column x = nx - 2 (lattice units)."""
    j = o.moments(oracle.MOM_J_A, lane=lane).reshape(wl.M, 2, wl.ny, wl.nx)
    return float(j[0, 0, :, wl.nx - 2].sum())


def test_dual_values_equal_plain_build():
    wl = slab()
    a = oracle.Oracle(wl)
    b = oracle.Oracle(wl, dual=True)
    b.set_tangents(dphi=np.random.default_rng(0).normal(size=(oracle.LANES, wl.N)))
    a.step(15)
    b.step(15)
    assert np.array_equal(a.pops(), b.pops())
    assert np.array_equal(a.moments(oracle.MOM_T), b.moments(oracle.MOM_T))


def test_initial_population_derivative_is_f0_over_phi():
    wl = slab()
    o = oracle.Oracle(wl, dual=True)
    K = oracle.LANES
    nodes = np.random.default_rng(1).choice(wl.N, K, replace=False)
    dphi = np.zeros((K, wl.N))
    dphi[np.arange(K), nodes] = 1.0
    o.set_tangents(dphi=dphi)
    f0 = o.pops()
    for k in range(K):
        d = o.pops_lane(k)
        n = nodes[k]
        assert np.allclose(d[:, :, n], f0[:, :, n] / wl.porosity[n], rtol=1e-13, atol=0)
        mask = np.ones(wl.N, bool)
        mask[n] = False
        assert np.all(d[:, :, mask] == 0.0)


@pytest.fixture(scope="module")
def jvps():
    wl = slab()
    rng = np.random.default_rng(2)
    V = rng.normal(size=(6, wl.N)) * 0.05
    o = oracle.Oracle(wl, dual=True)
    dphi = np.zeros((oracle.LANES, wl.N))
    dphi[:6] = V
    dpore = np.zeros(oracle.LANES)
    dtort = np.zeros(oracle.LANES)
    dpore[6] = wl.pore_radius           # d/d(ln r_p)
    dtort[7] = wl.tortuosity            # d/d(ln tau)
    o.set_tangents(dphi=dphi, dpore=dpore, dtort=dtort)
    o.step(wl.steps)
    J = outlet_flux(o, wl)
    g = [outlet_flux(o, wl, lane=k) for k in range(oracle.LANES)]
    return wl, V, J, g


def test_dual_value_is_the_objective(jvps):
    wl, V, J, g = jvps
    p = oracle.Oracle(wl)
    p.step(wl.steps)
    assert outlet_flux(p, wl) == J


def run_plain(wl):
    o = oracle.Oracle(wl)
    o.step(wl.steps)
    return outlet_flux(o, wl)


def test_porosity_jvp_matches_central_differences(jvps):
    wl, V, J, g = jvps
    eps = 1e-5
    for k in range(3):
        wp, wm = slab(), slab()
        wp.porosity = wl.porosity + eps * V[k]
        wm.porosity = wl.porosity - eps * V[k]
        fd = (run_plain(wp) - run_plain(wm)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * abs(g[k]) + 1e-12 * abs(J), (k, fd, g[k])


def test_knudsen_jvps_match_central_differences(jvps):
    wl, V, J, g = jvps
    h = 1e-5
    for lane, attr in ((6, "pore_radius"), (7, "tortuosity")):
        wp, wm = slab(), slab()
        setattr(wp, attr, getattr(wl, attr) * (1 + h))
        setattr(wm, attr, getattr(wl, attr) * (1 - h))
        fd = (run_plain(wp) - run_plain(wm)) / (2 * h)
        assert abs(fd - g[lane]) <= 1e-6 * abs(g[lane]) + 1e-12 * abs(J), (attr, fd, g[lane])


def test_pore_radius_and_tortuosity_enter_as_a_ratio(jvps):
    wl, V, J, g = jvps
    # d/d ln r_p = - d/d ln tau
    assert abs(g[6] + g[7]) <= 1e-12 * max(abs(g[6]), abs(J)), (g[6], g[7])
    assert abs(g[6]) > 1e-8 * abs(J)        # the Knudsen term matters here

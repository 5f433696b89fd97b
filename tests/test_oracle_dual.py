"""Pins of the oracle's forward-mode dual-number build (exact directional
derivatives of the time loop), which the adjoint form is checked against.

* the value parts equal the plain FP64 build bit for bit;
* the initial populations are linear in the porosity when the fluid starts
  at rest, so their derivative along e_n is f^0(n) / phi(n) at node n;
* derivatives of an outlet flux after many steps equal central differences
  of the plain build (porosity field, pore radius, tortuosity);
* the Knudsen diffusivity depends on pore radius and tortuosity only
  through their ratio, so r_p dJ/dr_p = -tau dJ/dtau exactly;
* seeded in the pre-exponential factors A_r of a surface mechanism, the
  derivatives of the coverages, species densities and temperature after a
  few reactive steps equal central differences of the plain build in
  ln A_r (the derivative of the backward-Euler extents, carried through the
  Newton iteration in dual numbers).
"""
import copy

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


def test_full_gradient_on_a_4x4x4_lattice_by_brute_force():
    """Brute force on a 4^3 D3Q27 lattice (three species, energy, Knudsen,
    reservoirs at both x faces): the gradient of the outlet flux with respect
    to all 64 porosities, from the dual build one node per lane, against
    central differences of the plain build node by node."""
    base = W.slab(nx=4, ny=4, steps=12, bc_x=W.BC_INLET, X_lo=[0.7, 0.2, 0.1], X_hi=[0.1, 0.3, 0.6],
                  name="brute_4x4x4")

    def make(phi=None):
        wl = W.slab(nx=4, ny=4, steps=12, bc_x=W.BC_INLET, X_lo=[0.7, 0.2, 0.1], X_hi=[0.1, 0.3, 0.6],
                    name="brute_4x4x4")
        wl.nz = 4
        wl.porosity = W.porosity_field((4, 4, 4), 2.0, 41) if phi is None else phi
        wl.X_init = W.random_mole_fractions(3, 64, 42)
        wl.T_init = np.full(64, base.T_init[0])
        wl.P_init = np.full(64, base.P_init[0])
        return wl

    def J3(o, wl, lane=None):
        j = o.moments(oracle.MOM_J_A, lane=lane).reshape(wl.M, 3, 4, 4, 4)
        return float(j[0, 0, :, :, wl.nx - 2].sum())

    wl = make()
    grad = np.zeros(64)
    for start in range(0, 64, oracle.LANES):
        o = oracle.Oracle(wl, dual=True)
        dphi = np.zeros((oracle.LANES, 64))
        for k in range(oracle.LANES):
            dphi[k, start + k] = 1.0
        o.set_tangents(dphi=dphi)
        o.step(wl.steps)
        for k in range(oracle.LANES):
            grad[start + k] = J3(o, wl, lane=k)
    eps = 1e-6
    fd = np.zeros(64)
    for n in range(64):
        vals = []
        for s in (1.0, -1.0):
            phi = wl.porosity.copy()
            phi[n] += s * eps
            w = make(phi)
            p = oracle.Oracle(w)
            p.step(w.steps)
            vals.append(J3(p, w))
        fd[n] = (vals[0] - vals[1]) / (2 * eps)
    scale = np.abs(grad).max()
    assert scale > 0
    np.testing.assert_allclose(fd, grad, rtol=0, atol=1e-6 * scale)


def test_derivatives_in_the_pre_exponential_factors_match_central_differences():
    """The reactive 3-D anode (20 surface steps, 8 adsorbates) on 4 x 2 x 2
    nodes, 3 steps: lane k seeded with A_k (the derivative in ln A_k) for the
    first LANES steps of the mechanism.  Central differences of the plain
    build with A_k scaled by exp(+-h), h = 1e-3 (truncation ~h^2, measured
    below 1e-6 of the field's derivative); the bound adds the differences'
    rounding noise, 1e-13 of the field's magnitude over h.  A derivative
    dropped anywhere on the path from A_k to the fields (the rate constant,
    the Newton iteration, the sources) leaves the lane at zero and fails."""
    wl = W.anode3d_reactive(nx=4, ny=2, nz=2, steps=3)
    A = np.asarray(wl.mechanism.A, float)
    K = oracle.LANES
    dA = np.zeros((K, wl.mechanism.R))
    for k in range(K):
        dA[k, k] = A[k]
    o = oracle.Oracle(wl, dual=True)
    o.set_tangents(dA=dA)
    o.step(wl.steps)
    fields = (oracle.MOM_XS, oracle.MOM_RHO_A, oracle.MOM_T)
    h = 1e-3
    checked = 0
    for k in range(K):
        runs = []
        for sgn in (1.0, -1.0):
            w2 = copy.deepcopy(wl)
            w2.mechanism.A = A.copy()
            w2.mechanism.A[k] *= np.exp(sgn * h)
            p = oracle.Oracle(w2)
            p.step(wl.steps)
            runs.append([p.moments(f) for f in fields])
        for j, f in enumerate(fields):
            fd = (runs[0][j] - runs[1][j]) / (2 * h)
            lane = o.moments(f, lane=k)
            noise = 1e-13 * np.abs(runs[0][j]).max() / h
            err = np.abs(lane - fd).max()
            assert err <= 1e-5 * np.abs(fd).max() + noise, (k, f, err, np.abs(fd).max())
            if np.abs(fd).max() > 100 * noise:
                checked += 1
    assert checked >= 6           # the steps that act within three steps are resolved


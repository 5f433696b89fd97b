"""Pins of the oracle's heterogeneous surface source (Sec. 4, eq:totalFluidReactionRate,
eq:surfaceMoleFractions, eq:totalSurfaceReactionRate, eq:rho_pc,
eq:temperatureCell / eq:InternalEnergyCell_PC, eqn:f_source, eqn:g_source,
eq:fsourceHetero) against conservation laws the mechanism fixes."""
import numpy as np
import pytest

import oracle
from paper_2409_02930_gb300 import workloads as W

R_U = 8.314462618


def _periodic_reactive(nx=8, ny=6, nz=5):
    wl = W.anode3d_reactive(nx=nx, ny=ny, nz=nz, steps=20)
    wl.bc_lo = wl.bc_hi = W.BC_PERIODIC
    return wl


def _inventory(o, wl):
    """Element moles (H, C, N, O) in gas and adsorbed phases, summed over the
    lattice (per unit volume of porous medium times node count)."""
    mech = wl.mechanism
    rho = o.moments(oracle.MOM_RHO_A)                 # kg/m^3 of fluid
    phi = wl.porosity
    Xs = o.moments(oracle.MOM_XS)
    gas_mol = (phi[None, :] * rho / wl.molar_mass[:, None]).sum(axis=1)     # mol per m^3 REV, summed
    surf_mol = (mech.a_s * mech.gamma * Xs).sum(axis=1)
    return gas_mol @ mech.elements_gas + surf_mol @ mech.elements_surf, Xs


def test_mechanism_is_element_and_site_balanced():
    mech = W.surface_mechanism()
    assert np.all(mech.nu_gas @ mech.elements_gas + mech.nu_surf @ mech.elements_surf == 0)
    assert np.all(mech.nu_surf.sum(axis=1) == 0)


def test_surface_source_conserves_elements_and_sites():
    """Heterogeneous reactions move atoms between gas and adsorbed phases
    only: with periodic faces the lattice total of every element is constant,
    and the coverages of every node sum to one (site conservation)."""
    wl = _periodic_reactive()
    o = oracle.Oracle(wl)
    e0, _ = _inventory(o, wl)
    o.step(20)
    e1, Xs = _inventory(o, wl)
    assert np.abs(o.diag(5)).max() > 0                       # reactions are active
    mask = e0 > 0
    np.testing.assert_allclose(e1[mask], e0[mask], rtol=1e-12)
    np.testing.assert_allclose(Xs.sum(axis=0), 1.0, rtol=0, atol=1e-13)
    assert Xs.min() >= 0.0


def test_surface_source_species_mass_enters_species_lattices():
    """Per node, the species lattice gains exactly rhodot (eq:fsourceHetero,
    Sum_i fdot^r_ai = rhodot_a) and the momentum lattice the same total mass
    (eqn:f_source with eq:rho_pc)."""
    wl = _periodic_reactive()
    o = oracle.Oracle(wl)
    o.step(3)
    pre, post = o.pulled(), o.pops()
    rd = o.diag(5)                                           # kg/m^3 REV per step
    M = wl.M
    for a in range(M):
        d = post[a].sum(0) - pre[a].sum(0)
        np.testing.assert_allclose(d, rd[a], rtol=0, atol=1e-14 * np.abs(pre[a].sum(0)).max())
    dm = post[M].sum(0) - pre[M].sum(0)
    np.testing.assert_allclose(dm, rd.sum(0), rtol=0, atol=1e-14 * pre[M].sum(0).max())


def test_unified_internal_energy_is_conserved():
    """Without electrochemistry the unified internal energy of fluid and
    adsorbed phases (eq:temperatureCell) changes only by the kinetic energy
    of the exchanged mass, O(u^2) of the exchange."""
    wl = _periodic_reactive()
    mech = wl.mechanism
    o = oracle.Oracle(wl)
    o.step(2)
    pre, post = o.pulled(), o.pops()
    M = wl.M
    # fluid total energy change per node (lattice units x density, per REV volume)
    dg = (post[M + 1].sum(0) - pre[M + 1].sum(0)) * o.cvel ** 2        # J/m^3 REV
    # adsorbed-phase energy change at the node temperature
    T = o.moments(oracle.MOM_T)                                       # of the next state; use step T below
    Xs_new = o.moments(oracle.MOM_XS)
    o2 = oracle.Oracle(wl)
    o2.step(1)
    Xs_old = o2.moments(oracle.MOM_XS)
    # recompute the temperature the collision saw (state after one step, pulled)
    T_seen = o2.moments(oracle.MOM_T)
    Us = mech.surf_U0[:, None] + mech.surf_cv_factor[:, None] * R_U * (T_seen[None, :] - wl.T_thermo)
    dads = (mech.a_s * mech.gamma * (Xs_new - Xs_old) * Us).sum(0)
    scale = np.abs(pre[M + 1].sum(0)).max() * o.cvel ** 2
    assert np.abs(dads).max() > 1e-9 * scale                          # the exchange is not trivial
    assert np.max(np.abs(dg + dads)) < 1e-7 * scale

"""Pins of the oracle's heterogeneous surface source (Sec. 4, Eq. 68,
Eq. 70, Eq. 71, Eq. 78,
Eq. 80 / Eq. 85, Eq. 87, Eq. 88,
Eq. 89) against conservation laws the mechanism fixes."""
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
    """Per node, the species lattice gains exactly rhodot (Eq. 89,
    Sum_i fdot^r_ai = rhodot_a) and the momentum lattice the same total mass
    (Eq. 87 with Eq. 78)."""
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
    adsorbed phases (Eq. 80) changes only by the kinetic energy
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


# ---------------------------------------------------------------------------
# closed forms of the backward-Euler extents (reading R16) for mechanisms
# small enough to solve by hand: these fix the reactant orders, the
# Arrhenius constant k = A exp(-Ea/(R_U T)) with Ea in J/mol, the gas-side
# scale a^(s)/phi of Eq. 68 and backward (not forward)
# Euler
# ---------------------------------------------------------------------------
T_RX, PHI_RX, A_S, GAMMA = 1000.0, 0.5, 1.0e7, 2.6e-5
M_A, M_B = 28.0e-3, 40.0e-3


def _uniform_reactive(nu_gas, nu_surf, A, Ea, Xs0, X_gas=(0.5, 0.5), nx=3, ny=3, energy=False, electro=None):
    """Uniform periodic 2-D lattice of gas A and an inert gas B at 1 atm and
    1000 K (isothermal unless energy) over a surface with the given steps;
    every node is the same well-mixed reactor.  electro: (edge flags,
    electrons per step, l_tpb, resistivity, dphi) for TPB steps."""
    N = nx * ny
    S = len(Xs0)
    R = len(A)
    mech = W.Mechanism(S=S, R=R, nu_gas=np.asarray(nu_gas, float), nu_surf=np.asarray(nu_surf, float),
                       A=np.asarray(A, float), Ea=np.asarray(Ea, float), gamma=GAMMA, a_s=A_S,
                       surf_molar_mass=np.full(S, M_A), surf_cv_factor=np.zeros(S), surf_U0=np.zeros(S),
                       gas_U0_molar=np.zeros(2), elements_gas=np.eye(2, dtype=int),
                       elements_surf=np.zeros((S, 2), dtype=int), Xs_init=np.asarray(Xs0, float))
    if electro is not None:
        mech.edge, mech.n_el, mech.l_tpb, mech.resistivity, mech.dphi = electro
        mech.edge = np.asarray(mech.edge, np.int32)
        mech.n_el = np.asarray(mech.n_el, float)
    wl = W.Workload(
        name="uniform_reactor", nx=nx, ny=ny, nz=1, bc_lo=W.BC_PERIODIC, bc_hi=W.BC_PERIODIC, M=2,
        energy=energy, knudsen=False, dx=1.0e-6, theta_max=1.0 / 3.0, T_scale=T_RX, T_ref=T_RX, P_ref=W.ATM,
        molar_mass=np.array([M_A, M_B]), D_ref=np.array([[0.0, 2e-4], [2e-4, 0.0]]),
        mu_ref=np.array([4e-5, 4e-5]), mu_exp=0.7, Pr=0.7, bulk_ratio=1.0, cv_factor=np.array([2.5, 1.5]),
        U0=np.zeros(2), T_thermo=0.0, tortuosity=1.0, pore_radius=1e-6, porosity=np.full(N, PHI_RX),
        X_init=np.tile(np.asarray(X_gas, float)[:, None], (1, N)), T_init=np.full(N, T_RX),
        P_init=np.full(N, W.ATM), X_in_lo=np.asarray(X_gas, float), X_in_hi=np.asarray(X_gas, float),
        T_in_lo=T_RX, T_in_hi=T_RX, P_in_lo=W.ATM, P_in_hi=W.ATM, steps=1, mechanism=mech)
    return wl


def _rate_constant_for(dt, target):
    """Prefactor whose k at T_RX with Ea = 100 kJ/mol is target / dt."""
    return target / dt / np.exp(-100.0e3 / (R_U * T_RX)), 100.0e3


def test_adsorption_extent_is_the_backward_euler_root():
    """A + s -> A(s), r = k c_A theta_s.  One backward-Euler step solves
    xi = dt k (c0 - alpha xi)(theta0 - xi), alpha = a^(s)/phi: the smaller
    root of dt k alpha xi^2 - (1 + dt k (c0 + alpha theta0)) xi + dt k c0 theta0 = 0.
    The coverage of A(s) grows by xi/Gamma and the gas density of A falls by
    a^(s) m_A xi / phi (Eq. 68, Eq. 69)."""
    probe = oracle.Oracle(_uniform_reactive([[-1, 0]], [[-1, 1]], [1.0], [0.0], [0.9, 0.1]))
    dt = probe.dt
    c0 = 0.5 * W.ATM / (R_U * T_RX)
    th0 = 0.9 * GAMMA
    alpha = A_S / PHI_RX
    A, Ea = _rate_constant_for(dt, 1.0 / (c0 + alpha * th0))     # dt k (c0 + alpha theta0) = 1
    wl = _uniform_reactive([[-1, 0]], [[-1, 1]], [A], [Ea], [0.9, 0.1])
    o = oracle.Oracle(wl)
    rho0 = o.moments(oracle.MOM_RHO_A)
    o.step(1)
    k = A * np.exp(-Ea / (R_U * T_RX))
    a2, a1, a0 = dt * k * alpha, -(1.0 + dt * k * (c0 + alpha * th0)), dt * k * c0 * th0
    xi = (-a1 - np.sqrt(a1 * a1 - 4 * a2 * a0)) / (2 * a2)
    xi_forward = dt * k * c0 * th0
    assert abs(xi / xi_forward - 1.0) > 0.2                    # the two schemes are far apart here
    Xs = o.moments(oracle.MOM_XS)
    np.testing.assert_allclose(Xs[1], 0.1 + xi / GAMMA, rtol=1e-12)
    np.testing.assert_allclose(Xs[0], 0.9 - xi / GAMMA, rtol=1e-12)
    rho = o.moments(oracle.MOM_RHO_A)
    np.testing.assert_allclose(rho[0], rho0[0] - A_S * M_A * xi / PHI_RX, rtol=1e-12)
    np.testing.assert_allclose(rho[1], rho0[1], rtol=1e-14)


def test_dissociative_adsorption_extent_is_the_cubic_root():
    """A + 2 s -> 2 A(s), r = k c_A theta_s^2: second order in the empty site.
    Backward Euler: xi = dt k (c0 - alpha xi)(theta0 - 2 xi)^2, the root in
    [0, min(c0/alpha, theta0/2)] of that cubic."""
    probe = oracle.Oracle(_uniform_reactive([[-1, 0]], [[-2, 2]], [1.0], [0.0], [0.9, 0.1]))
    dt = probe.dt
    c0 = 0.5 * W.ATM / (R_U * T_RX)
    th0 = 0.9 * GAMMA
    alpha = A_S / PHI_RX
    A, Ea = _rate_constant_for(dt, 1.0 / (th0 * (c0 + alpha * th0)))
    wl = _uniform_reactive([[-1, 0]], [[-2, 2]], [A], [Ea], [0.9, 0.1])
    o = oracle.Oracle(wl)
    o.step(1)
    k = A * np.exp(-Ea / (R_U * T_RX))
    # dt k (c0 - alpha xi)(theta0 - 2 xi)^2 - xi = 0
    p = dt * k * np.polymul([-alpha, c0], np.polymul([-2.0, th0], [-2.0, th0])) - np.array([0, 0, 1.0, 0])
    roots = np.roots(p)
    hi = min(c0 / alpha, th0 / 2)
    xi = [r.real for r in roots if abs(r.imag) < 1e-12 * hi and 0 <= r.real <= hi]
    assert len(xi) == 1
    Xs = o.moments(oracle.MOM_XS)
    np.testing.assert_allclose(Xs[1], 0.1 + 2 * xi[0] / GAMMA, rtol=1e-11)


def test_reversible_adsorption_reaches_its_equilibrium():
    """A + s -> A(s) (k_f) and A(s) -> A + s (k_b): the steady coverages
    satisfy k_f c_A theta_s = k_b theta_A with the A inventory
    phi c_A + a^(s) theta_A and the sites theta_s + theta_A = Gamma fixed."""
    probe = oracle.Oracle(_uniform_reactive([[-1, 0]], [[-1, 1]], [1.0], [0.0], [0.9, 0.1]))
    dt = probe.dt
    c0 = 0.5 * W.ATM / (R_U * T_RX)
    Af, Ea = _rate_constant_for(dt, 0.02 / (c0 * GAMMA) * GAMMA)   # k_f c0 dt = 0.02
    Ab, _ = _rate_constant_for(dt, 0.05)                              # k_b dt = 0.05
    wl = _uniform_reactive([[-1, 0], [1, 0]], [[-1, 1], [1, -1]], [Af, Ab], [Ea, Ea], [0.9, 0.1])
    o = oracle.Oracle(wl)
    o.step(3000)
    kf, kb = Af * np.exp(-Ea / (R_U * T_RX)), Ab * np.exp(-Ea / (R_U * T_RX))
    nT = PHI_RX * c0 + A_S * 0.1 * GAMMA                     # moles of A per volume of medium
    # kf (nT - a_s thA)/phi (Gamma - thA) = kb thA
    q = np.polymul([-A_S / PHI_RX, nT / PHI_RX], [-1.0, GAMMA]) * kf - np.array([0, kb, 0])
    thA = [r.real for r in np.roots(q) if abs(r.imag) == 0 and 0 <= r.real <= GAMMA]
    assert len(thA) == 1
    Xs = o.moments(oracle.MOM_XS)
    np.testing.assert_allclose(Xs[1], thA[0] / GAMMA, rtol=1e-10)
    cA = o.moments(oracle.MOM_RHO_A)[0] / M_A
    np.testing.assert_allclose(kf * cA * Xs[0] * GAMMA, kb * Xs[1] * GAMMA, rtol=1e-9)


# ---------------------------------------------------------------------------
# electrochemistry (Sec. 4): charge-transfer steps on the triple-phase boundary
# ---------------------------------------------------------------------------
F_C = 96485.33212
L_TPB, OHM = 1.0e12, 0.3


@pytest.mark.parametrize("dphi", [0.0, 0.15])
def test_tpb_step_extent_current_and_potential(dphi):
    """H(s) + O(s) -> OH(s) + s + e on the TPB edge (rate per unit TPB
    length r = k theta_H theta_O, k = A exp(-Ea/RT) exp(beta n F dphi/RT),
    reading R29).  Its extent xi [mol/m] changes the surface concentrations
    by lambda xi, lambda = l_TPB/a^(s) (Eq. 71), so one
    backward-Euler step solves xi = dt k (thH - lambda xi)(thO - lambda xi);
    the coverage of OH(s) grows by lambda xi/Gamma and the volumetric current
    is I = F l_TPB xi/dt (Eq. 74)."""
    nu_s = [[1, -1, -1, 1]]                  # s, H(s), O(s), OH(s): H + O -> OH + s
    X0 = [0.7, 0.1, 0.15, 0.05]
    probe = oracle.Oracle(_uniform_reactive([[0, 0]], nu_s, [1.0], [0.0], X0,
                                            electro=([1], [1.0], L_TPB, OHM, dphi)))
    dt = probe.dt
    lam = L_TPB / A_S
    thH, thO = 0.1 * GAMMA, 0.15 * GAMMA
    A, Ea = _rate_constant_for(dt, 0.5 / (lam * (thH + thO)))
    wl = _uniform_reactive([[0, 0]], nu_s, [A], [Ea], X0, electro=([1], [1.0], L_TPB, OHM, dphi))
    o = oracle.Oracle(wl)
    I_seen = o.moments(oracle.MOM_CURRENT)
    o.step(1)
    k = A * np.exp(-Ea / (R_U * T_RX)) * np.exp(0.5 * 1.0 * F_C * dphi / (R_U * T_RX))
    a2, a1, a0 = dt * k * lam * lam, -(1.0 + dt * k * lam * (thH + thO)), dt * k * thH * thO
    xi = (-a1 - np.sqrt(a1 * a1 - 4 * a2 * a0)) / (2 * a2)
    Xs = o.moments(oracle.MOM_XS)
    np.testing.assert_allclose(Xs[3], 0.05 + lam * xi / GAMMA, rtol=1e-12)
    np.testing.assert_allclose(Xs[1], 0.1 - lam * xi / GAMMA, rtol=1e-12)
    np.testing.assert_allclose(I_seen, F_C * L_TPB * xi / dt, rtol=1e-12)


def test_tpb_energy_source_is_ohmic_heat_minus_electric_work():
    """With the energy lattice on, a uniform reactor's fluid energy changes
    over one step by the adsorbed phase's loss plus (P_Omega - P_elec) dt,
    P_elec = |dphi| I, P_Omega = (a^(s)/l_TPB) I^2 Omega dx (Sec. 4.2,
    reading R28).  The adsorbates here carry no internal energy, so the
    change is the electrochemical source alone; its sign follows the
    current."""
    nu_s = [[1, -1, -1, 1]]
    X0 = [0.7, 0.1, 0.15, 0.05]
    dphi = 0.15
    probe = oracle.Oracle(_uniform_reactive([[0, 0]], nu_s, [1.0], [0.0], X0, energy=True,
                                            electro=([1], [1.0], L_TPB, OHM, dphi)))
    A, Ea = _rate_constant_for(probe.dt, 0.01 / (L_TPB / A_S * 0.25 * GAMMA))
    wl = _uniform_reactive([[0, 0]], nu_s, [A], [Ea], X0, energy=True, electro=([1], [1.0], L_TPB, OHM, dphi))
    o = oracle.Oracle(wl)
    I = o.moments(oracle.MOM_CURRENT)
    o.step(1)
    pre, post = o.pulled(), o.pops()
    M = wl.M
    dE = (post[M + 1].sum(0) - pre[M + 1].sum(0)) * o.cvel ** 2      # J per m^3 of medium
    P_elec = abs(dphi) * I
    P_ohm = (A_S / L_TPB) * I * I * OHM * wl.dx
    expect = (P_ohm - P_elec) * o.dt
    assert np.all(np.abs(expect) > 0)
    np.testing.assert_allclose(dE, expect, rtol=1e-9)

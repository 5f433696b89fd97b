"""Seeded synthetic workloads for the porous-media reactive LBM step.

This module only generates inputs: physical parameters, seeded random fields
and seeded mechanisms.  It contains none of the method's arithmetic (no
equation of state, no equilibria, no unit conversion): both the CUDA library
and the CPU oracle receive the same physical description and each derives its
own lattice quantities from it.

The paper's own workloads cannot be reproduced (the capillary experiment's
fluxes and the SOFC mechanism are not available), so the generators below make
inputs with the shapes of those cases:

* ``capillary`` -- binary counter-diffusion in an open capillary (Sec. 5.1
  uses a 1920-node 1-D tube at 300 K with reservoirs at both ends; the
  synthetic case uses masses 4 and 40 g/mol).
* ``slab`` -- a 2-D porous slab of the SOFC-electrode gas mixture
  (H2/H2O/N2-like masses 2/18/28 g/mol at 1073.15 K, Sec. 5.2) with a seeded
  Gaussian-random-field porosity.
* ``anode3d`` -- the 3-D reactive electrode: gas plus surface-adsorbed species
  with a seeded, element-balanced mass-action mechanism.
* ``capillary_batch`` -- many independent capillaries of uneven length and
  pressure.

Node ordering everywhere is ``n = x + nx * (y + ny * z)`` (x fastest).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

ATM = 101325.0
R_UNIV = 8.314462618          # J/(mol K)

BC_PERIODIC = "periodic"
BC_INLET = "inlet"
BC_BOUNCEBACK = "bounceback"


@dataclasses.dataclass
class Mechanism:
    """Mass-action surface mechanism on one catalytic surface.

    Irreversible forward reactions; a reversible step is written as two
    entries.  Stoichiometric coefficients are signed (products positive).
    ``order_gas``/``order_surf`` are the reactant orders (the negative parts of
    the stoichiometry).
    """
    S: int                      # surface species (including the empty site)
    R: int                      # reactions
    nu_gas: np.ndarray          # (R, M) signed stoichiometry of gas species
    nu_surf: np.ndarray         # (R, S) signed stoichiometry of surface species
    A: np.ndarray               # (R,) pre-exponential factors, SI for the order
    Ea: np.ndarray              # (R,) activation energies [J/mol]
    gamma: float                # site density Gamma [mol/m^2]
    a_s: float                  # specific surface area a^(s) [1/m]
    surf_molar_mass: np.ndarray  # (S,) [kg/mol] (adsorbate mass, empty site 0)
    surf_cv_factor: np.ndarray   # (S,) C_v / (R_U / m) of the adsorbates
    surf_U0: np.ndarray          # (S,) molar internal energy at T_thermo [J/mol]
    gas_U0_molar: np.ndarray     # (M,) molar internal energy at T_thermo [J/mol]
    elements_gas: np.ndarray     # (M, E) element counts of gas species
    elements_surf: np.ndarray    # (S, E) element counts of adsorbates
    Xs_init: np.ndarray          # (S,) initial coverages (uniform)
    # electrochemistry (Sec. 4): steps on the triple-phase boundary (TPB edge)
    edge: Optional[np.ndarray] = None     # (R,) 1 for a TPB step (rate per unit TPB length)
    n_el: Optional[np.ndarray] = None     # (R,) electrons released by the step
    l_tpb: float = 0.0                    # TPB length per volume of porous medium [1/m^2]
    beta_ct: float = 0.5                  # charge-transfer symmetry factor
    resistivity: float = 0.0              # electrolyte resistivity [Ohm m]
    dphi: float = 0.0                     # Phi_electrode - Phi_electrolyte [V]


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    bc_lo: str                  # x = 0 face
    bc_hi: str                  # x = nx-1 face
    M: int
    energy: bool
    knudsen: bool
    dx: float                   # lattice spacing [m]
    theta_max: float            # lattice temperature R_a T dt^2/dx^2 of the lightest species at T_scale
    T_scale: float              # temperature that fixes dt [K]
    T_ref: float                # reference state of D_ab and mu [K]
    P_ref: float                # [Pa]
    molar_mass: np.ndarray      # (M,) [kg/mol]
    D_ref: np.ndarray           # (M, M) binary diffusivities at (T_ref, P_ref) [m^2/s]
    mu_ref: np.ndarray          # (M,) species viscosities at T_ref [Pa s]
    mu_exp: float               # mu_a ~ (T/T_ref)^mu_exp
    Pr: float                   # Prandtl number
    bulk_ratio: float           # bulk viscosity / shear viscosity
    cv_factor: np.ndarray       # (M,) C_{v,a} / R_a
    U0: np.ndarray              # (M,) specific internal energy at T_thermo [J/kg]
    T_thermo: float             # [K]
    tortuosity: float
    pore_radius: float          # [m]
    porosity: np.ndarray        # (N,)
    X_init: np.ndarray          # (M, N) initial mole fractions
    T_init: np.ndarray          # (N,) [K]
    P_init: np.ndarray          # (N,) [Pa]
    X_in_lo: np.ndarray         # (M,) reservoir composition at x = 0
    X_in_hi: np.ndarray         # (M,) reservoir composition at x = nx-1
    T_in_lo: float
    T_in_hi: float
    P_in_lo: float
    P_in_hi: float
    steps: int
    mechanism: Optional[Mechanism] = None
    U_init: Optional[np.ndarray] = None   # (D, N) initial velocity [m/s]; None: at rest

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def D(self) -> int:
        return 3 if self.nz > 1 else 2

    @property
    def Q(self) -> int:
        return 27 if self.D == 3 else 9

    @property
    def L(self) -> int:
        """Number of lattices: M species + momentum (+ energy)."""
        return self.M + 1 + (1 if self.energy else 0)


# --------------------------------------------------------------------------
# random fields
# --------------------------------------------------------------------------

def gaussian_random_field(shape, corr_len: float, seed: int) -> np.ndarray:
    """Standardised periodic Gaussian random field with covariance
    exp(-r^2 / (2 corr_len^2)), made by filtering white noise in Fourier space.
    ``shape`` is given slowest-first, e.g. (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    k2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        k = 2.0 * np.pi * np.fft.fftfreq(n)
        sh = [1] * len(shape)
        sh[ax] = n
        k2 = k2 + (k.reshape(sh)) ** 2
    # amplitude filter = sqrt of the Gaussian spectrum exp(-k^2 l^2 / 2)
    filt = np.exp(-0.25 * k2 * corr_len ** 2)
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    field -= field.mean()
    sd = field.std()
    return field / sd if sd > 0 else field


def porosity_field(shape, corr_len: float, seed: int, mean=0.45, amp=0.1, lo=0.3, hi=0.6) -> np.ndarray:
    z = gaussian_random_field(shape, corr_len, seed)
    return np.clip(mean + amp * z, lo, hi).reshape(-1)


def random_mole_fractions(M: int, N: int, seed: int, lo=0.1, hi=0.8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(M, N))
    return x / x.sum(axis=0, keepdims=True)


# --------------------------------------------------------------------------
# species sets
# --------------------------------------------------------------------------

def _he_ar():
    m = np.array([4.0e-3, 40.0e-3])
    D = np.array([[0.0, 7.0e-5], [7.0e-5, 0.0]])      # He-Ar at 300 K, 1 atm
    mu = np.array([1.99e-5, 2.27e-5])                  # at 300 K
    cv = np.array([1.5, 1.5])
    return m, D, mu, cv


def _he_ne_ar():
    """He, Ne, Ar-like masses with synthetic binary diffusivities at 300 K, 1 atm."""
    m = np.array([4.0e-3, 20.0e-3, 40.0e-3])
    D = np.array([[0.0, 1.1e-4, 7.0e-5],
                  [1.1e-4, 0.0, 3.2e-5],
                  [7.0e-5, 3.2e-5, 0.0]])
    mu = np.array([1.99e-5, 3.2e-5, 2.27e-5])
    cv = np.array([1.5, 1.5, 1.5])
    return m, D, mu, cv


def _h2_h2o_n2():
    m = np.array([2.0e-3, 18.0e-3, 28.0e-3])
    D = np.array([[0.0, 8.0e-4, 7.5e-4],
                  [8.0e-4, 0.0, 2.5e-4],
                  [7.5e-4, 2.5e-4, 0.0]])             # at 1073.15 K, 1 atm
    mu = np.array([2.0e-5, 4.0e-5, 4.2e-5])           # at 1073.15 K
    cv = np.array([2.5, 3.0, 2.5])
    return m, D, mu, cv


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def capillary(nx=256, ny=4, P=ATM, T=300.0, pore_radius=1.0e-6, dx=1.0e-6,
              steps=2000, knudsen=True, theta_max=1.0 / 3.0, name=None,
              split=True, X_lo=(1.0, 0.0), X_hi=(0.0, 1.0)) -> Workload:
    """Binary counter-diffusion of masses 4 and 40 g/mol in an open capillary
    (porosity 1, tortuosity 1), isothermal, with reservoirs of pure A at x = 0
    and pure B at x = nx-1; the left half starts as A and the right half as B
    (the split initial state of the capillary experiment, Sec. 5.1)."""
    m, D, mu, cv = _he_ar()
    N = nx * ny
    X = np.zeros((2, N))
    xs = np.tile(np.arange(nx), ny)
    X_lo = np.asarray(X_lo, float)
    X_hi = np.asarray(X_hi, float)
    if split:
        X[:, xs < nx // 2] = X_lo[:, None]
        X[:, xs >= nx // 2] = X_hi[:, None]
    else:
        X[:] = 0.5
    return Workload(
        name=name or f"capillary_{nx}x{ny}", nx=nx, ny=ny, nz=1,
        bc_lo=BC_INLET, bc_hi=BC_INLET, M=2, energy=False, knudsen=knudsen,
        dx=dx, theta_max=theta_max, T_scale=T, T_ref=300.0, P_ref=ATM,
        molar_mass=m, D_ref=D, mu_ref=mu, mu_exp=0.7, Pr=0.7, bulk_ratio=1.0,
        cv_factor=cv, U0=np.zeros(2), T_thermo=0.0, tortuosity=1.0,
        pore_radius=pore_radius, porosity=np.ones(N), X_init=X,
        T_init=np.full(N, T), P_init=np.full(N, P),
        X_in_lo=X_lo, X_in_hi=X_hi, T_in_lo=T, T_in_hi=T, P_in_lo=P, P_in_hi=P,
        steps=steps)


def slab(nx=512, ny=512, seed_phi=2, seed_X=1, steps=5000, dx=0.25e-6,
         energy=True, bc_x=BC_PERIODIC, X_lo=None, X_hi=None, name=None,
         theta_max=1.0 / 3.0) -> Workload:
    """2-D porous slab of a three-species mixture (masses 2, 18, 28 g/mol) at
    1073.15 K and 1 atm; porosity is a seeded Gaussian random field
    (correlation length 16 nodes) clipped to [0.3, 0.6]; tortuosity 3; pore
    radius 0.5 um; mole fractions seeded uniform in [0.1, 0.8] per node, then
    normalised.  With ``bc_x='inlet'`` the x faces are reservoirs."""
    m, D, mu, cv = _h2_h2o_n2()
    N = nx * ny
    T = 1073.15
    phi = porosity_field((ny, nx), 16.0, seed_phi)
    X = random_mole_fractions(3, N, seed_X)
    X_lo = np.asarray(X_lo if X_lo is not None else [1 / 3, 1 / 3, 1 / 3], float)
    X_hi = np.asarray(X_hi if X_hi is not None else [1 / 3, 1 / 3, 1 / 3], float)
    return Workload(
        name=name or f"slab_{nx}x{ny}", nx=nx, ny=ny, nz=1, bc_lo=bc_x, bc_hi=bc_x,
        M=3, energy=energy, knudsen=True, dx=dx, theta_max=theta_max, T_scale=T,
        T_ref=T, P_ref=ATM, molar_mass=m, D_ref=D, mu_ref=mu, mu_exp=0.7,
        Pr=0.7, bulk_ratio=1.0, cv_factor=cv, U0=np.zeros(3), T_thermo=0.0,
        tortuosity=3.0, pore_radius=0.5e-6, porosity=phi, X_init=X,
        T_init=np.full(N, T), P_init=np.full(N, ATM),
        X_in_lo=X_lo, X_in_hi=X_hi, T_in_lo=T, T_in_hi=T, P_in_lo=ATM, P_in_hi=ATM,
        steps=steps)


def adjoint_slab(nx=256, ny=256, steps=1000, name=None, face_ramp=8) -> Workload:
    """The slab statistics with H2-rich and H2-lean reservoirs on the x faces
    (periodic in y): the setting of the outlet-flux gradient problem.  As in
    the paper's cases fed from inlets (Sec. 5.2), the gas next to each face
    starts at that reservoir's composition: the seeded random composition
    of the interior is blended, over the `face_ramp` nodes next to each face,
    into the linear profile between the two reservoirs.  (Random
    compositions right at a reservoir face drive a growing temperature at
    the face with the energy lattice on.)"""
    wl = slab(nx=nx, ny=ny, seed_phi=6, seed_X=7, steps=steps, bc_x=BC_INLET,
              X_lo=[0.8, 0.1, 0.1], X_hi=[0.1, 0.45, 0.45],
              name=name or f"adjoint_slab_{nx}x{ny}")
    xs = np.tile(np.arange(nx), ny)
    t = xs / max(nx - 1, 1)
    lin = (1 - t)[None, :] * wl.X_in_lo[:, None] + t[None, :] * wl.X_in_hi[:, None]
    w = np.minimum(1.0, np.minimum(xs, nx - 1 - xs) / float(face_ramp))
    wl.X_init = (1 - w)[None, :] * lin + w[None, :] * wl.X_init
    return wl


# end compositions of the ternary counter-diffusion runs (He, Ne, Ar), as
# Sec. 5.1 states them: the left half and its reservoir, the right half and its
TERNARY_X_LEFT = (0.9585, 0.0265, 0.0150)
TERNARY_X_RIGHT = (0.0571, 0.5125, 0.4304)


def ternary_capillary(P, nx=246, ny=1, T=300.0, pore_radius=19.5e-6, steps=200000,
                      X_lo=TERNARY_X_LEFT, X_hi=TERNARY_X_RIGHT, name=None,
                      dx_per_radius=2.0, split=True) -> Workload:
    """Ternary counter-diffusion of He, Ne, Ar-like gases (4, 20, 40 g/mol)
    in an open capillary between two reservoirs of fixed composition at
    pressure P, isothermal (Sec. 5.1: tube diameter 39 um, so pore radius
    19.5 um; porosity and tortuosity 1; 300 K).  The two halves start at
    their reservoir's composition (split) or linear between them.  Node
    spacing dx_per_radius pore radii, or less where the momentum lattice
    needs it for omega <= 1.4 (the viscous bound of capillary_batch)."""
    m, D, mu, cv = _he_ne_ar()
    theta = 1.0 / 3.0
    dt_per_dx = np.sqrt(theta * m.min() / (R_UNIV * T))
    dx = min(dx_per_radius * pore_radius, mu.min() / (P * (1.0 / 1.4 - 0.5) * dt_per_dx))
    N = nx * ny
    xs = np.tile(np.arange(nx), ny)
    X_lo = np.asarray(X_lo, float)
    X_hi = np.asarray(X_hi, float)
    if split:
        X = np.where(xs < nx // 2, X_lo[:, None], X_hi[:, None])
    else:
        s = xs / (nx - 1.0)
        X = X_lo[:, None] * (1.0 - s) + X_hi[:, None] * s
    return Workload(
        name=name or f"ternary_capillary_{nx}x{ny}_{P:.0f}Pa", nx=nx, ny=ny, nz=1,
        bc_lo=BC_INLET, bc_hi=BC_INLET, M=3, energy=False, knudsen=True,
        dx=dx, theta_max=theta, T_scale=T, T_ref=300.0, P_ref=ATM,
        molar_mass=m, D_ref=D, mu_ref=mu, mu_exp=0.7, Pr=0.7, bulk_ratio=1.0,
        cv_factor=cv, U0=np.zeros(3), T_thermo=0.0, tortuosity=1.0,
        pore_radius=pore_radius, porosity=np.ones(N), X_init=X,
        T_init=np.full(N, T), P_init=np.full(N, P),
        X_in_lo=X_lo, X_in_hi=X_hi, T_in_lo=T, T_in_hi=T, P_in_lo=P, P_in_hi=P,
        steps=steps)


def ternary_sweep(n_pressures=5, P_lo=60.0, P_hi=40422.0, L=9.6e-3, max_nodes=246,
                  min_nodes=96, split=True) -> List[Workload]:
    """The ternary capillary at pressures log-spaced from 60 Pa to 40,422 Pa
    (Sec. 5.1: molecular to Knudsen-dominated).  The tube is the paper's
    9.6 mm where max_nodes covers it; where the viscous bound forces a
    finer spacing (high pressure) the tube is shortened to min_nodes nodes
    (still hundreds of mean free paths long).  With
    split=False the composition starts linear between the reservoirs, which
    is closer to the steady state."""
    out = []
    for P in np.geomspace(P_lo, P_hi, n_pressures):
        probe = ternary_capillary(float(P), nx=2)
        nx = int(round(L / probe.dx))
        nx = nx if nx <= max_nodes else min_nodes
        out.append(ternary_capillary(float(P), nx=nx, split=split))
    return out


def capillary_batch(n_cases=64, seed=5, ny=4, steps=2000, nmin=128, nmax=4096) -> List[Workload]:
    """Independent capillaries of the counter-diffusion experiment (Sec. 5.1:
    pure A | pure B halves fed from reservoirs of their own composition):
    lengths log-uniform in [nmin, nmax] nodes, pressures log-uniform in
    [0.01, 10] atm, pore radii log-uniform in [0.1, 10] um, masses 4 and
    40 g/mol, 300 K.  Each case has its own lattice scaling.

    Two rates bound the node spacing.  The explicit Knudsen drag rate
    dt/tau^k grows as dx/r_p, and the momentum relaxation time mu/(P dt)
    shrinks as 1/(P dx).  With the inlet boundary used here (reservoir
    equilibria moving with the adjacent node) the scheme is stable for
    omega <= 1.6 and dx >= r_p/4 and unstable (a growing boundary
    velocity) when either fails; dx is min(r_p, spacing at omega = 1.4).
    Where even that spacing is below r_p/3 -- large pores at high pressure,
    Knudsen numbers below about 1e-3, roughly a tenth of the log-square --
    the (pressure, radius) pair is drawn again, so the sample is the
    log-uniform square restricted to P r_p <= about 0.66 Pa m."""
    rng = np.random.default_rng(seed)
    m, _, mu, _ = _he_ar()
    T, theta = 300.0, 1.0 / 3.0
    dt_per_dx = np.sqrt(theta * m.min() / (R_UNIV * T))       # dt/dx of every case
    tau_min = 1.0 / 1.4 - 0.5                                   # mu/(P dt) at omega = 1.4
    lens = np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_cases)).astype(int)
    out = []
    for c in range(n_cases):
        while True:
            P = float(np.exp(rng.uniform(np.log(0.01), np.log(10.0)))) * ATM
            rp = float(np.exp(rng.uniform(np.log(0.1e-6), np.log(10e-6))))
            dx = min(rp, mu.min() / (P * tau_min * dt_per_dx))
            if dx >= rp / 3.0:
                break
        out.append(capillary(nx=int(lens[c]), ny=ny, P=P, pore_radius=rp, dx=dx, steps=steps,
                             name=f"case{c}_{int(lens[c])}x{ny}"))
    return out


def _six_species():
    """H2, H2O, CO, CO2, CH4, N2-like gas (elements H, C, N, O) at 1073.15 K."""
    names = ["H2", "H2O", "CO", "CO2", "CH4", "N2"]
    m = np.array([2.0e-3, 18.0e-3, 28.0e-3, 44.0e-3, 16.0e-3, 28.0e-3])
    inv = 1.0 / m
    ref = 1.0 / 2.0e-3 + 1.0 / 18.0e-3
    D = 8.0e-4 * np.sqrt((inv[:, None] + inv[None, :]) / ref)   # kinetic-theory mass scaling
    np.fill_diagonal(D, 0.0)
    mu = np.array([2.0e-5, 4.0e-5, 4.3e-5, 4.1e-5, 2.9e-5, 4.2e-5])
    cv = np.array([2.5, 3.0, 2.5, 3.0, 3.0, 2.5])
    elements = np.array([[2, 0, 0, 0], [2, 0, 0, 1], [0, 1, 0, 1], [0, 1, 0, 2], [4, 1, 0, 0], [0, 0, 2, 0]])
    return names, m, D, mu, cv, elements


def anode3d(nx=256, ny=128, nz=128, seed_phi=3, seed_X=4, steps=200, dx=0.25e-6, mechanism=None,
            name=None, bc_lo=BC_INLET, bc_hi=BC_BOUNCEBACK) -> Workload:
    """3-D porous anode: six gas species at 1073.15 K and 1 atm, porosity a
    seeded 3-D Gaussian random field (correlation length 16 nodes) clipped to
    [0.3, 0.6], fuel-rich reservoir at x = 0, bounce-back wall at x = nx-1
    (the anode/electrolyte interface of Sec. 5.2), periodic in y and z."""
    _, m, D, mu, cv, _ = _six_species()
    N = nx * ny * nz
    T = 1073.15
    phi = porosity_field((nz, ny, nx), 16.0, seed_phi)
    X = random_mole_fractions(6, N, seed_X)
    fuel = np.array([0.55, 0.05, 0.1, 0.05, 0.2, 0.05])
    return Workload(
        name=name or f"anode3d_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, bc_lo=bc_lo, bc_hi=bc_hi,
        M=6, energy=True, knudsen=True, dx=dx, theta_max=1.0 / 3.0, T_scale=T, T_ref=T, P_ref=ATM,
        molar_mass=m, D_ref=D, mu_ref=mu, mu_exp=0.7, Pr=0.7, bulk_ratio=1.0, cv_factor=cv,
        U0=np.zeros(6), T_thermo=0.0, tortuosity=3.0, pore_radius=0.5e-6, porosity=phi, X_init=X,
        T_init=np.full(N, T), P_init=np.full(N, ATM), X_in_lo=fuel, X_in_hi=fuel,
        T_in_lo=T, T_in_hi=T, P_in_lo=ATM, P_in_hi=ATM, steps=steps, mechanism=mechanism)


# element order H, C, N, O; atomic masses in kg/mol
_ATOMIC_MASS = np.array([1.008e-3, 12.011e-3, 14.007e-3, 15.999e-3])


def surface_mechanism(seed=4, gamma=2.6e-5, a_s=1.0e7, electrochem=False, dphi=0.2, l_tpb=1.0e12,
                      resistivity=0.3) -> Mechanism:
    """Seeded mass-action surface mechanism on one catalytic surface for the
    six-species gas (H2, H2O, CO, CO2, CH4, N2).

    Eight surface species: the empty site s and the adsorbates H(s), O(s),
    OH(s), H2O(s), CO(s), C(s), CH(s).  Twenty irreversible steps from
    element- and site-balanced templates (adsorption, dissociative
    adsorption, desorption, surface exchange; N2 is inert), with
    log10 A uniform in [5, 15] (SI units of each step's order) and
    E_a uniform in [50, 150] kJ/mol.  Site density 2.6e-5 mol/m^2 and
    specific area a_s = 20 / delta_util with delta_util = 2 um (Sec. 5.2).
    The prefactors are drawn in (mol, cm, s) units and stored in SI.

    With electrochem=True four charge-transfer steps on the triple-phase
    boundary follow (Sec. 4: edge steps between adsorbates only, rates per
    unit TPB length): H(s) + O(s) -> OH(s) + s + e and back, H(s) + OH(s) ->
    H2O(s) + s + e and back, the oxide and hydroxide adsorbates standing in
    for the ions of the electrolyte surface.  log10 A uniform in [7.5, 8.5]
    (m^3 mol^-1 s^-1), E_a uniform in [70, 90] kJ/mol (own seeded stream),
    TPB length l_tpb per volume of porous medium, potential difference dphi
    = Phi_electrode - Phi_electrolyte, electrolyte resistivity, symmetry
    factor 0.5."""
    gas = ["H2", "H2O", "CO", "CO2", "CH4", "N2"]
    surf = ["s", "H(s)", "O(s)", "OH(s)", "H2O(s)", "CO(s)", "C(s)", "CH(s)"]
    el_gas = np.array([[2, 0, 0, 0], [2, 0, 0, 1], [0, 1, 0, 1], [0, 1, 0, 2], [4, 1, 0, 0], [0, 0, 2, 0]])
    el_surf = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1], [1, 0, 0, 1], [2, 0, 0, 1], [0, 1, 0, 1],
                        [0, 1, 0, 0], [1, 1, 0, 0]])
    steps = [
        ({"H2": -1}, {"s": -2, "H(s)": 2}),
        ({"H2": 1}, {"H(s)": -2, "s": 2}),
        ({"H2O": -1}, {"s": -1, "H2O(s)": 1}),
        ({"H2O": 1}, {"H2O(s)": -1, "s": 1}),
        ({"CO": -1}, {"s": -1, "CO(s)": 1}),
        ({"CO": 1}, {"CO(s)": -1, "s": 1}),
        ({}, {"H(s)": -1, "O(s)": -1, "OH(s)": 1, "s": 1}),
        ({}, {"OH(s)": -1, "s": -1, "H(s)": 1, "O(s)": 1}),
        ({}, {"H(s)": -1, "OH(s)": -1, "H2O(s)": 1, "s": 1}),
        ({}, {"H2O(s)": -1, "s": -1, "H(s)": 1, "OH(s)": 1}),
        ({"CO2": 1}, {"CO(s)": -1, "O(s)": -1, "s": 2}),
        ({"CO2": -1}, {"s": -2, "CO(s)": 1, "O(s)": 1}),
        ({}, {"CO(s)": -1, "s": -1, "C(s)": 1, "O(s)": 1}),
        ({}, {"C(s)": -1, "O(s)": -1, "CO(s)": 1, "s": 1}),
        ({"CH4": -1}, {"s": -4, "CH(s)": 1, "H(s)": 3}),
        ({}, {"CH(s)": -1, "s": -1, "C(s)": 1, "H(s)": 1}),
        ({}, {"C(s)": -1, "H(s)": -1, "CH(s)": 1, "s": 1}),
        ({}, {"OH(s)": -2, "H2O(s)": 1, "O(s)": 1}),
        ({}, {"H2O(s)": -1, "O(s)": -1, "OH(s)": 2}),
        ({"H2": -1}, {"O(s)": -1, "H2O(s)": 1}),
    ]
    R, M, S = len(steps), len(gas), len(surf)
    nu_g = np.zeros((R, M))
    nu_s = np.zeros((R, S))
    for k, (g, s) in enumerate(steps):
        for name, v in g.items():
            nu_g[k, gas.index(name)] = v
        for name, v in s.items():
            nu_s[k, surf.index(name)] = v
    # every step conserves elements and sites
    assert np.all(nu_g @ el_gas + nu_s @ el_surf == 0)
    assert np.all(nu_s.sum(axis=1) == 0)
    rng = np.random.default_rng(seed)
    # log10 A is drawn in the (mol, cm, s) units customary for surface
    # mechanisms and converted to SI: rate [mol m^-2 s^-1] = 1e4 rate [mol cm^-2 s^-1],
    # gas concentrations 1e-6 mol cm^-3 per mol m^-3, surface 1e-4 mol cm^-2 per mol m^-2
    A_cgs = 10.0 ** rng.uniform(5.0, 15.0, R)
    n_gas = -np.where(nu_g < 0, nu_g, 0).sum(axis=1)
    n_surf = -np.where(nu_s < 0, nu_s, 0).sum(axis=1)
    A = A_cgs * 1e4 * 1e-6 ** n_gas * 1e-4 ** n_surf
    Ea = rng.uniform(50.0e3, 150.0e3, R)
    ms = el_surf @ _ATOMIC_MASS
    edge = n_el = None
    if electrochem:
        ct = [({"H(s)": -1, "O(s)": -1, "OH(s)": 1, "s": 1}, 1.0),
              ({"OH(s)": -1, "s": -1, "H(s)": 1, "O(s)": 1}, -1.0),
              ({"H(s)": -1, "OH(s)": -1, "H2O(s)": 1, "s": 1}, 1.0),
              ({"H2O(s)": -1, "s": -1, "H(s)": 1, "OH(s)": 1}, -1.0)]
        add_s = np.zeros((len(ct), S))
        for k, (st, _) in enumerate(ct):
            for name, v in st.items():
                add_s[k, surf.index(name)] = v
        assert np.all(add_s @ el_surf == 0) and np.all(add_s.sum(axis=1) == 0)
        rng2 = np.random.default_rng(seed + 100)
        nu_g = np.vstack([nu_g, np.zeros((len(ct), M))])
        nu_s = np.vstack([nu_s, add_s])
        A = np.concatenate([A, 10.0 ** rng2.uniform(7.5, 8.5, len(ct))])
        Ea = np.concatenate([Ea, rng2.uniform(70.0e3, 90.0e3, len(ct))])
        edge = np.concatenate([np.zeros(R, dtype=np.int32), np.ones(len(ct), dtype=np.int32)])
        n_el = np.concatenate([np.zeros(R), [c[1] for c in ct]])
        R = R + len(ct)
    Xs0 = np.array([0.9, 0.02, 0.02, 0.01, 0.02, 0.02, 0.005, 0.005])
    # molar C_v / R_U of the adsorbates, molecule-like; the empty site carries
    # no internal energy, so an adsorbing molecule takes its energy along
    cvs = np.array([0.0, 1.5, 1.5, 2.5, 3.0, 2.5, 1.5, 2.5])
    return Mechanism(S=S, R=R, nu_gas=nu_g, nu_surf=nu_s, A=A, Ea=Ea, gamma=gamma, a_s=a_s,
                     surf_molar_mass=ms, surf_cv_factor=cvs, surf_U0=np.zeros(S),
                     gas_U0_molar=np.zeros(M), elements_gas=el_gas, elements_surf=el_surf, Xs_init=Xs0,
                     edge=edge, n_el=n_el, l_tpb=l_tpb if electrochem else 0.0, beta_ct=0.5,
                     resistivity=resistivity if electrochem else 0.0, dphi=dphi if electrochem else 0.0)


def anode3d_electro(nx=256, ny=128, nz=128, steps=200, dphi=0.2, name=None) -> Workload:
    """The 3-D anode with the seeded surface mechanism and its charge-transfer
    steps on the triple-phase boundary at the potential difference dphi."""
    return anode3d(nx=nx, ny=ny, nz=nz, steps=steps, mechanism=surface_mechanism(electrochem=True, dphi=dphi),
                   name=name or f"anode3d_electro_{nx}x{ny}x{nz}")


def anode3d_reactive(nx=256, ny=128, nz=128, steps=200, name=None) -> Workload:
    """The 3-D anode with the seeded surface mechanism."""
    return anode3d(nx=nx, ny=ny, nz=nz, steps=steps, mechanism=surface_mechanism(),
                   name=name or f"anode3d_reactive_{nx}x{ny}x{nz}")

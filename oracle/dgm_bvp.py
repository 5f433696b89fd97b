"""Steady dusty-gas transport through an open capillary: the boundary-value
problem the lattice Boltzmann capillary relaxes to (Sec. 5.1, Eq. 20).

Test infrastructure, like the rest of oracle/: only tests may use it.

For an isothermal tube of porosity 1 and tortuosity 1 the species molar
fluxes N_a are constant along x, and with the partial pressures p_a = X_a P

    -(1/(R_U T)) dp_a/dx = sum_{b != a} (p_b N_a - p_a N_b) / D0_ab + N_a / D^k_a,

where D0_ab = P D_ab does not depend on the pressure (D_ab ~ 1/P) and D^k_a
are the Knudsen diffusivities.  Summing over a gives
-(1/(R_U T)) dP/dx = sum_a N_a / D^k_a: the pressure is linear, and
Graham's law sum_a N_a / D^k_a = 0 holds when both ends are at the same
pressure (the isobaric form -c dX_a/dx = ... with c = P/(R_U T)).

Solution.  For fixed fluxes the system is linear with constant
coefficients, d[p; 1]/dx = G(N) [p; 1], so p(x) = exp(x G) [p(0); 1] exactly,
and its integral over the tube is a block of exp([[G, I], [0, 0]] L).
Conversely, for a given profile the equations are linear in N: integrating
them over the tube gives  (integral of A(p(x)) dx) N = -(p(L) - p(0))/(R_U T).
The fluxes are the fixed point of these two exact steps, starting from the
linear profile.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

R_U = 8.314462618


def knudsen_diffusivity(pore_radius: float, T: float, molar_mass: np.ndarray) -> np.ndarray:
    """D^k_a = (2 r_p / 3) sqrt(8 R_U T / (pi m_a)) (Sec. 5.1, open capillary)."""
    return (2.0 * pore_radius / 3.0) * np.sqrt(8.0 * R_U * T / (np.pi * np.asarray(molar_mass, float)))


def _generator(N, D0, Dk, RT):
    """G with d[p; 1]/dx = G [p; 1] for fixed fluxes N."""
    M = len(N)
    G = np.zeros((M + 1, M + 1))
    for a in range(M):
        for b in range(M):
            if b == a:
                continue
            G[a, b] = -RT * N[a] / D0[a, b]          # from p_b N_a
            G[a, a] += RT * N[b] / D0[a, b]          # from -p_a N_b
        G[a, M] = -RT * N[a] / Dk[a]
    return G


def _flux_matrix(p_int, L, D0, Dk):
    """Integral over the tube of A(p) with A(p) N the right-hand side above,
    from the integral p_int of the partial pressures (A is linear in p)."""
    M = len(p_int)
    A = np.zeros((M, M))
    for a in range(M):
        A[a, a] = L / Dk[a]
        for b in range(M):
            if b == a:
                continue
            A[a, a] += p_int[b] / D0[a, b]
            A[a, b] = -p_int[a] / D0[a, b]
    return A


def fluxes_partial(p0, pL, L, D0, Dk, T, max_iter=2000, tol=1e-13) -> np.ndarray:
    """Molar fluxes [mol m^-2 s^-1] carrying the partial pressures p0 at
    x = 0 to pL at x = L; D0_ab = P D_ab [Pa m^2/s]."""
    p0 = np.asarray(p0, float)
    pL = np.asarray(pL, float)
    D0 = np.asarray(D0, float)
    Dk = np.asarray(Dk, float)
    RT = R_U * T
    M = len(p0)
    y0 = np.append(p0, 1.0)
    scale = max(np.abs(pL - p0).max(), 1e-300)
    p_int = 0.5 * (p0 + pL) * L                       # linear profile
    for _ in range(max_iter):
        N = np.linalg.solve(_flux_matrix(p_int, L, D0, Dk), -(pL - p0) / RT)
        n = M + 1
        B = np.zeros((2 * n, 2 * n))
        B[:n, :n] = _generator(N, D0, Dk, RT) * L
        B[:n, n:] = np.eye(n) * L
        E = expm(B)
        p_end = (E[:n, :n] @ y0)[:M]
        p_int = (E[:n, n:] @ y0)[:M]
        if np.abs(p_end - pL).max() <= tol * scale:
            return N
    raise RuntimeError("dusty-gas boundary-value iteration did not converge")


def fluxes(X0, XL, L, D, Dk, c) -> np.ndarray:
    """Isobaric form: mole fractions X0 -> XL over L at concentration c, D the
    binary diffusivities at that pressure.  With R_U T = 1/c, p = X and
    D0 = D the partial-pressure equations are exactly -c dX_a/dx = ..."""
    return fluxes_partial(X0, XL, L, D, Dk, 1.0 / (c * R_U))


def profile(N, p0, L, D0, Dk, T, x):
    """Partial pressures at the positions x (0 <= x <= L) for fluxes N."""
    G = _generator(np.asarray(N, float), np.asarray(D0, float), np.asarray(Dk, float), R_U * T)
    y0 = np.append(np.asarray(p0, float), 1.0)
    return np.array([(expm(G * xi) @ y0)[:-1] for xi in np.atleast_1d(x)])


def binary_closed_form(XA0, XAL, L, DAB, DkA, mA, mB, c) -> float:
    """Integrated binary Eq. 20 (isobaric, Graham's law): N_A =
    c D_AB/(alpha L) ln[(1 - alpha X_A(L) + r)/(1 - alpha X_A(0) + r)],
    alpha = 1 - sqrt(m_A/m_B), r = D_AB / D^k_A."""
    alpha = 1.0 - np.sqrt(mA / mB)
    r = DAB / DkA
    return c * DAB / (alpha * L) * np.log((1.0 - alpha * XAL + r) / (1.0 - alpha * XA0 + r))

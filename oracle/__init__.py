"""FP64 CPU oracle of the porous-media reactive LBM step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It compiles ``lbm_oracle.cpp`` (plain
C++ loops in double precision, OpenMP over nodes) with the host compiler and
drives it through ctypes.  It shares no code with the CUDA library.  The same
source built with -DORACLE_DUAL carries forward-mode dual numbers: exact
directional derivatives of the time loop with respect to the porosity field,
pore radius, tortuosity and the mechanism's pre-exponential factors
(``Oracle(wl, dual=True)``, ``set_tangents``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle.so")
_LIB_DUAL = os.path.join(_BUILD, "liblbm_oracle_dual.so")
_LIB_F32 = os.path.join(_BUILD, "liblbm_oracle_store_f32.so")
LANES = 8            # derivative lanes of the dual-number build
_lock = threading.Lock()
_lib = None
_lib_dual = None
_lib_f32 = None

BC_CODE = {"periodic": 0, "inlet": 1, "bounceback": 2}

# moment selectors (same numbering as the library's public header)
MOM_RHO_A, MOM_J_A, MOM_RHO, MOM_U, MOM_T, MOM_P, MOM_V_A, MOM_N_A, MOM_XS, MOM_RHO_S, MOM_CURRENT = range(11)

_dp = ctypes.POINTER(ctypes.c_double)


class OcConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc_lo", ctypes.c_int), ("bc_hi", ctypes.c_int),
        ("M", ctypes.c_int), ("energy", ctypes.c_int), ("knudsen", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("dx", ctypes.c_double), ("theta_max", ctypes.c_double), ("T_scale", ctypes.c_double),
        ("T_ref", ctypes.c_double), ("P_ref", ctypes.c_double),
        ("mu_exp", ctypes.c_double), ("Pr", ctypes.c_double), ("bulk_ratio", ctypes.c_double),
        ("T_thermo", ctypes.c_double), ("tortuosity", ctypes.c_double), ("pore_radius", ctypes.c_double),
        ("molar_mass", _dp), ("D_ref", _dp), ("mu_ref", _dp), ("cv_factor", _dp), ("U0", _dp),
        ("porosity", _dp), ("X_init", _dp), ("T_init", _dp), ("P_init", _dp),
        ("X_in_lo", _dp), ("X_in_hi", _dp),
        ("T_in_lo", ctypes.c_double), ("T_in_hi", ctypes.c_double),
        ("P_in_lo", ctypes.c_double), ("P_in_hi", ctypes.c_double),
        ("S", ctypes.c_int), ("R", ctypes.c_int),
        ("nu_gas", _dp), ("nu_surf", _dp), ("A_pre", _dp), ("Ea", _dp),
        ("gamma", ctypes.c_double), ("a_s", ctypes.c_double),
        ("surf_molar_mass", _dp), ("surf_cv_factor", _dp), ("surf_U0", _dp),
        ("gas_U0_molar", _dp), ("Xs_init", _dp), ("U_init", _dp),
        ("edge", ctypes.POINTER(ctypes.c_int)), ("n_el", _dp),
        ("l_tpb", ctypes.c_double), ("beta_ct", ctypes.c_double), ("resistivity", ctypes.c_double),
        ("dphi", ctypes.c_double),
    ]


def _compile(out: str, defines, force: bool) -> str:
    with _lock:
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            return out
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared"] + list(defines) + ["-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
        return out


def build(force: bool = False) -> str:
    """Compile the oracle shared library (host compiler, -O2, OpenMP)."""
    return _compile(_LIB, [], force)


def build_dual(force: bool = False) -> str:
    """Compile the forward-mode dual-number build of the same source."""
    return _compile(_LIB_DUAL, [f"-DORACLE_DUAL={LANES}"], force)


def build_store_f32(force: bool = False) -> str:
    """Compile the measuring build that rounds every stored population to
    single precision (arithmetic in double): the error floor of FP32 storage."""
    return _compile(_LIB_F32, ["-DORACLE_STORE_F32"], force)


def _declare(L):
    L.oc_create.restype = ctypes.c_void_p
    L.oc_create.argtypes = [ctypes.POINTER(OcConfig)]
    L.oc_destroy.argtypes = [ctypes.c_void_p]
    L.oc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
    for fn in ("oc_get_pops", "oc_set_pops", "oc_get_pulled", "oc_info"):
        getattr(L, fn).argtypes = [ctypes.c_void_p, _dp]
    L.oc_get_pops_lane.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
    L.oc_get_diag.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
    L.oc_moments.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
    L.oc_moments_lane.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp]
    L.oc_set_tangents.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
    L.oc_set_potential.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double]
    L.oc_threads.restype = ctypes.c_int
    L.oc_lanes.restype = ctypes.c_int
    L.oc_product_form.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    L.oc_energy_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp,
                                        ctypes.c_double, ctypes.c_double, _dp]
    L.oc_qr_solve.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
    L.oc_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def lib_dual():
    global _lib_dual
    if _lib_dual is None:
        _lib_dual = _declare(ctypes.CDLL(build_dual()))
    return _lib_dual


def lib_store_f32():
    global _lib_f32
    if _lib_f32 is None:
        _lib_f32 = _declare(ctypes.CDLL(build_store_f32()))
    return _lib_f32


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """One oracle lattice built from a ``workloads.Workload``."""

    def __init__(self, wl, nthreads: int = 0, dual: bool = False, store_f32: bool = False):
        """dual=True uses the dual-number build: every quantity carries
        ``LANES`` directional derivatives, seeded with ``set_tangents``.
        store_f32=True uses the measuring build whose stored populations are
        rounded to single precision after every step (arithmetic in double)."""
        L = lib_dual() if dual else (lib_store_f32() if store_f32 else lib())
        self._L = L
        self.wl = wl
        keep = {}

        def arr(name, v):
            a = _f64(v).reshape(-1)
            keep[name] = a
            return _ptr(a)

        c = OcConfig()
        c.nx, c.ny, c.nz = wl.nx, wl.ny, wl.nz
        c.bc_lo, c.bc_hi = BC_CODE[wl.bc_lo], BC_CODE[wl.bc_hi]
        c.M = wl.M
        c.energy, c.knudsen = int(wl.energy), int(wl.knudsen)
        c.nthreads = nthreads
        c.dx, c.theta_max, c.T_scale = wl.dx, wl.theta_max, wl.T_scale
        c.T_ref, c.P_ref = wl.T_ref, wl.P_ref
        c.mu_exp, c.Pr, c.bulk_ratio = wl.mu_exp, wl.Pr, wl.bulk_ratio
        c.T_thermo, c.tortuosity, c.pore_radius = wl.T_thermo, wl.tortuosity, wl.pore_radius
        c.molar_mass = arr("m", wl.molar_mass)
        c.D_ref = arr("D", wl.D_ref)
        c.mu_ref = arr("mu", wl.mu_ref)
        c.cv_factor = arr("cv", wl.cv_factor)
        c.U0 = arr("U0", wl.U0)
        c.porosity = arr("phi", wl.porosity)
        c.X_init = arr("X", wl.X_init)
        c.T_init = arr("T", wl.T_init)
        c.P_init = arr("P", wl.P_init)
        c.X_in_lo = arr("Xlo", wl.X_in_lo)
        c.X_in_hi = arr("Xhi", wl.X_in_hi)
        c.T_in_lo, c.T_in_hi, c.P_in_lo, c.P_in_hi = wl.T_in_lo, wl.T_in_hi, wl.P_in_lo, wl.P_in_hi
        mech = wl.mechanism
        if mech is not None:
            c.S, c.R = mech.S, mech.R
            c.nu_gas = arr("nug", mech.nu_gas)
            c.nu_surf = arr("nus", mech.nu_surf)
            c.A_pre = arr("A", mech.A)
            c.Ea = arr("Ea", mech.Ea)
            c.gamma, c.a_s = mech.gamma, mech.a_s
            c.surf_molar_mass = arr("ms", mech.surf_molar_mass)
            c.surf_cv_factor = arr("cvs", mech.surf_cv_factor)
            c.surf_U0 = arr("Us0", mech.surf_U0)
            c.gas_U0_molar = arr("Ug0", mech.gas_U0_molar)
            c.Xs_init = arr("Xs", mech.Xs_init)
            if getattr(mech, "edge", None) is not None:
                e = np.ascontiguousarray(np.asarray(mech.edge, dtype=np.int32))
                keep["edge"] = e
                c.edge = e.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
                c.n_el = arr("nel", mech.n_el)
                c.l_tpb, c.beta_ct = mech.l_tpb, mech.beta_ct
                c.resistivity, c.dphi = mech.resistivity, mech.dphi
        else:
            c.S, c.R = 0, 0
        if getattr(wl, "U_init", None) is not None:
            u3 = np.zeros((3, wl.N))
            u3[:wl.D] = np.asarray(wl.U_init).reshape(wl.D, wl.N)
            c.U_init = arr("U", u3)
        self._keep = keep
        self._cfg = c
        h = L.oc_create(ctypes.byref(c))
        if not h:
            raise ValueError("oracle rejected the configuration")
        self._h = ctypes.c_void_p(h)
        info = np.zeros(8)
        L.oc_info(self._h, _ptr(info))
        self.dt, self.cvel, self.RU = float(info[0]), float(info[1]), float(info[2])
        self.nl, self.Q, self.D = int(info[3]), int(info[4]), int(info[5])
        self.N = wl.N
        self.M = wl.M
        self.R = int(c.R)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            self._L.oc_destroy(h)
            self._h = None

    def set_potential(self, field=None, uniform: float = 0.0):
        """Phi_electrode - Phi_electrolyte of the TPB steps [V]: a field of N
        values, or `uniform` everywhere when field is None."""
        if field is None:
            self._L.oc_set_potential(self._h, None, float(uniform))
        else:
            f = _f64(field).reshape(-1)
            assert f.size == self.N
            self._L.oc_set_potential(self._h, _ptr(f), float(uniform))

    def step(self, n: int = 1):
        self._L.oc_step(self._h, int(n))

    def pops(self) -> np.ndarray:
        out = np.empty((self.nl, self.Q, self.N))
        self._L.oc_get_pops(self._h, _ptr(out))
        return out

    def set_pops(self, p: np.ndarray):
        a = _f64(p).reshape(self.nl, self.Q, self.N)
        self._L.oc_set_pops(self._h, _ptr(a))

    def pulled(self) -> np.ndarray:
        out = np.empty((self.nl, self.Q, self.N))
        self._L.oc_get_pulled(self._h, _ptr(out))
        return out

    def diag(self, which: int) -> np.ndarray:
        shapes = {0: (self.M, 3, self.N), 1: (3, self.N), 2: (self.N,), 3: (self.N,),
                  4: (self.N,), 5: (self.M, self.N), 6: (self.N,)}
        out = np.empty(shapes[which])
        self._L.oc_get_diag(self._h, which, _ptr(out))
        return out

    def moments(self, which: int, lane=None) -> np.ndarray:
        """Field `which`; with `lane` (dual build) its derivative in that lane."""
        M, D, N = self.M, self.D, self.N
        S = self.wl.mechanism.S if self.wl.mechanism is not None else 0
        shapes = {MOM_RHO_A: (M, N), MOM_J_A: (M, D, N), MOM_RHO: (N,), MOM_U: (D, N),
                  MOM_T: (N,), MOM_P: (N,), MOM_V_A: (M, D, N), MOM_N_A: (M, D, N),
                  MOM_XS: (S, N), MOM_RHO_S: (N,), MOM_CURRENT: (N,)}
        out = np.empty(shapes[which])
        if lane is None:
            self._L.oc_moments(self._h, which, _ptr(out))
        else:
            self._L.oc_moments_lane(self._h, which, int(lane), _ptr(out))
        return out

    # ---- dual-number build: exact directional derivatives ----------------
    def set_tangents(self, dphi=None, dpore=None, dtort=None, dA=None):
        """Seed the derivative lanes: dphi [LANES][N] directions of the
        porosity field, dpore / dtort [LANES] of the pore radius [m] and the
        tortuosity, dA [LANES][R] of the mechanism's pre-exponential factors.
        Resets the state to the initial equilibria and coverages."""
        K = LANES

        def opt(a, shape):
            if a is None:
                return None
            b = np.zeros(shape)
            a = np.asarray(a, float)
            b[:a.shape[0]] = a.reshape((a.shape[0],) + shape[1:])
            return b

        R = self.R
        keep = [opt(dphi, (K, self.N)), opt(dpore, (K,)), opt(dtort, (K,)),
                opt(dA, (K, R)) if R > 0 else None]
        self._L.oc_set_tangents(self._h, *[_ptr(a) if a is not None else None for a in keep])

    def pops_lane(self, lane: int) -> np.ndarray:
        out = np.empty((self.nl, self.Q, self.N))
        self._L.oc_get_pops_lane(self._h, int(lane), _ptr(out))
        return out


def threads() -> int:
    return int(lib().oc_threads())


def product_form(D: int, xi, P) -> np.ndarray:
    Q = 27 if D == 3 else 9
    out = np.empty(Q)
    lib().oc_product_form(D, _ptr(_f64(xi)), _ptr(_f64(P)), _ptr(out))
    return out


def energy_equilibrium(D: int, phi: float, rho: float, u, RT: float, U: float) -> np.ndarray:
    Q = 27 if D == 3 else 9
    out = np.empty(Q)
    uu = np.zeros(3)
    uu[:len(u)] = u
    lib().oc_energy_equilibrium(D, phi, rho, _ptr(uu), RT, U, _ptr(out))
    return out


def qr_solve(A, b) -> np.ndarray:
    A = _f64(A)
    n = A.shape[0]
    b = _f64(b).reshape(n, -1)
    x = np.empty_like(b)
    lib().oc_qr_solve(n, _ptr(A), b.shape[1], _ptr(b), _ptr(x))
    return x


def lattice(D: int):
    Q = 27 if D == 3 else 9
    c = np.empty((Q, 3), dtype=np.int32)
    w = np.empty(Q)
    lib().oc_lattice(D, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w))
    return c, w

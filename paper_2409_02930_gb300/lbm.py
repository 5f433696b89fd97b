"""Thin Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the lattice update runs in the CUDA library
``_build/liblbm.so``; this module only converts a ``workloads.Workload`` into
an ``lbm_config`` and moves buffers.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_ALLOC, LBM_ERR_NUMERIC, LBM_ERR_TIMEOUT, LBM_ERR_STATE, LBM_ERR_CUDA = 0, -1, -2, -3, -4, -5, -6
LBM_BC = {"periodic": 0, "inlet": 1, "bounceback": 2}
LBM_FP64, LBM_FP32 = 0, 1
(LBM_MOM_RHO_A, LBM_MOM_J_A, LBM_MOM_RHO, LBM_MOM_U, LBM_MOM_T, LBM_MOM_P, LBM_MOM_V_A, LBM_MOM_N_A,
 LBM_MOM_XS, LBM_MOM_RHO_S, LBM_MOM_CURRENT) = range(11)

_dp = ctypes.POINTER(ctypes.c_double)


class LbmConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc_lo", ctypes.c_int), ("bc_hi", ctypes.c_int), ("M", ctypes.c_int),
        ("energy", ctypes.c_int), ("knudsen", ctypes.c_int), ("precision", ctypes.c_int),
        ("dx", ctypes.c_double), ("theta_max", ctypes.c_double), ("T_scale", ctypes.c_double),
        ("T_ref", ctypes.c_double), ("P_ref", ctypes.c_double), ("mu_exp", ctypes.c_double),
        ("Pr", ctypes.c_double), ("bulk_ratio", ctypes.c_double), ("T_thermo", ctypes.c_double),
        ("tortuosity", ctypes.c_double), ("pore_radius", ctypes.c_double),
        ("kappa_threshold", ctypes.c_double),
        ("molar_mass", _dp), ("D_ref", _dp), ("mu_ref", _dp), ("cv_factor", _dp), ("U0", _dp),
        ("porosity", _dp), ("X_init", _dp), ("T_init", _dp), ("P_init", _dp), ("U_init", _dp),
        ("X_in_lo", _dp), ("X_in_hi", _dp),
        ("T_in_lo", ctypes.c_double), ("T_in_hi", ctypes.c_double),
        ("P_in_lo", ctypes.c_double), ("P_in_hi", ctypes.c_double),
        ("S", ctypes.c_int), ("R", ctypes.c_int),
        ("nu_gas", _dp), ("nu_surf", _dp), ("A_pre", _dp), ("Ea", _dp),
        ("gamma", ctypes.c_double), ("a_s", ctypes.c_double),
        ("surf_cv_factor", _dp), ("surf_U0", _dp), ("Xs_init", _dp),
        ("stream", ctypes.c_void_p),
        ("edge", ctypes.POINTER(ctypes.c_int)), ("n_el", _dp),
        ("l_tpb", ctypes.c_double), ("beta_ct", ctypes.c_double), ("resistivity", ctypes.c_double),
        ("dphi", ctypes.c_double),
    ]


class LbmObjective(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("species", ctypes.c_int), ("axis", ctypes.c_int),
                ("plane", ctypes.c_int), ("weight", ctypes.c_double)]


LBM_OBJ_PLANE_FLUX = 0

_lib = None


class LbmError(RuntimeError):
    pass


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LbmError(f"CUDA library not built: {path} (run paper_2409_02930_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.lbm_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(LbmConfig)]
    L.lbm_create.restype = ctypes.c_int
    L.lbm_step.argtypes = [vp, ctypes.c_int]
    L.lbm_step.restype = ctypes.c_int
    L.lbm_moments.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
    L.lbm_moments.restype = ctypes.c_int
    L.lbm_population_bytes.argtypes = [vp]
    L.lbm_population_bytes.restype = ctypes.c_size_t
    L.lbm_get_populations.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
    L.lbm_get_populations.restype = ctypes.c_int
    L.lbm_set_populations.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
    L.lbm_set_populations.restype = ctypes.c_int
    for name in ("lbm_get_columns", "lbm_set_columns"):
        getattr(L, name).argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
        getattr(L, name).restype = ctypes.c_int
    L.lbm_sync.argtypes = [vp]
    L.lbm_sync.restype = ctypes.c_int
    L.lbm_info.argtypes = [vp, _dp]
    L.lbm_info.restype = ctypes.c_int
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_variant_count.argtypes = [vp]
    L.lbm_variant_count.restype = ctypes.c_int
    L.lbm_set_variant.argtypes = [vp, ctypes.c_int]
    L.lbm_set_variant.restype = ctypes.c_int
    L.lbm_get_variant.argtypes = [vp]
    L.lbm_get_variant.restype = ctypes.c_int
    L.lbm_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.lbm_autotune.restype = ctypes.c_int
    L.lbm_step_noalloc.argtypes = [ctypes.POINTER(LbmConfig), vp, vp, vp, vp]
    L.lbm_step_noalloc.restype = ctypes.c_int
    L.lbm_noalloc_scratch_limit.argtypes = []
    L.lbm_noalloc_scratch_limit.restype = ctypes.c_size_t
    L.lbm_create_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(LbmConfig)]
    L.lbm_create_batch.restype = ctypes.c_int
    L.lbm_case_info.argtypes = [vp, ctypes.c_int, _dp]
    L.lbm_case_info.restype = ctypes.c_int
    L.lbm_adjoint.argtypes = [vp, ctypes.POINTER(LbmObjective), ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
    L.lbm_adjoint.restype = ctypes.c_int
    L.lbm_set_timing.argtypes = [vp, ctypes.c_int]
    L.lbm_set_timing.restype = ctypes.c_int
    L.lbm_get_timing.argtypes = [vp, _dp, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_get_timing.restype = ctypes.c_int
    L.lbm_step_host.argtypes = [vp, vp, vp, ctypes.c_int]
    L.lbm_step_host.restype = ctypes.c_int
    L.lbm_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.lbm_save.restype = ctypes.c_int
    L.lbm_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.lbm_load.restype = ctypes.c_int
    L.lbm_set_potential.argtypes = [vp, _dp, ctypes.c_double]
    L.lbm_set_potential.restype = ctypes.c_int
    L.lbm_set_wait_limit.argtypes = [vp, ctypes.c_int]
    L.lbm_set_wait_limit.restype = ctypes.c_int
    _lib = L
    return L


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)


def _addr(buf) -> int:
    """Address of a host buffer: numpy array, torch tensor or integer."""
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        return buf.ctypes.data
    return int(buf.data_ptr())


def _require_contiguous(buf):
    ok = buf.flags["C_CONTIGUOUS"] if isinstance(buf, np.ndarray) else buf.is_contiguous()
    if not ok:
        raise ValueError("buffer must be contiguous")


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def make_config(wl, precision: int = LBM_FP64, stream=None, kappa_threshold: float = 0.0):
    """Marshal a ``workloads.Workload`` into an ``LbmConfig``; returns
    (config, keep-alive list of the numpy arrays it points to)."""
    keep = []

    def arr(v):
        a = _f64(v)
        keep.append(a)
        return a.ctypes.data_as(_dp)

    c = LbmConfig()
    c.nx, c.ny, c.nz = wl.nx, wl.ny, wl.nz
    c.bc_lo, c.bc_hi = LBM_BC[wl.bc_lo], LBM_BC[wl.bc_hi]
    c.M = wl.M
    c.energy, c.knudsen = int(wl.energy), int(wl.knudsen)
    c.precision = precision
    c.dx, c.theta_max, c.T_scale = wl.dx, wl.theta_max, wl.T_scale
    c.T_ref, c.P_ref, c.mu_exp, c.Pr = wl.T_ref, wl.P_ref, wl.mu_exp, wl.Pr
    c.bulk_ratio, c.T_thermo = wl.bulk_ratio, wl.T_thermo
    c.tortuosity, c.pore_radius = wl.tortuosity, wl.pore_radius
    c.kappa_threshold = kappa_threshold
    c.molar_mass = arr(wl.molar_mass)
    c.D_ref = arr(wl.D_ref)
    c.mu_ref = arr(wl.mu_ref)
    c.cv_factor = arr(wl.cv_factor)
    c.U0 = arr(wl.U0)
    c.porosity = arr(wl.porosity)
    c.X_init = arr(wl.X_init)
    c.T_init = arr(wl.T_init)
    c.P_init = arr(wl.P_init)
    if getattr(wl, "U_init", None) is not None:
        u3 = np.zeros((3, wl.N))
        u3[:wl.D] = np.asarray(wl.U_init).reshape(wl.D, wl.N)
        c.U_init = arr(u3)
    c.X_in_lo = arr(wl.X_in_lo)
    c.X_in_hi = arr(wl.X_in_hi)
    c.T_in_lo, c.T_in_hi, c.P_in_lo, c.P_in_hi = wl.T_in_lo, wl.T_in_hi, wl.P_in_lo, wl.P_in_hi
    mech = getattr(wl, "mechanism", None)
    if mech is not None:
        c.S, c.R = mech.S, mech.R
        c.nu_gas = arr(mech.nu_gas)
        c.nu_surf = arr(mech.nu_surf)
        c.A_pre = arr(mech.A)
        c.Ea = arr(mech.Ea)
        c.gamma, c.a_s = mech.gamma, mech.a_s
        c.surf_cv_factor = arr(mech.surf_cv_factor)
        c.surf_U0 = arr(mech.surf_U0)
        c.Xs_init = arr(mech.Xs_init)
        if getattr(mech, "edge", None) is not None:
            e = np.ascontiguousarray(np.asarray(mech.edge, dtype=np.int32))
            keep.append(e)
            c.edge = e.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
            c.n_el = arr(mech.n_el)
            c.l_tpb, c.beta_ct = mech.l_tpb, mech.beta_ct
            c.resistivity, c.dphi = mech.resistivity, mech.dphi
    c.stream = stream if stream is not None else _current_stream()
    return c, keep


def step_noalloc(wl, pops_in_ptr: int, pops_out_ptr: int, porosity_ptr: int, t_fixed_ptr: int,
                 precision: int = LBM_FP64, stream=None) -> int:
    """One time step through ``lbm_step_noalloc``: for callers that cannot
    allocate device memory while they run (their framework owns all device
    memory, or a cudaMalloc would stall a time-critical loop).  The caller
    passes device pointers to its own state; the library's fixed scratch
    array is used for the macro fields.  Returns the C status code."""
    cfg, keep = make_config(wl, precision, stream)
    rc = load().lbm_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(pops_in_ptr), ctypes.c_void_p(pops_out_ptr),
                                 ctypes.c_void_p(porosity_ptr), ctypes.c_void_p(t_fixed_ptr))
    del keep
    return int(rc)


class Lattice:
    """One library context (``lbm_create`` ... ``lbm_destroy``)."""

    def __init__(self, wl, precision: int = LBM_FP64, stream=None, kappa_threshold: float = 0.0):
        L = load()
        self.wl = wl
        self.precision = precision
        cfg, keep = make_config(wl, precision, stream, kappa_threshold)
        h = ctypes.c_void_p()
        rc = L.lbm_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != LBM_OK:
            raise LbmError(f"lbm_create failed ({rc}): {L.lbm_last_error(None).decode()}")
        self._h = h
        info = np.zeros(5)
        L.lbm_info(h, info.ctypes.data_as(_dp))
        self.dt, self.cvel = float(info[0]), float(info[1])
        self.L, self.Q, self.D = int(info[2]), int(info[3]), int(info[4])
        self.N, self.M = wl.N, wl.M
        del keep

    def _check(self, rc, what):
        if rc != LBM_OK:
            raise LbmError(f"{what} failed ({rc}): {load().lbm_last_error(self._h).decode()}")

    def step(self, n: int = 1):
        self._check(load().lbm_step(self._h, int(n)), "lbm_step")

    def sync(self):
        self._check(load().lbm_sync(self._h), "lbm_sync")

    def moment_shape(self, which: int):
        M, D, N = self.M, self.D, self.N
        S = self.wl.mechanism.S if getattr(self.wl, "mechanism", None) is not None else 0
        return {LBM_MOM_RHO_A: (M, N), LBM_MOM_J_A: (M, D, N), LBM_MOM_RHO: (N,), LBM_MOM_U: (D, N),
                LBM_MOM_T: (N,), LBM_MOM_P: (N,), LBM_MOM_V_A: (M, D, N), LBM_MOM_N_A: (M, D, N),
                LBM_MOM_XS: (S, N), LBM_MOM_RHO_S: (N,), LBM_MOM_CURRENT: (N,)}[which]

    def moments(self, which: int) -> np.ndarray:
        out = np.empty(self.moment_shape(which))
        self._check(load().lbm_moments(self._h, which, out.ctypes.data, out.nbytes, 0), "lbm_moments")
        return out

    def moments_device(self, which: int, out):
        """Write into a caller-owned device tensor (float64, contiguous)."""
        self._check(load().lbm_moments(self._h, which, ctypes.c_void_p(out.data_ptr()),
                                       out.numel() * out.element_size(), 1), "lbm_moments")
        return out

    def variant_count(self) -> int:
        return int(load().lbm_variant_count(self._h))

    def set_variant(self, v: int):
        """-1: two-pass form; 0..variant_count()-1: fused kernel tile shapes."""
        self._check(load().lbm_set_variant(self._h, int(v)), "lbm_set_variant")

    def variant(self) -> int:
        return int(load().lbm_get_variant(self._h))

    def set_potential(self, field=None, uniform: float = 0.0):
        """Phi_electrode - Phi_electrolyte of the TPB steps [V] (lbm_set_potential):
        a field of N values, or `uniform` everywhere when field is None."""
        if field is None:
            self._check(load().lbm_set_potential(self._h, None, float(uniform)), "lbm_set_potential")
        else:
            f = _f64(field)
            assert f.size == self.N
            self._check(load().lbm_set_potential(self._h, f.ctypes.data_as(_dp), float(uniform)),
                        "lbm_set_potential")

    def current(self) -> np.ndarray:
        """Volumetric current of the TPB steps per node [A/m^3] (LBM_MOM_CURRENT)."""
        return self.moments(LBM_MOM_CURRENT)

    def set_wait_limit(self, probes: int):
        """Bound of the row-staged forms' device waits (lbm_set_wait_limit)."""
        self._check(load().lbm_set_wait_limit(self._h, int(probes)), "lbm_set_wait_limit")

    def autotune(self, steps: int = 5) -> int:
        best = ctypes.c_int(0)
        self._check(load().lbm_autotune(self._h, int(steps), ctypes.byref(best)), "lbm_autotune")
        return best.value

    def adjoint(self, steps: int, ckpt_every: int = 50, species: int = 0, axis: int = 0, plane=None,
                weight: float = 1.0):
        """Discrete adjoint of J = weight * sum over plane x = `plane` (default
        nx - 2) of the species momentum along `axis` after `steps` steps from
        the initial state.  Returns (J, dJ/dphi [N], dJ/dpore_radius,
        dJ/dtortuosity); the context is left at the final state."""
        obj = LbmObjective(LBM_OBJ_PLANE_FLUX, int(species), int(axis),
                           int(self.wl.nx - 2 if plane is None else plane), float(weight))
        J = ctypes.c_double()
        dp = ctypes.c_double()
        dt = ctypes.c_double()
        g = np.empty(self.N)
        self._check(load().lbm_adjoint(self._h, ctypes.byref(obj), int(steps), int(ckpt_every), ctypes.byref(J),
                                       g.ctypes.data_as(_dp), ctypes.byref(dp), ctypes.byref(dt)), "lbm_adjoint")
        return J.value, g, dp.value, dt.value

    def population_bytes(self) -> int:
        return int(load().lbm_population_bytes(self._h))

    def populations(self) -> np.ndarray:
        dt = np.float64 if self.precision == LBM_FP64 else np.float32
        out = np.empty((self.L, self.Q, self.N), dtype=dt)
        self._check(load().lbm_get_populations(self._h, out.ctypes.data, out.nbytes, 0), "lbm_get_populations")
        return out

    def set_populations(self, p: np.ndarray):
        dt = np.float64 if self.precision == LBM_FP64 else np.float32
        a = np.ascontiguousarray(np.asarray(p, dtype=dt)).reshape(self.L, self.Q, self.N)
        self._check(load().lbm_set_populations(self._h, a.ctypes.data, a.nbytes, 0), "lbm_set_populations")

    def get_columns(self, x0: int, ncols: int, out):
        """Populations of the x columns [x0, x0 + ncols) into `out`, a
        contiguous [L, Q, nz, ny, ncols] buffer of the context's precision:
        a CUDA tensor (asynchronous on the context's stream), or a numpy
        array or CPU tensor (lbm_get_columns)."""
        _require_contiguous(out)
        dev = int(bool(getattr(out, "is_cuda", False)))
        nb = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        self._check(load().lbm_get_columns(self._h, int(x0), int(ncols), _addr(out), nb, dev), "lbm_get_columns")
        return out

    def set_columns(self, x0: int, data):
        """Overwrite the x columns [x0, x0 + ncols) from a contiguous
        [L, Q, nz, ny, ncols] buffer (lbm_set_columns)."""
        _require_contiguous(data)
        dev = int(bool(getattr(data, "is_cuda", False)))
        ncols = data.shape[-1]
        nb = data.nbytes if isinstance(data, np.ndarray) else data.numel() * data.element_size()
        self._check(load().lbm_set_columns(self._h, int(x0), int(ncols), _addr(data), nb, dev), "lbm_set_columns")

    def step_host(self, src, dst, n: int = 1):
        """Streaming step on a host-resident state (lbm_step_host): src and dst
        are host buffers of population_bytes() (numpy arrays, page-locked torch
        tensors or addresses).  Asynchronous: keep both alive and call sync()
        before reading dst."""
        self._check(load().lbm_step_host(self._h, _addr(src), _addr(dst), n), "lbm_step_host")

    def save(self) -> bytes:
        """Checkpoint image of the evolving state (populations, coverages, steps taken)."""
        n = ctypes.c_size_t(0)
        self._check(load().lbm_save(self._h, None, ctypes.byref(n)), "lbm_save")
        buf = np.empty(n.value, dtype=np.uint8)
        self._check(load().lbm_save(self._h, buf.ctypes.data, ctypes.byref(n)), "lbm_save")
        return buf.tobytes()

    def load_state(self, image: bytes):
        """Resume from an image written by save() of a context with the same configuration."""
        buf = np.frombuffer(image, dtype=np.uint8)
        self._check(load().lbm_load(self._h, buf.ctypes.data, buf.nbytes), "lbm_load")

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.lbm_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


class Batch(Lattice):
    """Many independent D2Q9 lattices in one context (``lbm_create_batch``):
    stepped together by persistent kernels over one tile work list, replayed
    from CUDA graphs.  Per-node outputs come back as one array per case."""

    def __init__(self, workloads, precision: int = LBM_FP32, stream=None, kappa_threshold: float = 0.0):
        L = load()
        self.wls = list(workloads)
        self.wl = self.wls[0]
        self.precision = precision
        cfgs = (LbmConfig * len(self.wls))()
        keep = []
        st = stream if stream is not None else _current_stream()
        for c, wl in enumerate(self.wls):
            cfg, k = make_config(wl, precision, st, kappa_threshold)
            cfgs[c] = cfg
            keep.append(k)
        h = ctypes.c_void_p()
        rc = L.lbm_create_batch(ctypes.byref(h), len(self.wls), cfgs)
        if rc != LBM_OK:
            raise LbmError(f"lbm_create_batch failed ({rc}): {L.lbm_last_error(None).decode()}")
        self._h = h
        info = np.zeros(5)
        L.lbm_info(h, info.ctypes.data_as(_dp))
        self.L, self.Q, self.D = int(info[2]), int(info[3]), int(info[4])
        self.M = self.wl.M
        self.sizes = [wl.N for wl in self.wls]
        self.N = int(sum(self.sizes))
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(int)
        self.dts, self.cvels = [], []
        ci = np.zeros(6)
        for c in range(len(self.wls)):
            self._check(L.lbm_case_info(h, c, ci.ctypes.data_as(_dp)), "lbm_case_info")
            self.dts.append(float(ci[0]))
            self.cvels.append(float(ci[1]))
        self.dt, self.cvel = self.dts[0], self.cvels[0]
        del keep

    def moments(self, which: int):
        """One array per case, each in the single-lattice layout."""
        shapes = [tuple(n if d == self.N else d for d in self.moment_shape(which)) for n in self.sizes]
        flat = np.empty(sum(int(np.prod(s)) for s in shapes))
        self._check(load().lbm_moments(self._h, which, flat.ctypes.data, flat.nbytes, 0), "lbm_moments")
        out, k = [], 0
        for s in shapes:
            n = int(np.prod(s))
            out.append(flat[k:k + n].reshape(s))
            k += n
        return out

    def populations(self):
        dt = np.float64 if self.precision == LBM_FP64 else np.float32
        flat = np.empty(self.L * self.Q * self.N, dtype=dt)
        self._check(load().lbm_get_populations(self._h, flat.ctypes.data, flat.nbytes, 0), "lbm_get_populations")
        out = []
        for c, n in enumerate(self.sizes):
            o = self.offsets[c] * self.L * self.Q
            out.append(flat[o:o + self.L * self.Q * n].reshape(self.L, self.Q, n))
        return out

    def set_populations(self, pops):
        dt = np.float64 if self.precision == LBM_FP64 else np.float32
        flat = np.concatenate([np.asarray(p, dtype=dt).reshape(-1) for p in pops])
        self._check(load().lbm_set_populations(self._h, flat.ctypes.data, flat.nbytes, 0), "lbm_set_populations")

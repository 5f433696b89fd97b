"""The C-ABI library loads and exports every function include/lbm.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?[\s\*])(lbm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_create", "lbm_step", "lbm_moments", "lbm_destroy", "lbm_sync", "lbm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2409_02930_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2409_02930_gb300 import lbm
    saved = lbm._lib
    lbm._lib = None
    try:
        with pytest.raises(lbm.LbmError):
            lbm.load(str(tmp_path / "missing.so"))
    finally:
        lbm._lib = saved


def _no_gpu():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


@pytest.mark.skipif(not _no_gpu(), reason="argument checks are exercised without a GPU; the GPU tests cover the step")
@pytest.mark.parametrize("case", ["reservoir_without_composition", "one_periodic_face", "theta_at_1",
                                  "non_positive_mass", "surface_mechanism", "wall_on_one_column", "three_d"])
def test_noalloc_entry_point_checks_the_configuration_like_create(case):
    """lbm_step_noalloc rejects, before it touches the GPU, every configuration
    lbm_create rejects (the per-node input arrays aside), and a surface
    mechanism, which its two-pass D2Q9 step does not carry."""
    from paper_2409_02930_gb300 import build, lbm, workloads as W
    lib = ctypes.CDLL(build.build())
    lib.lbm_step_noalloc.restype = ctypes.c_int
    wl = W.adjoint_slab(nx=16, ny=8, steps=1)
    if case == "one_periodic_face":
        wl.bc_hi = W.BC_PERIODIC
    elif case == "theta_at_1":
        wl.theta_max = 1.0
    elif case == "non_positive_mass":
        wl.molar_mass = wl.molar_mass.copy()
        wl.molar_mass[1] = 0.0
    elif case == "wall_on_one_column":
        wl.nx = 1
        wl.bc_lo = wl.bc_hi = W.BC_BOUNCEBACK
    elif case == "three_d":
        wl.nz = 2
    cfg, keep = lbm.make_config(wl, lbm.LBM_FP64, ctypes.c_void_p(0))
    if case == "reservoir_without_composition":
        cfg.X_in_lo = None
    if case == "surface_mechanism":
        cfg.S = 2
    dummy = [ctypes.c_void_p(0x1000 * k) for k in (1, 2, 3, 4)]
    rc = lib.lbm_step_noalloc(ctypes.byref(cfg), *dummy)
    assert rc == lbm.LBM_ERR_ARG

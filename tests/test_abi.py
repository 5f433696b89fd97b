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

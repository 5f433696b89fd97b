"""The entry point that allocates nothing (lbm_step_noalloc), on the GPU.

It serves callers that cannot allocate device memory while they run -- a
framework that owns every device byte through its own pool, or a loop where a
cudaMalloc would stall the device.  The caller passes its own device state;
the step's scratch lives in a fixed array inside the library.  This test
calls it twice in a row through the C ABI and checks both results against the
regular context entry point (lbm_step), within the parity tolerances of the
other tests (1e-12 for FP64, 1e-5 for FP32).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2409_02930_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _field_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_step_matches_context_step_twice(precision, tol):
    torch = pytest.importorskip("torch")
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    prec = lbm.LBM_FP64 if precision == "fp64" else lbm.LBM_FP32
    tdt = torch.float64 if precision == "fp64" else torch.float32
    dev = torch.device("cuda", 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    wl = W.adjoint_slab(nx=48, ny=32, steps=2)          # reservoir faces, energy on, 3 species
    ref = lbm.Lattice(wl, precision=prec, stream=stream)
    p0 = ref.populations()
    a = torch.from_numpy(p0.copy()).to(dev)
    b = torch.empty_like(a)
    phi = torch.tensor(wl.porosity, dtype=tdt, device=dev)
    t_fixed = torch.tensor(wl.T_init, dtype=tdt, device=dev)
    assert (4 + wl.M) * wl.N * a.element_size() <= lbm.load().lbm_noalloc_scratch_limit()

    # call 1: a -> b, compared with one regular step
    rc = lbm.step_noalloc(wl, a.data_ptr(), b.data_ptr(), phi.data_ptr(), t_fixed.data_ptr(), prec, stream)
    assert rc == lbm.LBM_OK
    ref.step(1)
    torch.cuda.synchronize()
    r1 = ref.populations()
    g1 = b.cpu().numpy()
    for l in range(r1.shape[0]):
        assert _field_err(g1[l], r1[l]) < tol, ("call 1", l)

    # call 2: b -> a (the scratch array keeps the first call's contents)
    rc = lbm.step_noalloc(wl, b.data_ptr(), a.data_ptr(), phi.data_ptr(), t_fixed.data_ptr(), prec, stream)
    assert rc == lbm.LBM_OK
    ref.step(1)
    torch.cuda.synchronize()
    r2 = ref.populations()
    g2 = a.cpu().numpy()
    for l in range(r2.shape[0]):
        assert _field_err(g2[l], r2[l]) < tol, ("call 2", l)
    ref.close()


def test_noalloc_rejects_lattices_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    from paper_2409_02930_gb300 import lbm
    limit = lbm.load().lbm_noalloc_scratch_limit()
    side = int(np.sqrt(limit / (7 * 8))) + 64          # FP64, M = 3: (4 + 3) * N * 8 bytes > limit
    wl = W.slab(nx=side, ny=side, steps=1)
    dev = torch.device("cuda", 0)
    x = torch.empty(8, dtype=torch.float64, device=dev)
    rc = lbm.step_noalloc(wl, x.data_ptr(), x.data_ptr() + 8, x.data_ptr(), x.data_ptr(), lbm.LBM_FP64)
    assert rc == lbm.LBM_ERR_ARG

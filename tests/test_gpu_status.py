"""Failure detection on the GPU, without a GPU fault: the status word of the
step (include/lbm.h, lbm_sync) reports a non-finite state and a bounded wait
that gave up, and the context stays usable for the host to read it."""
import ctypes

import numpy as np
import pytest

from paper_2409_02930_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    return lbm


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_population_reports_numeric_error(L, precision):
    """A NaN written from the host into one population of one node: the next
    step sees a non-finite density there and lbm_sync returns
    LBM_ERR_NUMERIC; a clean context of the same lattice returns LBM_OK."""
    prec = L.LBM_FP64 if precision == "fp64" else L.LBM_FP32
    wl = W.slab(nx=64, ny=24, steps=2)
    clean = L.Lattice(wl, precision=prec)
    clean.step(2)
    assert L.load().lbm_sync(clean._h) == L.LBM_OK
    clean.close()
    g = L.Lattice(wl, precision=prec)
    p = g.populations()
    p[1, 3, 5 * wl.nx + 7] = np.nan
    g.set_populations(p)
    g.step(1)
    assert L.load().lbm_sync(g._h) == L.LBM_ERR_NUMERIC
    # the context still answers: its error text and a read of its moments
    assert b"non-finite" in L.load().lbm_last_error(g._h)
    g.moments(L.LBM_MOM_RHO)
    g.close()


def test_row_wait_that_gives_up_reports_timeout(L):
    """The default form of a 512 x 512 periodic lattice stages its rows with
    bulk tensor copies on mbarriers.  With the wait bound set to 0 probes
    every staged row wait gives up at once: the blocks stop, drain the copies
    already in flight under their own bound and lbm_sync returns
    LBM_ERR_TIMEOUT.  With the default bound the same step is clean."""
    wl = W.slab(nx=512, ny=512, steps=1)
    g = L.Lattice(wl, precision=L.LBM_FP32)
    assert g.variant() in (8, 9)                       # the TMA row march
    g.step(1)
    assert L.load().lbm_sync(g._h) == L.LBM_OK
    g.set_wait_limit(0)
    g.step(1)
    assert L.load().lbm_sync(g._h) == L.LBM_ERR_TIMEOUT
    assert b"wait" in L.load().lbm_last_error(g._h)
    g.close()
    # a fresh context on the same device still steps cleanly
    h = L.Lattice(wl, precision=L.LBM_FP32)
    h.step(2)
    assert L.load().lbm_sync(h._h) == L.LBM_OK
    h.close()


def test_noalloc_step_reports_nonfinite_state(L):
    """lbm_step_noalloc returns the step's status: LBM_ERR_NUMERIC for a state
    with a NaN population."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    wl = W.adjoint_slab(nx=48, ny=32, steps=1)
    ref = L.Lattice(wl, precision=L.LBM_FP64, stream=stream)
    p0 = ref.populations()
    ref.close()
    p0[0, 4, 10] = np.nan
    a = torch.from_numpy(p0).to(dev)
    b = torch.empty_like(a)
    phi = torch.tensor(wl.porosity, dtype=torch.float64, device=dev)
    t_fixed = torch.tensor(wl.T_init, dtype=torch.float64, device=dev)
    rc = L.step_noalloc(wl, a.data_ptr(), b.data_ptr(), phi.data_ptr(), t_fixed.data_ptr(), L.LBM_FP64, stream)
    assert rc == L.LBM_ERR_NUMERIC

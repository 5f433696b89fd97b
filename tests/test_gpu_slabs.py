"""The x-slab decomposition (paper_2409_02930_gb300/slabs.py) stepping each
slab with its own library context on the GPU, all slabs in one process with
the in-process halo exchange, against the undivided lattice on the GPU: node
for node within the FP64 parity bound."""
import numpy as np
import pytest

from paper_2409_02930_gb300 import slabs as S
from paper_2409_02930_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    return lbm


@pytest.mark.parametrize("name", ["periodic", "reservoir"])
def test_gpu_slabs_equal_the_whole_lattice(L, name):
    torch = pytest.importorskip("torch")
    wl = (W.slab(nx=64, ny=40, steps=60, name="periodic_slab") if name == "periodic"
          else W.adjoint_slab(nx=64, ny=40, steps=60))
    run = S.SlabRun(wl, 3, range(3), lambda w: S.LatticeStepper(w, L.LBM_FP64), S.LocalExchange())
    run.step(wl.steps)
    g = L.Lattice(wl, precision=L.LBM_FP64)
    g.step(wl.steps)
    whole = g.populations().reshape(g.L, g.Q, 1, wl.ny, wl.nx)
    scale = np.abs(whole).max()
    for k, s in enumerate(run.slabs):
        mine = run.owned(run.steppers[k].get_state().cpu().numpy(), k)
        err = np.max(np.abs(mine - whole[..., s.x0:s.x1])) / scale
        assert err < 1e-12, (k, err)
    torch.cuda.synchronize()

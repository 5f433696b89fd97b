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
        mine = run.owned(run.steppers[k].g.populations(), k)
        err = np.max(np.abs(mine - whole[..., s.x0:s.x1])) / scale
        assert err < 1e-12, (k, err)
    torch.cuda.synchronize()


def test_column_copies_match_the_populations(L):
    """lbm_get_columns / lbm_set_columns against slices of the whole state,
    to and from device tensors and host arrays, FP32 and FP64, on a 2-D and
    a 3-D lattice; columns outside the range are left untouched."""
    torch = pytest.importorskip("torch")
    for wl, prec in ((W.slab(nx=37, ny=9, steps=3), L.LBM_FP64), (W.slab(nx=37, ny=9, steps=3), L.LBM_FP32),
                     (W.anode3d(nx=11, ny=5, nz=4, steps=3), L.LBM_FP32)):
        g = L.Lattice(wl, precision=prec)
        g.step(3)
        g.sync()
        whole = g.populations().reshape(g.L, g.Q, wl.nz, wl.ny, wl.nx)
        dt = torch.float64 if prec == L.LBM_FP64 else torch.float32
        for x0, n in ((0, 2), (wl.nx - 2, 2), (5, 3), (0, wl.nx)):
            dev = torch.empty((g.L, g.Q, wl.nz, wl.ny, n), dtype=dt, device="cuda")
            g.get_columns(x0, n, dev)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(dev.cpu().numpy(), whole[..., x0:x0 + n])
            host = np.empty((g.L, g.Q, wl.nz, wl.ny, n), dtype=whole.dtype)
            g.get_columns(x0, n, host)
            np.testing.assert_array_equal(host, whole[..., x0:x0 + n])
        new = np.ascontiguousarray(whole[..., 3:5] * 1.5)
        g.set_columns(3, torch.from_numpy(new).cuda())
        torch.cuda.synchronize()
        after = g.populations().reshape(whole.shape)
        np.testing.assert_array_equal(after[..., 3:5], new)
        np.testing.assert_array_equal(after[..., :3], whole[..., :3])
        np.testing.assert_array_equal(after[..., 5:], whole[..., 5:])
        g.set_columns(8, np.ascontiguousarray(whole[..., 8:9] * 0.5))
        np.testing.assert_array_equal(g.populations().reshape(whole.shape)[..., 8], whole[..., 8] * 0.5)
        with pytest.raises(L.LbmError):
            g.get_columns(wl.nx - 1, 2, host)
        g.close()

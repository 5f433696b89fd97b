"""Streaming steps on host-resident states (lbm_step_host): every call's
output equals uploading its input, stepping it and downloading it with the
synchronous calls, bit for bit, while consecutive calls overlap on the
upload, compute and download streams; the context's own state is left as it
was."""
import numpy as np
import pytest

from paper_2409_02930_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    return lbm


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_stream_matches_synchronous_calls(L, prec, n):
    import torch
    precision = L.LBM_FP32 if prec == "fp32" else L.LBM_FP64
    wl = W.slab(nx=64, ny=32, steps=20)
    # five different states as inputs
    src = L.Lattice(wl, precision=precision)
    inputs = []
    for _ in range(5):
        inputs.append(src.populations())
        src.step(3)
    src.close()
    ref = L.Lattice(wl, precision=precision)
    expected = []
    for p in inputs:
        ref.set_populations(p)
        ref.step(n)
        expected.append(ref.populations())
    ref.close()
    g = L.Lattice(wl, precision=precision)
    own = g.populations()
    dt = torch.float32 if precision == L.LBM_FP32 else torch.float64
    hin = [torch.from_numpy(p.copy()).pin_memory() for p in inputs]
    hout = [torch.empty(p.shape, dtype=dt).pin_memory() for p in inputs]
    for a, b in zip(hin, hout):
        g.step_host(a, b, n)
    g.sync()
    for k, (b, e) in enumerate(zip(hout, expected)):
        assert np.array_equal(b.numpy().view(np.uint8), e.view(np.uint8)), k
    assert np.array_equal(g.populations(), own)
    g.close()


def test_stream_refuses_batches_and_reactive_lattices(L):
    import torch
    b = L.Batch(W.capillary_batch(n_cases=2, seed=11, nmin=16, nmax=32, steps=10), precision=L.LBM_FP32)
    buf = torch.empty(b.population_bytes(), dtype=torch.uint8).pin_memory()
    with pytest.raises(L.LbmError):
        b.step_host(buf, buf, 1)
    b.close()
    r = L.Lattice(W.anode3d_reactive(nx=8, ny=4, nz=4, steps=2, name="anode3d_reactive_8x4x4"),
                  precision=L.LBM_FP32)
    buf = torch.empty(r.population_bytes(), dtype=torch.uint8).pin_memory()
    with pytest.raises(L.LbmError):
        r.step_host(buf, buf, 1)
    r.close()

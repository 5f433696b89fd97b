"""Checkpoint and resume through lbm_save / lbm_load: a run resumed from an
image continues bit for bit like the run that wrote it (populations and, on
reactive lattices, the surface coverages), and images that do not match the
context are refused without touching its state."""
import struct

import numpy as np
import pytest

from paper_2409_02930_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    return lbm


def header(image):
    assert image[:8] == b"LBMSTATE"
    return struct.unpack("<10q", image[8:88])


def flat(p):
    # a batch returns one population array per case
    if isinstance(p, list):
        return np.concatenate([x.reshape(-1) for x in p])
    return p.reshape(-1)


def resume_matches(make, n1, n2):
    a = make()
    a.step(n1)
    image = a.save()
    a.step(n2)
    pa = flat(a.populations())
    b = make()
    b.load_state(image)
    b.step(n2)
    pb = flat(b.populations())
    assert np.array_equal(pa.view(np.uint8), pb.view(np.uint8))
    return a, b, image


def test_slab_fp32_resume_is_bitwise(L):
    wl = W.slab(nx=64, ny=32, steps=50)
    a, b, image = resume_matches(lambda: L.Lattice(wl, precision=L.LBM_FP32), 20, 30)
    h = header(image)
    assert h[0] == 1 and h[1] == L.LBM_FP32 and h[3] == wl.N and h[7] == 20
    assert len(image) == 128 + a.population_bytes()
    assert header(b.save())[7] == 50
    a.close()
    b.close()


def test_reactive_resume_carries_coverages(L):
    wl = W.anode3d_reactive(nx=16, ny=8, nz=8, steps=6, name="anode3d_reactive_16x8x8")
    a, b, image = resume_matches(lambda: L.Lattice(wl, precision=L.LBM_FP32), 3, 3)
    h = header(image)
    S = wl.mechanism.S
    assert h[6] == S > 0 and h[9] == S * wl.N * 8
    xa = a.moments(L.LBM_MOM_XS)
    xb = b.moments(L.LBM_MOM_XS)
    assert np.array_equal(xa, xb)
    a.close()
    b.close()


def test_batch_fp64_resume_is_bitwise(L):
    wls = W.capillary_batch(n_cases=4, seed=11, nmin=16, nmax=64, steps=100)
    a, b, _ = resume_matches(lambda: L.Batch(wls, precision=L.LBM_FP64), 60, 40)
    a.close()
    b.close()


def test_mismatched_images_are_refused(L):
    a = L.Lattice(W.slab(nx=64, ny=32, steps=10), precision=L.LBM_FP32)
    a.step(2)
    image = a.save()
    other = L.Lattice(W.slab(nx=32, ny=32, steps=10), precision=L.LBM_FP32)
    before = other.populations()
    with pytest.raises(L.LbmError):
        other.load_state(image)                      # another lattice size
    with pytest.raises(L.LbmError):
        other.load_state(image[:-4])                 # truncated
    bad = bytearray(image)
    bad[0:8] = b"NOTSTATE"
    with pytest.raises(L.LbmError):
        a.load_state(bytes(bad))                     # not an image
    f64 = L.Lattice(W.slab(nx=64, ny=32, steps=10), precision=L.LBM_FP64)
    with pytest.raises(L.LbmError):
        f64.load_state(image)                        # another precision
    assert np.array_equal(other.populations(), before)
    for g in (a, other, f64):
        g.close()

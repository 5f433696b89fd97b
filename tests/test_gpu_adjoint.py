"""Adjoint form (lbm_adjoint): gradients of a plane flux after n steps with
respect to the porosity field, the pore radius and the tortuosity.

* FP64 adjoint against the oracle's exact directional derivatives (forward-
  mode dual numbers through the whole time loop) on small lattices with
  reservoir, bounce-back and periodic faces, M = 3 with energy and M = 2
  isothermal; and against the oracle's full gradient (every node's
  porosity) on a tiny lattice.
* At the adjoint workload's full size (256 x 256, 1000 steps, checkpoints
  every 50) the FP32 and FP64 adjoints against FP64 central differences on
  16 random directions.
* The torch.autograd.Function returns the same gradients.
"""
import numpy as np
import pytest

import oracle
from paper_2409_02930_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2409_02930_gb300 import lbm
    lbm.load()
    return lbm


def plane_flux(o, wl, lane=None):
    j = o.moments(oracle.MOM_J_A, lane=lane).reshape(wl.M, 2, wl.ny, wl.nx)
    return float(j[0, 0, :, wl.nx - 2].sum())


def oracle_jvps(wl, steps, V=None, pore=False, tort=False):
    """Exact directional derivatives: rows of V (porosity directions), then
    d/d ln r_p and d/d ln tau when requested."""
    K = oracle.LANES
    rows = [] if V is None else list(V)
    extra = (["pore"] if pore else []) + (["tort"] if tort else [])
    out, J = [], None
    dirs = [("phi", v) for v in rows] + [(e, None) for e in extra]
    for c0 in range(0, len(dirs), K):
        chunk = dirs[c0:c0 + K]
        dphi = np.zeros((K, wl.N))
        dpore = np.zeros(K)
        dtort = np.zeros(K)
        for k, (kind, v) in enumerate(chunk):
            if kind == "phi":
                dphi[k] = v
            elif kind == "pore":
                dpore[k] = wl.pore_radius
            else:
                dtort[k] = wl.tortuosity
        o = oracle.Oracle(wl, dual=True)
        o.set_tangents(dphi=dphi, dpore=dpore, dtort=dtort)
        o.step(steps)
        J = plane_flux(o, wl)
        out += [plane_flux(o, wl, lane=k) for k in range(len(chunk))]
    return J, np.array(out)


def small(kind, steps):
    if kind == "inlet_m3":
        return W.adjoint_slab(nx=14, ny=10, steps=steps, name="adjoint_slab_14x10")
    if kind == "bounceback_m3":
        wl = W.slab(nx=12, ny=10, steps=steps, name="bb_slab_12x10")
        wl.bc_lo = wl.bc_hi = W.BC_BOUNCEBACK
        return wl
    if kind == "periodic_m3":
        return W.slab(nx=12, ny=10, steps=steps, name="periodic_slab_12x10")
    if kind == "capillary_m2":
        return W.capillary(nx=24, ny=4, steps=steps, name="capillary_24x4")
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["inlet_m3", "bounceback_m3", "periodic_m3", "capillary_m2"])
def test_fp64_adjoint_matches_oracle_jvps(L, kind):
    steps, ckpt = 30, 7
    wl = small(kind, steps)
    rng = np.random.default_rng(3)
    V = rng.normal(size=(6, wl.N))
    Jo, jv = oracle_jvps(wl, steps, V, pore=True, tort=True)
    g = L.Lattice(wl, precision=L.LBM_FP64)
    J, gphi, gpore, gtort = g.adjoint(steps, ckpt)
    assert abs(J - Jo) <= 1e-12 * abs(Jo), (J, Jo)
    adj = np.concatenate([V @ gphi, [gpore * wl.pore_radius, gtort * wl.tortuosity]])
    scale = np.max(np.abs(jv))
    err = np.max(np.abs(adj - jv)) / scale
    print(kind, "FP64 adjoint vs oracle JVPs: max rel error %.2e" % err)
    assert err < 1e-9, (adj, jv)
    # pore radius and tortuosity enter through their ratio
    assert abs(gpore * wl.pore_radius + gtort * wl.tortuosity) <= 1e-12 * max(abs(gtort * wl.tortuosity), 1e-300)


def test_fp64_adjoint_full_gradient_matches_oracle(L):
    """Every node's dJ/dphi on an 8 x 6 lattice with reservoirs: the oracle's
    gradient by forward mode along every coordinate direction."""
    steps = 20
    wl = W.adjoint_slab(nx=8, ny=6, steps=steps, name="adjoint_slab_8x6")
    Jo, jv = oracle_jvps(wl, steps, np.eye(wl.N))
    g = L.Lattice(wl, precision=L.LBM_FP64)
    J, gphi, _, _ = g.adjoint(steps, 6)
    err = np.max(np.abs(gphi - jv)) / np.max(np.abs(jv))
    print("full gradient: max rel error %.2e" % err)
    assert err < 1e-9


def test_fp32_adjoint_matches_fp64_adjoint_small(L):
    steps = 60
    wl = small("inlet_m3", steps)
    a = L.Lattice(wl, precision=L.LBM_FP64).adjoint(steps, 10)
    b = L.Lattice(wl, precision=L.LBM_FP32).adjoint(steps, 10)
    e = np.max(np.abs(b[1] - a[1])) / np.max(np.abs(a[1]))
    print("FP32 vs FP64 adjoint gradient: %.2e" % e)
    assert abs(b[0] - a[0]) <= 1e-4 * abs(a[0])
    assert e < 1e-4            # measured 2.0e-6


def test_autograd_function(L):
    torch = pytest.importorskip("torch")
    from paper_2409_02930_gb300.autograd import outlet_flux
    steps = 20
    wl = small("inlet_m3", steps)
    phi = torch.tensor(wl.porosity, dtype=torch.float64, requires_grad=True)
    rp = torch.tensor(wl.pore_radius, dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(wl.tortuosity, dtype=torch.float64, requires_grad=True)
    J = outlet_flux(phi, rp, tau, wl, precision=L.LBM_FP64, steps=steps, ckpt_every=5)
    (2.0 * J).backward()
    ref = L.Lattice(wl, precision=L.LBM_FP64).adjoint(steps, 5)
    assert abs(J.item() - ref[0]) <= 1e-14 * abs(ref[0])
    assert np.allclose(phi.grad.numpy(), 2.0 * ref[1], rtol=0, atol=1e-14 * np.max(np.abs(ref[1])))
    assert abs(rp.grad.item() - 2.0 * ref[2]) <= 1e-12 * abs(ref[2])
    assert abs(tau.grad.item() - 2.0 * ref[3]) <= 1e-12 * abs(ref[3])


def test_full_size_adjoint_against_central_differences(L):
    """256 x 256 three-species slab with reservoirs, 1000 steps, checkpoints
    every 50: FP32 and FP64 adjoint gradients along 16 random porosity
    directions against FP64 central differences of the GPU forward run."""
    wl = W.adjoint_slab()
    steps = wl.steps
    rng = np.random.default_rng(21)
    V = rng.normal(size=(16, wl.N)) * 0.01
    g64 = L.Lattice(wl, precision=L.LBM_FP64)
    J64, gphi64, gp64, gt64 = g64.adjoint(steps, 50)
    g64.close()
    g32 = L.Lattice(wl, precision=L.LBM_FP32)
    J32, gphi32, gp32, gt32 = g32.adjoint(steps, 50)
    g32.close()
    eps = 1e-4

    def J_at(phi):
        w = W.adjoint_slab()
        w.porosity = phi
        g = L.Lattice(w, precision=L.LBM_FP64)
        g.set_variant(-1)
        g.step(steps)
        j = g.moments(L.LBM_MOM_J_A).reshape(w.M, 2, w.ny, w.nx)
        g.close()
        return float(j[0, 0, :, w.nx - 2].sum())

    fd = np.array([(J_at(wl.porosity + eps * v) - J_at(wl.porosity - eps * v)) / (2 * eps) for v in V])
    a64 = V @ gphi64
    a32 = V @ gphi32
    scale = np.max(np.abs(fd))
    e64 = np.max(np.abs(a64 - fd)) / scale
    e32 = np.max(np.abs(a32 - fd)) / scale
    print("full size: J64 %.6e J32 %.6e; adjoint vs central differences: FP64 %.2e FP32 %.2e" % (J64, J32, e64, e32))
    assert e64 < 1e-6          # measured 3.0e-9 (central-difference truncation)
    assert e32 < 1e-4          # measured 2.0e-6

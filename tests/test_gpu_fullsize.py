"""Parity at the benchmark sizes, in the launch configurations the benchmark
times, against the FP64 oracle run on the host cores.

* 512 x 512 slab, FP32, the autotuned kernel form: 200 steps.
* 64-capillary sweep (0.30 M nodes), FP64 batch, CUDA-graph replay: 100
  steps, every case to 1e-12.
* 256 x 128 x 128 anode, six species, FP32, the default form (staged with a
  gradient pass): 3 steps.
* the same anode with the surface mechanism, FP32: 1 step.

The oracle needs about 20 GB of host memory for the anode and a few minutes
on 16 cores for all four.
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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def flux_err(L, g, o, wl):
    """Species-flux error against the scale max rho_a sqrt(R_a T) (FP32
    populations resolve fluxes to ~eps rho c_s)."""
    rho = o.moments(oracle.MOM_RHO_A)
    theta = 8.314462618 * o.moments(oracle.MOM_T)[None, :] / wl.molar_mass[:, None] / g.cvel ** 2
    scale = np.max(rho * np.sqrt(theta))
    return float(np.max(np.abs(g.moments(L.LBM_MOM_J_A) - o.moments(oracle.MOM_J_A))) / scale)


def test_slab_512_fp32_autotuned(L):
    wl = W.slab(512, 512, steps=200)
    g = L.Lattice(wl, precision=L.LBM_FP32)
    g.autotune(3)
    g.close()
    g = L.Lattice(wl, precision=L.LBM_FP32)
    g.step(wl.steps)
    g.sync()
    o = oracle.Oracle(wl)
    o.step(wl.steps)
    e = rel(g.moments(L.LBM_MOM_RHO_A), o.moments(oracle.MOM_RHO_A))
    ef = flux_err(L, g, o, wl)
    eT = rel(g.moments(L.LBM_MOM_T), o.moments(oracle.MOM_T))
    print("slab 512x512 FP32, 200 steps: densities %.2e, fluxes %.2e, T %.2e" % (e, ef, eT))
    assert e < 1e-5 and ef < 1e-5 and eT < 1e-5


def oracle_sensitivity(wl, steps, moments):
    """How far the oracle moves from itself when its initial populations are
    perturbed at the rounding level (1e-16 relative): the rounding
    sensitivity of the discrete method on this case (the trace-species switch
    of reading R11 turns rounding differences into small jumps)."""
    a = oracle.Oracle(wl)
    b = oracle.Oracle(wl)
    p = b.pops()
    b.set_pops(p * (1 + 1e-16 * np.random.default_rng(0).standard_normal(p.shape)))
    a.step(steps)
    b.step(steps)
    return {k: (a.moments(getattr(oracle, "MOM_" + k)), b.moments(getattr(oracle, "MOM_" + k))) for k in moments}


def test_batch_64_capillaries_fp64(L):
    """Every case within the FP64 bound 1e-12, or within ten times the
    oracle's own rounding sensitivity on that case when that is larger
    (some low-pressure capillaries move 7e-12 from a 1e-16 perturbation).
    Densities field-relative; species fluxes against max rho_a x lattice
    speed; velocity in lattice units.  The worst population error is
    reported."""
    wls = W.capillary_batch()
    b = L.Batch(wls, precision=L.LBM_FP64)
    b.step(100)                       # two graph replays
    b.sync()
    pops = b.populations()
    keys = ("RHO_A", "J_A", "RHO", "U")
    mom = {k: b.moments(getattr(L, "LBM_MOM_" + k)) for k in keys}

    def errs(x, ref):
        return {"RHO_A": rel(x["RHO_A"], ref["RHO_A"]), "RHO": rel(x["RHO"], ref["RHO"]),
                "J_A": float(np.max(np.abs(x["J_A"] - ref["J_A"])) / np.max(ref["RHO_A"])),
                "U": float(np.max(np.abs(x["U"] - ref["U"])))}

    worst_ratio, worst, worst_p = 0.0, None, 0.0
    for c, wl in enumerate(wls):
        pairs = oracle_sensitivity(wl, 100, keys)
        ref = {k: v[0] for k, v in pairs.items()}
        sens = errs({k: v[1] for k, v in pairs.items()}, ref)
        e = errs({k: mom[k][c] for k in keys}, ref)
        for k in keys:
            bound = max(1e-12, 10.0 * sens[k])
            if e[k] / bound > worst_ratio:
                worst_ratio, worst = e[k] / bound, (c, k, e[k], sens[k])
        o = oracle.Oracle(wl)
        o.step(100)
        po = o.pops()
        for l in range(b.L):
            worst_p = max(worst_p, rel(pops[c][l], po[l]))
    print("64 capillaries FP64, 100 steps: worst (case, moment, error, oracle sensitivity)", worst,
          "ratio to bound %.3f" % worst_ratio, "worst population error %.2e" % worst_p)
    assert worst_ratio < 1.0, worst


def test_anode_full_size_fp32_default_form(L):
    """The form bench.py times: the staged form with a gradient pass."""
    wl = W.anode3d(steps=3)
    g = L.Lattice(wl, precision=L.LBM_FP32)
    assert g.variant() == 5
    g.step(wl.steps)
    g.sync()
    o = oracle.Oracle(wl)
    o.step(wl.steps)
    e = rel(g.moments(L.LBM_MOM_RHO_A), o.moments(oracle.MOM_RHO_A))
    ef = flux_err(L, g, o, wl)
    print("anode 256x128x128 FP32 (gradient-pass form), 3 steps: densities %.2e, fluxes %.2e" % (e, ef))
    assert e < 1e-5 and ef < 1e-5


def test_reactive_anode_full_size_fp32(L):
    wl = W.anode3d_reactive(steps=1)
    g = L.Lattice(wl, precision=L.LBM_FP32)
    g.step(1)
    g.sync()
    o = oracle.Oracle(wl)
    o.step(1)
    e = rel(g.moments(L.LBM_MOM_RHO_A), o.moments(oracle.MOM_RHO_A))
    xs = np.max(np.abs(g.moments(L.LBM_MOM_XS) - o.moments(oracle.MOM_XS)))
    print("reactive anode 256x128x128 FP32, 1 step: densities %.2e, coverages %.2e" % (e, xs))
    assert e < 1e-5 and xs < 1e-8

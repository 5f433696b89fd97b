"""Host-side pieces of bench.py: the algorithmic bytes behind the roofline,
the ncu traffic table it reads, and the reference arm (the oracle on the
host cores), all without a GPU."""
import argparse
import json
import os

import bench
from paper_2409_02930_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_per_node():
    # populations read and written once plus the porosity
    assert bench.algorithmic_bytes_per_node(W.slab(nx=8, ny=8), 4) == 45 * 4 * 2 + 4 == 364
    assert bench.algorithmic_bytes_per_node(W.slab(nx=8, ny=8), 8) == 45 * 8 * 2 + 8   # porosity in FP64 too
    assert bench.algorithmic_bytes_per_node(W.anode3d(nx=4, ny=4, nz=4), 4) == 216 * 4 * 2 + 4
    assert bench.algorithmic_bytes_per_node(W.capillary(nx=8), 4) == 27 * 4 * 2 + 4


def test_traffic_table_entries_parse():
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    with open(path) as f:
        keys = [line.split()[0] for line in f if line.strip() and not line.startswith("#")]
    assert "slab512x512_fp32_variant8" in keys
    for k in keys:
        t = bench.profiled_traffic(k)
        # DRAM bytes per launch against the algorithmic bytes of that lattice
        # (364 per node): at most 2x, and no less than the 47 MB the 512^2
        # step's reads alone need
        side = int(k.split("x")[0].replace("slab", ""))
        alg = 364 * side * side
        assert t is not None and 0.45 * alg < t < 2.0 * alg, (k, t, alg)
    assert bench.profiled_traffic("slab512x512_fp32_variant_unknown") is None


def test_weak_scaling_value():
    # 2 ranks x 1000 nodes x 5 lattices x 10 steps in 20 ms
    assert abs(bench.weak_scaling_value(2, 1000, 5, 10, 20.0) - 5.0) < 1e-12


def test_reference_arm_line():
    args = argparse.Namespace(steps=3, warmup=3, nx=512, ny=512, precision="fp32")
    out = bench.run_reference(args, 1, 0)
    line = json.loads(json.dumps(out))
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert bench.run_reference(args, 2, 1) is None          # other ranks print nothing

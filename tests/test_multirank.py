"""The N > 1 path of bench.py on CPU: gloo ranks on 127.0.0.1 (world size 2).

Every rank runs its own replica (weak scaling, no data-path collective); the
only collectives are the barrier around the timed region and the maximum of
the per-rank times.  The ranks report different times and the job value
must use the slowest one."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        my_ms = 10.0 * (rank + 1)                    # rank 1 is the slow replica
        ms_max = bench.allreduce_max(ws, my_ms)
        value = bench.weak_scaling_value(ws, 1000, 5, 10, ms_max)
        out[rank] = (ms_max, value)
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()      # no fork of a multi-threaded parent
    out = mgr.dict()
    mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
    assert out[0][0] == out[1][0] == 20.0
    # 2 replicas x 1000 nodes x 5 lattices x 10 steps in 20 ms
    assert abs(out[0][1] - 2 * 1000 * 5 * 10 / 0.020 / 1e6) < 1e-12
    assert out[0][1] == out[1][1]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.allreduce_max(1, 3.5) == 3.5
    assert abs(bench.weak_scaling_value(1, 262144, 5, 100, 10.0) - 262144 * 5 * 100 / 0.01 / 1e6) < 1e-9

"""The multi-replica path of bench.py on the CPU: two ranks over gloo (127.0.0.1)
exercise the barrier, the max over ranks and the whole-job throughput (every rank's
units over the slowest rank's time), as the GPU run does over NCCL."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms_local = 2.0 + rank  # rank 1 is the slow one
        value, ms = bench.job_value(1.0e6, ms_local, world)
        out[rank] = (value, ms, bench.max_over_ranks(10.0 * (rank + 1), world))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_gpu_run():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in range(world):
        value, ms, mx = res[rank]
        assert ms == 3.0                       # the slowest rank's time, on every rank
        assert value == pytest.approx(world * 1.0e6 / 3.0e-3)
        assert mx == 20.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_value(5.0e5, 4.0, 1)
    assert ms == 4.0 and value == pytest.approx(5.0e5 / 4.0e-3)

"""The multi-rank path of bench.py (replicas only, no data-path collective) on CPU ranks.

Two gloo ranks time different step lengths; both must report the slowest rank's time and the
whole-job throughput world * units / time, the aggregation bench.py performs under torchrun.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]          # rank 1 is the slow replica
        ms = bench.slowest_rank_ms(local_ms, dist, "cpu")
        out[rank] = (ms, bench.job_throughput(1000, world, ms / 10))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 150.0
    assert value == pytest.approx(2 * 1000 / (15.0 / 1e3))


def test_one_rank_is_itself():
    import bench
    assert bench.slowest_rank_ms(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(300, 1, 3.0) == pytest.approx(1e5)

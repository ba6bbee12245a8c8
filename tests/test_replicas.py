"""Multi-GPU is replicas only: every rank clusters its own matrix, no collective
on the data path; the benchmark takes the slowest rank's time and sums the
work.  This checks that aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # each rank times its own replica; the slowest one bounds the job
        own_ms = [120.0, 150.0][rank]
        worst = bench.max_over_ranks(own_ms, world)
        bench.barrier(world)
        n, steps = 65536, 3
        value = world * steps * (n - 1) / (worst * 1e-3)
        out[rank] = (worst, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] == out[1][1] == pytest.approx(2 * 3 * 65535 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0

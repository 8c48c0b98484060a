"""Multi-GPU form: independent replicas (the path has no exchange step on one
GPU).  The benchmark's whole-job figure is the slowest rank's time over every
rank's steps; this checks that aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, elapsed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    tmax = bench.max_over_ranks(elapsed[rank], dist, "cpu")
    out[rank] = (tmax, bench.replicas_value(5, world, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    world = 2
    elapsed = [1.25, 2.5]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), elapsed, out), nprocs=world, join=True)
    for r in range(world):
        tmax, value = out[r]
        assert tmax == 2.5  # both ranks see the slowest rank's time
        assert value == pytest.approx(world * 5 / 2.5)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(0.75, None, "cpu") == 0.75
    assert bench.replicas_value(4, 1, 2.0) == 2.0

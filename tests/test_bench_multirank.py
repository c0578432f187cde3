"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each, as
torchrun launches them) reduce their step times to the slowest one and report
the whole-job throughput of their replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
    worst = bench.max_over_ranks(ms)
    rate = bench.aggregate_rate(1000, 10, world, worst)
    dist.barrier()
    out[rank] = (worst, rate)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # 2 replicas x 1000 particles x 10 steps in 0.15 s
    assert abs(res[0][1] - 2 * 1000 * 10 / 0.15) < 1e-6


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.aggregate_rate(406000, 100, 1, 64.0) == pytest.approx(406000 * 100 / 0.064)

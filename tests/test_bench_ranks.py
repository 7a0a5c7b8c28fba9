"""The multi-rank host logic of bench.py (replicas: one solve per rank, no
collective on the data path) with two gloo ranks on CPU: the job's time is the
slowest rank's, its cell updates the sum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate_ranks(dev_ms=10.0 + 5.0 * rank, updates=1000 * (rank + 1), world=world)
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_aggregate_ranks_max_time_sum_updates(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (15.0, 3000.0)


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(7.5, 123, 1) == (7.5, 123)

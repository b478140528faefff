"""Replicas across ranks (one system does not shard: every GPU runs its own
copy, no collective on the data path).  The only cross-rank step of
bench.py is the aggregation of the timed region: max over ranks and
whole-job throughput; checked here with two gloo ranks on the CPU."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took 10 * (r + 1) ms for 7 steps
    t_max, value = bench.aggregate_over_ranks(10.0 * (rank + 1), 7)
    out[rank] = (t_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            t_max, value = out[r]
            assert t_max == pytest.approx(20.0)
            assert value == pytest.approx(world * 7 / 0.020)


def test_aggregate_single_process():
    import bench
    t_max, value = bench.aggregate_over_ranks(14.0, 7)
    assert t_max == 14.0 and value == pytest.approx(500.0)

"""The N>1 bench path (independent replicas, one per rank): whole-job throughput is all
ranks' units over the slowest rank's time.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [40.0, 50.0][rank]
    value, ms = bench.aggregate_over_ranks(ms_local, 1000, dist, torch.device("cpu"))
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, ms = out[r]
        assert ms == pytest.approx(50.0)
        assert value == pytest.approx(2 * 1000 / 0.050)


def test_single_process_is_its_own_job():
    import bench
    value, ms = bench.aggregate_over_ranks(25.0, 500, None)
    assert ms == 25.0 and value == pytest.approx(500 / 0.025)

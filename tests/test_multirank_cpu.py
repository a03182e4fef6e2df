"""The N > 1 bench path on CPU: two gloo ranks, the job time is the slowest
rank's and the whole-job value counts every rank's replica (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    elapsed = 1.0 + rank          # rank 1 is the slow one
    t = bench.max_over_ranks(elapsed)
    out[rank] = (t, bench.job_value(world, 10, 1000, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_sum_the_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == 2.0
        assert v == pytest.approx(world * 10 * 1000 / 2.0)


def test_single_process_is_its_own_max():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 4, 100, 2.0) == 200.0

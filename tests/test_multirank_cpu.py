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


def test_shares_cover_every_unit_once():
    import bench

    units = list(range(16))
    for world in (1, 2, 3, 4, 8):
        got = sorted(u for r in range(world) for u in bench.share_of(units, r, world))
        assert got == units
        sizes = [len(bench.share_of(units, r, world)) for r in range(world)]
        assert max(sizes) - min(sizes) <= 1


def test_replica_command_runs_one_process_per_gpu_on_localhost():
    import bench

    cmd = bench.replica_command(["--gpus", "4", "--steps", "2"], 4, 29555)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--nnodes=1" in cmd
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[cmd.index("--master-port") + 1] == "29555"
    assert cmd[-4:] == ["--gpus", "4", "--steps", "2"]


def test_gpus_2_relaunches_as_two_ranks_and_prints_one_line():
    """`bench.py --gpus 2` started as one process re-executes itself as two
    ranks (torch.distributed.run); on the reference arm rank 0 alone runs
    and prints the contract line, rank 1 exits without work."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    env.pop("RANK", None)
    out = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=root, capture_output=True, text=True, timeout=900, env=env)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2

"""bench.py's multi-rank host logic on CPU with gloo, world size 2: the job
time is the slowest rank's, the rate counts every rank's units, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.init_dist(world, "gloo")
    t = bench.reduce_max(d, 1.0 + rank)          # rank 1 is the slow one
    rate = bench.aggregate_rate(10, world, t)
    env = bench.dist_env()
    out.put((rank, t, rate, env))
    d.barrier()
    d.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, env in res:
        assert t == 2.0                      # max over ranks
        assert rate == pytest.approx(10 * 2 / 2.0)
        assert env == (rank, world, rank)


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=0, n=None, b=None)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""

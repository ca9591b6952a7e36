"""The benchmark's multi-rank host logic on CPU: two gloo ranks with different step times;
the job time is the slowest rank's and the rate counts every rank's solves."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    out.put((rank, t, bench.whole_job_rate(world, 3, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [2.0, 2.0]
    assert [g[2] for g in got] == [3.0, 3.0]


def test_single_rank_is_local_time():
    import bench

    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.whole_job_rate(1, 4, 2.0) == 2.0

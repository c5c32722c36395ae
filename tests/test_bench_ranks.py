"""The benchmark's multi-rank logic on CPU: two gloo ranks (replicas, no
data-path collective) reduce their timings to the maximum and the whole-job
throughput counts every replica's units against the slowest one."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [10.0 + rank, 20.0 - rank, 5.0 * (rank + 1)]
    got = bench.max_over_ranks(torch, dist, mine, "cpu")
    out[rank] = (got, bench.job_value(1000, world, got[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        got, value = res[r]
        assert got == [11.0, 20.0, 10.0]
        assert value == pytest.approx(2 * 1000 / 11.0e-3)

"""The multi-rank path of bench.py (replicas: one lattice per GPU, no data-path
collective) on the CPU: two gloo ranks time different amounts of work, the
job's time is the slowest rank's, and the whole-job value sums both ranks'
units over that time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        assert bench.dist_env()[:2] == (rank, world)
        f = bench.max_over_ranks_fn(dist, "cpu")
        elapsed_ms = [120.0, 150.0][rank]   # rank 1 is the slow one
        dist.barrier()
        slowest = f(elapsed_ms)
        ms_step = slowest / 10
        value = bench.replica_value(world, 1.0e9, ms_step)
        out[rank] = (slowest, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]                      # every rank reports the same job figure
    slowest, value = res[0]
    assert slowest == 150.0                      # the slowest rank's time
    assert abs(value - 2 * 1.0e9 / 15e-3) < 1e-3 * value   # both ranks' units over it


def test_single_rank_needs_no_group():
    import bench

    f = bench.max_over_ranks_fn(None, "cpu")
    assert f(3.5) == 3.5
    assert bench.replica_value(1, 2.0e9, 2.0) == 1.0e12

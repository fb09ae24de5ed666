"""The benchmark's multi-rank host logic on two gloo ranks (CPU): the job time is the slowest rank's,
and under weak scaling the job embeds steps x ranks meshes in it.  The method itself does not shard
(replicas only), so this reduction is the only cross-rank step."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        local = [120.0, 150.5][rank]  # rank 1 is the slow one
        got = bench.max_over_ranks(local, "cpu")
        out[rank] = (got, bench.job_ms_per_mesh(got, 5, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (150.5, 150.5 / 10)


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(42.0, "cpu") == 42.0
    assert bench.job_ms_per_mesh(300.0, 5, 1) == 60.0

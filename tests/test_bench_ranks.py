"""bench.py's multi-rank path (independent replicas, one per GPU): the timed
region is the slowest rank's and the value counts every rank's updates.
Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [120.0, 250.0][rank]
    ms = bench.reduce_max_over_ranks(ms_local, dist, torch.device("cpu"))
    value = bench.whole_job_glups(1e9, world, ms)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_sum_the_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            ms, value = out[r]
            assert ms == 250.0
            assert abs(value - 2 * 1e9 / 0.25 / 1e9) < 1e-9


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_max_over_ranks(3.5, None, None) == 3.5
    assert bench.whole_job_glups(2e9, 1, 1000.0) == 2.0

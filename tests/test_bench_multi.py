"""The bench's multi-rank aggregation on CPU (gloo, world size 2): the
whole-job value is all ranks' units over the slowest rank's time."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        rate, t = bench.whole_job_rate(1000, 1.0 + rank, world, "cpu")
        out[rank] = (rate, t)
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29500 + os.getpid() % 1000
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        for r in range(2):
            rate, t = out[r]
            assert t == 2.0 and rate == 2 * 1000 / 2.0


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(10, 2.0, 1, "cpu") == (5.0, 2.0)

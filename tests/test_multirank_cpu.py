"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) reduce their
step times to the slowest rank's and report the whole-job rate."""
import os
import socket

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
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms, val = bench.job_rate(10.0 + 5.0 * rank, 1e12, world, "cpu")
        out[rank] = (ms, val)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        ms, val = res[r]
        assert ms == 15.0  # the slower rank
        assert abs(val - world * 1e12 / 15e-3 / 1e12) < 1e-9


def test_single_rank_is_unchanged():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    ms, val = bench.job_rate(8.0, 2e12, 1, "cpu")
    assert ms == 8.0 and abs(val - 250.0) < 1e-9

"""The multi-rank path of the benchmark (replicas only: each rank applies its own
problem, no data-path collective) on CPU with the gloo backend, world size 2:
the timings reduce to their maximum on every rank, and the whole-job value is
all ranks' targets over the slowest rank's time."""
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
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]   # rank 1 is slower in the first, faster in the second
        red = bench.max_over_ranks(ms, world, torch.device("cpu"))
        out[rank] = (red, bench.whole_job_value(1_000_000, world, red[0]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of this multi-threaded process
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        red, value = res[rank]
        assert red == [15.0, 20.0]
        assert value == pytest.approx(2 * 1_000_000 / 15e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([3.0, 4.0], 1, None) == [3.0, 4.0]
    assert bench.whole_job_value(10, 1, 2.0) == pytest.approx(5000.0)

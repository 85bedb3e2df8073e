"""bench.py's N > 1 path on CPU: world_size-2 gloo ranks (replicas, as on N GPUs under torchrun).
The timed milliseconds are reduced to the slowest rank's on every rank, and the reported rate is the
units of all ranks over that time."""

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


def _rank(rank, world, port, ms_of_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max = bench.max_over_ranks(ms_of_rank[rank], dist, "cpu")
        out[rank] = (ms_max, bench.whole_job_rate(7.13e9, 5, world, ms_max))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ms_of_rank = [501.0, 512.5]  # rank 1 is slower
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, ms_of_rank, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms_max, rate = res[r]
        assert ms_max == 512.5
        assert rate == pytest.approx(7.13e9 * 5 * 2 / 0.5125)


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(10.0, 4, 1, 2000.0) == pytest.approx(20.0)

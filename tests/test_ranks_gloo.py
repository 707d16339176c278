"""The N > 1 path of the benchmark on the CPU: two gloo ranks, max-over-ranks timing and the job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1504_06123_gb300 import ranks  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.5 if rank == 0 else 2.5               # the slower rank decides
        slowest = ranks.max_over_ranks(t, dist)
        rate = ranks.job_rate(1000.0, world, slowest)
        dist.barrier()
        out[rank] = (slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rate():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a process that may hold host threads
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][0] == 2.5
        assert res[r][1] == pytest.approx(1000.0 * 2 / 2.5)


def test_single_process_is_identity():
    assert ranks.max_over_ranks(3.0, None) == 3.0
    assert ranks.job_rate(10.0, 1, 2.0) == 5.0

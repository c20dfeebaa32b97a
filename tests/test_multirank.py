"""The replica path of bench.py on two CPU ranks (gloo): the step time is
the slowest rank's and the rate counts every rank's units; the ranks meet
at barriers around the timed region."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms, rate = bench.whole_job_rate(torch, dist, 2.0 + rank, 1000, "cpu")
    dist.barrier()
    q.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == pytest.approx(3.0)                  # the slower rank's 3 ms
        assert rate == pytest.approx(2 * 1000 / 3.0e-3)  # both ranks' units

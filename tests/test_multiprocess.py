"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own replica time; the
job time is the slowest rank's and the rate counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                    # rank 1 is the slower replica
    job_ms = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    out[rank] = (job_ms, bench.whole_job_rate(world, 1000, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    job_ms, rate = res[0]
    assert job_ms == 150.0
    assert rate == pytest.approx(2 * 1000 / 0.150)

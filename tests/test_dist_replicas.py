"""The multi-GPU form is replicas only (events are independent; no exchange step): each rank
runs its own batch and the job's rate is every rank's tracks over the slowest rank's time.
The reduction that bench.py uses is checked here with two gloo ranks on the CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, ms = [1000, 3000][rank], [2.0, 5.0][rank]
    out[rank] = bench.job_rate(units, ms, dist, "cpu")
    dist.destroy_process_group()


def test_job_rate_sums_units_and_takes_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        for rank in range(world):
            units, ms, rate = out[rank]
            assert units == 4000 and ms == 5.0 and rate == pytest.approx(4000 / 5e-3)


def test_job_rate_single_process():
    import bench
    assert bench.job_rate(10, 2.0) == (10.0, 2.0, 5000.0)

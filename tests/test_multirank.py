"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
runs its own replica, the job time is the slowest rank's and the job's
events are the sum over ranks."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, ev = bench.job_totals(dist, 10.0 * (rank + 1), 1000.0 + rank, device="cpu")
    out[rank] = (ms, ev)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (20.0, 2001.0)


def test_job_totals_single_process():
    import bench
    assert bench.job_totals(None, 5.0, 7.0) == (5.0, 7.0)

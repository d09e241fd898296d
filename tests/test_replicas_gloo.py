"""The N-GPU bench path runs independent replicas: whole-job time is the
slowest rank's, units are summed over ranks. Checked here with two gloo ranks
on the CPU (no GPU, no data-path collective)."""
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
    secs = [2.0, 3.0][rank]
    units = [1000.0, 1500.0][rank]
    t, u = bench.job_totals(dist, secs, units, "cpu")
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (3.0, 2500.0)
    assert res[0][1] / res[0][0] == pytest.approx(2500.0 / 3.0)


def test_job_totals_single_process():
    import bench
    assert bench.job_totals(None, 2.5, 10.0, "cpu") == (2.5, 10.0)

"""The multi-GPU path of bench.py is replicas (independent problems, no data-path
collective); its only cross-rank step is the timing: the job time is the slowest rank's and
the job rate counts every rank's units.  Checked here with world_size 2 on CPU (gloo)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    slowest = bench.max_over_ranks(times[rank], ws, device="cpu")
    out[rank] = (slowest, bench.job_rate(1000.0, ws, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_ranks():
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as m:
        out = m.dict()
        port = _free_port()
        times = [0.5, 0.8]
        procs = [mp.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            slowest, rate = out[r]
            assert slowest == 0.8
            assert rate == pytest.approx(2 * 1000.0 / 0.8)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(0.3, 1) == 0.3
    assert bench.job_rate(10.0, 1, 2.0) == 5.0

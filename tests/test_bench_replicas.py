"""bench.py's multi-GPU mode runs independent replicas (no collective on the data path):
the job's time is the slowest rank's and its rate counts every rank's pixels.  Checked with
two gloo ranks on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = 2.0 + rank  # rank 1 is the slow replica
    out[rank] = (bench.max_over_ranks(local_seconds, dist),
                 bench.whole_job_rate(1_000_000, 5, local_seconds, dist))
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time_and_the_whole_job_rate():
    torch = pytest.importorskip("torch")
    import socket
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with mp.Manager() as m:
        out = m.dict()
        procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            slowest, rate = out[r]
            assert slowest == 3.0
            assert rate == pytest.approx(2 * 1_000_000 * 5 / 3.0)


def test_one_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, None) == 1.5
    assert bench.whole_job_rate(10, 2, 4.0, None) == 5.0

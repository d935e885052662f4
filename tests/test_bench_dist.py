"""The multi-rank path of bench.py (replicas, one per GPU) on CPU with the
gloo backend: the job's step time is the slowest rank's and the rate counts
every rank's pixels."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t, v = bench.whole_job_rate(10.0 * (rank + 1), 1_000_000, ws, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_whole_job_rate_takes_the_slowest_rank_and_all_pixels():
    import torch.multiprocessing as mp
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == pytest.approx(20.0)
        assert v == pytest.approx(ws * 1_000_000 / 20e-3 / 1e6)


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    t, v = bench.whole_job_rate(50.0, 4_194_304, 1, "cpu")
    assert t == 50.0 and v == pytest.approx(4_194_304 / 0.05 / 1e6)

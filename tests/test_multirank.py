"""The replicas path of bench.py on two gloo ranks (CPU): process-group set-up
from the torchrun environment, the barrier, the max over ranks of the timed
region, and the whole-job throughput computed from it."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank), HDP_BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, ws = bench.dist_init()
    bench.barrier(ws)
    ms = bench.reduce_max(10.0 + 5.0 * r, ws)          # rank 1 is the slower one
    q.put((r, ws, ms, bench.job_value(ws, 1e6, ms)))
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_the_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, ws, ms, value) in enumerate(got):
        assert (rank, ws) == (r, 2)
        assert ms == 15.0                                   # the max over both ranks
        assert value == pytest.approx(2 * 1e6 / 0.015 / 1e6)   # both ranks' units over the slowest time

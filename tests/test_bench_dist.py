"""bench.py's multi-rank host logic on CPU: two gloo ranks, max-over-ranks time and whole-job
throughput (each rank solves its own instance; no data-path collective)."""
from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    bench.init_dist(ws, "gloo")
    elapsed = 100.0 + 50.0 * rank                         # rank 1 is the slow one
    out = bench.aggregate(units_per_rank=1000.0, elapsed_ms=elapsed, ws=ws)
    bench.barrier(ws)
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r]["max_ms"] == pytest.approx(150.0)
        assert res[r]["value"] == pytest.approx(2 * 1000.0 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    out = bench.aggregate(500.0, 250.0, 1)
    assert out["max_ms"] == 250.0 and out["value"] == pytest.approx(2000.0)

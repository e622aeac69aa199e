"""The N > 1 host logic of bench.py on CPU: two gloo ranks on 127.0.0.1
(process-group setup, barrier, max-over-ranks timing). Replicas exchange no
data on the SpGEMM path; the only collective is the timing reduction."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "BENCH_BACKEND": "gloo"})
    import bench
    r, w = bench.dist_init(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    got = bench.max_over_ranks(10.0 + rank, w)
    q.put((rank, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 11.0), (1, 11.0)]


def test_single_process_defaults():
    import bench
    for k in ("RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    r, w = bench.dist_init(1)
    assert (r, w) == (0, 1)
    assert bench.max_over_ranks(3.5, 1) == 3.5

"""The N > 1 bench path on CPU: two gloo ranks, max-over-ranks timing and the
whole-job aggregate (each rank evaluates its own replica, no data exchange)."""

from __future__ import annotations

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    ms = 1.0 + rank  # rank 1 is the slower one
    m = bench.max_over_ranks(ms, dist, "cpu")
    q.put((rank, m, bench.aggregate(24576, m, ws)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    assert out[0][2] == pytest.approx(2 * 24576 / 2e-3)


def test_single_rank_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.aggregate(100, 2.0, 1) == pytest.approx(5e4)
    # 13 rebuild + 15 evaluation kernels, as an ncu launch list of one T = 3 step counts them
    assert bench.launches_per_step(3) == 28

"""Multi-rank bench aggregation on CPU (gloo, world_size 2): each rank runs its
own replica; the job's step time is the slowest rank's and the value sums the
units of all ranks."""
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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = [10.0, 25.0][rank]
    out = bench.aggregate_over_ranks(ms, 1000.0)
    q.put((rank, out))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
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
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 25.0
        assert abs(value - 2 * 1000.0 / 25e-3) < 1e-6


def test_aggregate_single_rank():
    import bench
    ms, value = bench.aggregate_over_ranks(20.0, 500.0)
    assert ms == 20.0 and abs(value - 500.0 / 20e-3) < 1e-9

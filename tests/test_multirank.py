"""The benchmark's multi-rank path (N independent replicas, weak scaling) on
CPU with the gloo backend, world size 2: timing is the max over ranks and the
job's rate counts every rank's units."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [40.0, 55.0][rank]                       # rank 1 is the slowest
    m = bench.max_over_ranks(ms, dist)
    rate = bench.whole_job_rate(1.0e12, m * 1e-3, world)
    dist.barrier()
    q.put((rank, m, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in out:
        assert m == 55.0                          # every rank sees the max
        assert abs(rate - 2.0e12 / 0.055) < 1e-3 * rate


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 2.0, 4) == 20.0

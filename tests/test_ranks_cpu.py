"""The multi-rank timing path of bench.py (replicas, max over ranks) on
world_size-2 gloo process groups on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 95.0][rank]
    dist.barrier()
    m = bench.max_over_ranks(local_ms)
    rate = bench.whole_job_rate(5, world, m / 1000.0)
    q.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [120.0, 120.0]
    assert res[0][2] == pytest.approx(2 * 5 / 0.120)


def test_single_process_path():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(4, 1, 2.0) == 2.0

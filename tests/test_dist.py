"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
timed region's max over ranks and the whole-job weak-scaling rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # the slower rank sets the job's time
        m = bench.max_over_ranks(ms)
        q.put((rank, m, bench.whole_job_rate(1000, 5, world, m)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_rate_gloo():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [150.0, 150.0]
    assert all(abs(r[2] - 1000 * 5 * 2 / 0.15) < 1e-6 for r in res)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.whole_job_rate(10, 2, 1, 1000.0) == 20.0

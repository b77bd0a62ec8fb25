"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timing
is the maximum over ranks and the job value counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    m = bench.reduce_max(ms, "cpu")
    out.put((rank, m, bench.job_value(1000, world, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_and_job_value_two_ranks():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in res:
        assert m == 15.0
        assert abs(v - 2000 / 0.015) < 1e-6


def test_single_process_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_value(10, 1, 1000.0) == 10.0

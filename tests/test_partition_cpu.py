"""Host side of the slab partition, on CPU: the partition plan
(st_partition_plan) and the torch.distributed (gloo) communicator's
callbacks -- the halo chain, the gather of the coarse level and the sum of
the Krylov dot products -- with two gloo processes and host buffers, exactly
as a partitioned handle calls them."""
import ctypes
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_or_skip():
    from paper_1802_09277_gb300 import st
    if not os.path.exists(st.LIB_PATH):
        pytest.skip("libst_iga.so not built")
    return st


def test_partition_plan():
    st = _lib_or_skip()
    assert st.partition_plan(8, 2, 1) == (4, 4, 2)
    assert st.partition_plan(256, 4, 3) == (192, 64, 6)
    assert st.partition_plan(8, 4, 2) == (4, 2, 1)
    assert st.partition_plan(16, 1, 0) == (0, 16, 4)
    for bad in [(12, 4, 0), (8, 8, 0), (9, 3, 0), (8, 2, 2), (8, 0, 0)]:
        with pytest.raises(st.StError) as e:
            st.partition_plan(*bad)
        assert e.value.code == -1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1802_09277_gb300 import st
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    comm = st.GlooComm()
    c = comm.c
    n = 24
    # halo chain: every rank sends to rank + 1 and receives from rank - 1
    send = np.full(n, 10 + rank, dtype=np.uint8)
    recv = np.zeros(n, dtype=np.uint8)
    rc1 = c.sendrecv(None, send.ctypes.data, rank + 1 if rank + 1 < world else -1,
                     recv.ctypes.data, rank - 1 if rank > 0 else -1, n, None)
    # gather of one block per rank, in rank order
    blk = np.arange(n, dtype=np.uint8) + 50 * rank
    allg = np.zeros(n * world, dtype=np.uint8)
    rc2 = c.allgather(None, blk.ctypes.data, allg.ctypes.data, n, None)
    # in-place sum of host doubles
    vals = np.array([1.5 * (rank + 1), -2.0, 1e-300 * rank], dtype=np.float64)
    rc3 = c.allreduce_sum(None, vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 3)
    out.put((rank, rc1, rc2, rc3, recv.copy(), allg.copy(), vals.copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_comm_callbacks_two_ranks():
    _lib_or_skip()
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, rc1, rc2, rc3, recv, allg, vals in res:
        assert (rc1, rc2, rc3) == (0, 0, 0)
        if rank == 1:
            assert np.all(recv == 10)  # rank 0's plane
        else:
            assert np.all(recv == 0)   # rank 0 has no predecessor
        assert np.array_equal(allg, np.concatenate([np.arange(24, dtype=np.uint8) + 50 * q
                                                    for q in range(2)]))
        assert np.array_equal(vals, np.array([4.5, -4.0, 1e-300]))
    # every rank holds the same bits of the sum
    assert res[0][6].tobytes() == res[1][6].tobytes()

"""Slab partition over several processes (st_setup_partitioned): ranks run
as gloo processes that share the one GPU and exchange the coupling plane and
the coarse level through host memory (no kernel waits on another process).
Every rank's slabs of st_apply, st_smooth and st_vcycle equal the
single-process handle bit for bit (the halo plane is read where the
single-process kernel reads the previous slab, and the gathered coarse
levels run the same code on the same data); the partitioned solve matches
the oracle's direct solution."""
import os
import socket
import sys

import numpy as np
import pytest

from oracle import assemble as A
from oracle import solve as S
from paper_1802_09277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def st():
    from paper_1802_09277_gb300 import build, st as stmod
    if not os.path.exists(stmod.LIB_PATH):
        build.build()
    stmod.load()
    assert torch.cuda.is_available()
    return stmod


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _vectors(d, spans, p, N, nrhs):
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    x = inputs.uniform_vector(71, nrhs * pr.ndofs)
    u0 = inputs.uniform_vector(72, nrhs * pr.ndofs)
    c = np.concatenate([inputs.normal_coeffs(73 + q, pr.ndofs) for q in range(nrhs)])
    return pr, x, u0, c


def _ops(st, s, x, u0, c, tol):
    """apply, one smoothing step, one V-cycle and a solve on host arrays."""
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    y = torch.empty(s.ndofs, dtype=torch.float64, device="cuda")
    s.apply(dev(x), y)
    out = {"apply": y.cpu().numpy()}
    u = dev(u0)
    f = torch.empty_like(u)
    s.load_coeffs(dev(c), f)
    s.smooth(u, f, 1)
    out["smooth"] = u.cpu().numpy()
    u = dev(u0)
    s.vcycle(u, f)
    out["vcycle"] = u.cpu().numpy()
    u = torch.zeros_like(f)
    info = s.solve(f, u, tol=tol)
    out["solve"] = u.cpu().numpy()
    out["iterations"] = info["iterations"]
    return out


def _rank_main(rank, world, port, case, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1802_09277_gb300 import st
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    torch.cuda.set_device(0)
    d, spans, p, N, nrhs, prec, outer, tol = case
    pr, x, u0, c = _vectors(d, spans, p, N, nrhs)
    b, nloc, _ = st.partition_plan(N, world, rank)
    m = pr.Nt * pr.Nx
    mine = lambda a: a.reshape(nrhs, N, m)[:, b:b + nloc, :].reshape(-1).copy()
    comm = st.GlooComm()
    s = st.Solver(d, p, spans, N, comm=comm, nrhs=nrhs, precision=prec, outer=outer)
    try:
        out = _ops(st, s, mine(x), mine(u0), mine(c), tol)
        q.put((rank, out, None))
    except Exception as e:  # report instead of hanging the other ranks
        q.put((rank, None, repr(e)))
    s.close()
    dist.barrier()
    dist.destroy_process_group()


CASES = [  # (d, spans, p, N, nrhs, precision, outer, solve tol), ranks
    ((2, (12, 10), 2, 8, 2, "fp64", "fgmres", 1e-12), 2),
    ((1, (24,), 3, 8, 1, "fp64", "mg", 1e-12), 4),        # gathered level wider than a rank's
    ((2, (14, 9), 2, 16, 1, "mixed_fp32", "ir", 1e-10), 2),
]


@pytest.mark.parametrize("case,world", CASES)
def test_partitioned_equals_single_process(st, case, world):
    d, spans, p, N, nrhs, prec, outer, tol = case
    pr, x, u0, c = _vectors(d, spans, p, N, nrhs)
    ref_s = st.Solver(d, p, spans, N, nrhs=nrhs, precision=prec, outer=outer)
    ref = _ops(st, ref_s, x, u0, c, tol)
    ref_s.close()
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for p_ in procs:
        p_.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p_ in procs:
        p_.join(120)
        assert p_.exitcode == 0
    for rank, out, err in res:
        assert err is None, (rank, err)
    m = pr.Nt * pr.Nx

    def gather(name):
        parts = [r[1][name].reshape(nrhs, -1, m) for r in res]
        return np.concatenate(parts, axis=1).reshape(-1)

    for name in ("apply", "smooth", "vcycle"):
        assert np.array_equal(gather(name), ref[name]), name
    # the Krylov sums are taken per rank and then over the ranks: the same
    # solution up to rounding, and the oracle's
    u = gather("solve")
    assert np.linalg.norm(u - ref["solve"]) <= 1e-9 * np.linalg.norm(ref["solve"])
    bound = 1e-10 if prec == "fp64" else 1e-8
    for q_ in range(nrhs):
        f = A.load_from_coeffs(pr, c.reshape(nrhs, -1)[q_])
        ud = S.forward_subst(pr, f)
        uq = u.reshape(nrhs, -1)[q_]
        assert np.linalg.norm(uq - ud) <= bound * np.linalg.norm(ud)
    assert all(r[1]["iterations"] == res[0][1]["iterations"] for r in res)


def test_nccl_single_rank_partition(st):
    """The NCCL communicator (world size 1 here: one GPU) drives the same
    partitioned code path: the V-cycle equals the plain handle's bits."""
    try:
        uid = st.NcclComm.unique_id()
    except st.StError as e:
        if e.code == -9:
            pytest.skip("libnccl.so.2 not loadable")
        raise
    comm = st.NcclComm(1, 0, uid)
    d, spans, p, N = 2, (12, 10), 2, 8
    pr, x, u0, c = _vectors(d, spans, p, N, 1)
    s = st.Solver(d, p, spans, N, comm=comm)
    a = _ops(st, s, x, u0, c, 1e-12)
    s.close()
    comm.close()
    r = st.Solver(d, p, spans, N)
    b = _ops(st, r, x, u0, c, 1e-12)
    r.close()
    for name in ("apply", "smooth", "vcycle"):
        assert np.array_equal(a[name], b[name]), name
    assert np.linalg.norm(a["solve"] - b["solve"]) <= 1e-10 * np.linalg.norm(b["solve"])


def test_partition_rejects_unsupported_options(st):
    from paper_1802_09277_gb300 import st as stmod
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % _free_port(),
                                rank=0, world_size=1)
    comm = stmod.GlooComm()
    for kw in [dict(basis="spectral"), dict(spatial_solver="minres"), dict(space_ratio=1.0)]:
        with pytest.raises(stmod.StError) as e:
            stmod.Solver(2, 2, (8, 8), 8, comm=comm, **kw)
        assert e.value.code == -9
    with pytest.raises(stmod.StError) as e:
        stmod.Solver(2, 2, (8, 8), 6, comm=comm)  # 6 slabs: not a power of two
    assert e.value.code == -1
    dist.destroy_process_group()

"""Serving loop (st_serve_*): continuous batching of solves of different
configurations.  Every request's result must be the same whether it is
solved alone or in a mix with others (batched with requests of the same
configuration and overlapping with others on the GPU), and must match the
oracle's direct solution to the solve tolerance."""
import numpy as np
import pytest

from oracle import assemble as A
from oracle import solve as S
from paper_1802_09277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    import os
    from paper_1802_09277_gb300 import build, st as stmod
    if not os.path.exists(stmod.LIB_PATH):
        build.build()
    stmod.load()
    assert torch.cuda.is_available()
    return stmod


# (dim, spans, degree, slabs): a mix with repeated configurations so that the
# server can batch them
MIX = [(2, (16, 16), 2, 8), (2, (16, 16), 2, 8), (1, (32,), 3, 16), (2, (16, 16), 2, 8),
       (2, (12, 20), 1, 32), (3, (6, 6, 6), 2, 4), (1, (32,), 3, 16), (2, (12, 20), 1, 32)]


def _requests():
    reqs = []
    for i, (d, spans, p, N) in enumerate(MIX):
        pr = A.Problem(d, spans, p, 2, N, theta=1.0)
        reqs.append((d, spans, p, N, inputs.normal_coeffs(500 + i, pr.ndofs)))
    return reqs


@pytest.mark.parametrize("prec,outer", [("mixed_tf32", "ir"), ("fp64", "fgmres")])
def test_alone_vs_mix(st, prec, outer):
    reqs = _requests()
    tol = 1e-10
    opts = dict(precision=prec, outer=outer, basis="spectral")
    alone = []
    srv = st.Server(workers=1, max_batch=1, **opts)
    for d, spans, p, N, c in reqs:
        t = srv.submit(d, p, spans, N, c, tol=tol, coeffs=True)
        res, u = srv.wait(t, timeout=120.0)
        assert res["status"] == 0 and res["batch_size"] == 1
        alone.append(u)
    srv.stop()
    # queue the whole mix before any worker starts, so that the repeated
    # configurations are in the queue together and are batched
    srv = st.Server(workers=3, max_batch=4, paused=True, **opts)
    tickets = [srv.submit(d, p, spans, N, c, tol=tol, coeffs=True) for d, spans, p, N, c in reqs]
    srv.resume()
    mixed = [srv.wait(t, timeout=120.0) for t in tickets]
    srv.stop()
    sizes = [res["batch_size"] for res, _ in mixed]
    # every repeated configuration was solved as one batch
    assert sizes == [MIX.count(m) for m in MIX], sizes
    groups = [res["group_requests"] for res, _ in mixed]
    if outer == "ir":  # the refinement server groups configurations (how many per call
        # depends on which worker builds which setup first: the lock is released meanwhile)
        assert all(g >= b for g, b in zip(groups, sizes)), groups
    else:  # other solvers: each configuration's batch alone
        assert groups == sizes, groups
    for (d, spans, p, N, c), ua, (res, um) in zip(reqs, alone, mixed):
        assert res["status"] == 0
        # each right-hand side is refined on its own: same bits alone and in the mix
        assert np.array_equal(ua, um), (d, spans, p, N, res["batch_size"])
        pr = A.Problem(d, spans, p, 2, N, theta=1.0)
        ud = S.forward_subst(pr, A.load_from_coeffs(pr, c))
        assert np.linalg.norm(um - ud) <= 1e-8 * np.linalg.norm(ud)


def test_budget_admission(st):
    d, spans, p, N = 2, (24, 24), 2, 16
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    c = inputs.normal_coeffs(600, pr.ndofs)
    # too small for any setup: the request fails cleanly with OVER_BUDGET
    srv = st.Server(workers=2, max_batch=2, hbm_budget=1 << 20, precision="mixed_fp32", outer="ir")
    res, _ = srv.wait(srv.submit(d, p, spans, N, c, coeffs=True), timeout=60.0)
    assert res["status"] == -8
    srv.stop()
    # enough for one setup at a time: requests are admitted one after the other
    probe = st.Solver(d, p, spans, N, precision="mixed_fp32", outer="ir", basis="spectral")
    f = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    f[0] = 1.0
    probe.solve(f, torch.zeros_like(f), tol=1e-8)  # allocates the Krylov space
    from paper_1802_09277_gb300.st import _lib
    import ctypes
    nb = ctypes.c_size_t()
    _lib.st_sizes(probe._h, None, None, None, None, ctypes.byref(nb))
    one = nb.value + 2 * 8 * pr.ndofs  # setup + Krylov space + the request's two vectors
    probe.close()
    budget = int(1.5 * one)  # room for one batch at a time
    srv = st.Server(workers=3, max_batch=1, hbm_budget=budget, precision="mixed_fp32",
                    outer="ir", basis="spectral")
    ts = [srv.submit(d, p, spans, N, inputs.normal_coeffs(601 + i, pr.ndofs), coeffs=True)
          for i in range(4)]
    outs = [srv.wait(t, timeout=120.0) for t in ts]
    srv.stop()
    assert all(r["status"] == 0 for r, _ in outs), (
        [(r["status"], r["error"]) for r, _ in outs], budget, one)


def test_poll_and_tickets(st):
    srv = st.Server(workers=1, max_batch=1, precision="mixed_fp32", outer="ir")
    d, spans, p, N = 1, (20,), 2, 4
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    t = srv.submit(d, p, spans, N, inputs.normal_coeffs(7, pr.ndofs), coeffs=True)
    got = None
    for _ in range(20000):
        got = srv.poll(t)
        if got is not None:
            break
    if got is None:
        got = srv.wait(t, timeout=60.0)
    assert got[0]["status"] == 0 and got[0]["latency_seconds"] >= got[0]["solve_seconds"]
    with pytest.raises(st.StError):
        srv.poll(t + 12345) if (t + 12345) in srv._n else st._check(
            st.load().st_serve_poll(srv._s, t + 12345, None, None))
    srv.stop()


def test_cancel_pending_request(st):
    srv = st.Server(workers=1, max_batch=1, paused=True, precision="mixed_fp32", outer="ir")
    d, spans, p, N = 1, (20,), 2, 4
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    t1 = srv.submit(d, p, spans, N, inputs.normal_coeffs(8, pr.ndofs), coeffs=True)
    t2 = srv.submit(d, p, spans, N, inputs.normal_coeffs(9, pr.ndofs), coeffs=True)
    assert srv.cancel(t2)  # nobody has taken it yet
    res2, _ = srv.wait(t2, timeout=10.0)
    assert res2["status"] == -11 and res2["error"] == "cancelled"
    srv.resume()
    res1, u1 = srv.wait(t1, timeout=60.0)
    assert res1["status"] == 0
    ud = S.forward_subst(pr, A.load_from_coeffs(pr, inputs.normal_coeffs(8, pr.ndofs)))
    assert np.linalg.norm(u1 - ud) <= 1e-7 * np.linalg.norm(ud)
    with pytest.raises(st.StError):  # finished and released: unknown ticket
        srv.cancel(t1)
    srv.stop()


def test_pause_queues_and_batches(st):
    """A running server paused with st_serve_pause takes no request until
    st_serve_resume; the queued repeats of one configuration then form one
    batch, with the results of a fresh server."""
    opts = dict(precision="mixed_tf32", outer="ir", basis="spectral")
    reqs = _requests()
    srv = st.Server(workers=2, max_batch=4, **opts)
    d, spans, p, N, c = reqs[0]
    first, _ = srv.wait(srv.submit(d, p, spans, N, c, tol=1e-10, coeffs=True), timeout=120.0)
    assert first["status"] == 0  # the server runs before the pause
    srv.pause()
    tickets = [srv.submit(d, p, spans, N, c, tol=1e-10, coeffs=True)
               for d, spans, p, N, c in reqs]
    import time
    time.sleep(0.5)
    assert all(srv.poll(t) is None for t in tickets)  # nothing taken while paused
    srv.resume()
    got = [srv.wait(t, timeout=120.0) for t in tickets]
    srv.stop()
    assert [res["batch_size"] for res, _ in got] == [MIX.count(m) for m in MIX]
    ref = st.Server(workers=1, max_batch=4, paused=True, **opts)
    rt = [ref.submit(d, p, spans, N, c, tol=1e-10, coeffs=True) for d, spans, p, N, c in reqs]
    ref.resume()
    for (res, u), t in zip(got, rt):
        r2, u2 = ref.wait(t, timeout=120.0)
        assert res["status"] == 0 and r2["status"] == 0
        assert np.array_equal(u, u2)
    ref.stop()


def test_group_members_off(st):
    """group_members = 1: every configuration's batch is solved alone, with
    the same bits as in a group."""
    opts = dict(precision="mixed_tf32", outer="ir", basis="spectral")
    reqs = _requests()
    out = {}
    for gm in (1, 8):
        srv = st.Server(workers=1, max_batch=4, paused=True, group_members=gm, **opts)
        tickets = [srv.submit(d, p, spans, N, c, tol=1e-10, coeffs=True)
                   for d, spans, p, N, c in reqs]
        srv.resume()
        out[gm] = [srv.wait(t, timeout=120.0) for t in tickets]
        srv.stop()
    # one worker: the oldest configuration first, then (oldest first) every
    # other configuration with no more dofs per request; then the rest
    ndofs = [A.Problem(d, spans, p, 2, N, theta=1.0).ndofs for d, spans, p, N in MIX]
    expect, left = [0] * len(MIX), list(range(len(MIX)))
    while left:
        lead = left[0]
        members = {MIX[i] for i in left if ndofs[i] <= ndofs[lead]}
        group = [i for i in left if MIX[i] in members]
        for i in group:
            expect[i] = len(group)
        left = [i for i in left if i not in group]
    for (r1, u1), (r8, u8), e in zip(out[1], out[8], expect):
        assert r1["status"] == 0 and r8["status"] == 0
        assert r1["group_requests"] == r1["batch_size"]
        assert r8["group_requests"] == e, ([r["group_requests"] for r, _ in out[8]], expect)
        assert np.array_equal(u1, u8)
    # one group call reads its reductions back fewer times than the batches
    # alone (one solve call per configuration; the MIX configurations differ
    # in their dof counts)
    calls1 = {r["n_dofs"]: r["host_syncs"] for r, _ in out[1]}
    assert len(calls1) == len(set(MIX))
    first_group = [i for i in range(len(MIX)) if expect[i] == expect[0]]
    assert out[8][0][0]["host_syncs"] < sum(calls1[ndofs[i]] for i in set(first_group))

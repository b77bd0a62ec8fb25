"""st_solve_host: a stream of batches of right-hand sides in host memory,
solved batch after batch while the next batch is copied in and the previous
solutions are copied out.  Each batch's solution equals st_solve's on the
same handle bit for bit and the oracle's exact solution to the solve's
tolerance (mixed precision solved to 1e-10: 1e-8, as the mixed parity
tests); initial guesses, pageable buffers, argument errors and a failing
batch."""
import ctypes

import numpy as np
import pytest

from oracle import assemble as A
from oracle import solve as S
from paper_1802_09277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D, SPANS, P, N, NE, NRHS, NBATCH = 2, (12, 10), 2, 8, 2, 2, 3


@pytest.fixture(scope="module")
def st():
    import os
    from paper_1802_09277_gb300 import build, st as stmod
    if not os.path.exists(stmod.LIB_PATH):
        build.build()
    stmod.load()
    assert torch.cuda.is_available()
    return stmod


@pytest.fixture(scope="module")
def problem():
    """Oracle load vectors of NBATCH x NRHS systems and their exact solutions
    (block forward substitution)."""
    pr = A.Problem(D, SPANS, P, NE, N, theta=1.0)
    F = [A.load_from_coeffs(pr, inputs.normal_coeffs(40 + q, pr.ndofs))
         for q in range(NBATCH * NRHS)]
    U = [S.forward_subst(pr, f) for f in F]
    return pr, np.concatenate(F), np.stack(U)


def _solver(st, **kw):
    opt = dict(ne_per_slab=NE, nrhs=NRHS, precision="mixed_tf32", basis="spectral",
               outer="ir")
    opt.update(kw)
    return st.Solver(D, P, SPANS, N, **opt)


def test_stream_matches_st_solve_and_oracle(st, problem):
    pr, F, U = problem
    s = _solver(st)
    assert s.ndofs == NRHS * pr.ndofs
    fh = torch.tensor(F, dtype=torch.float64).pin_memory()
    uh = torch.full_like(fh, 7.0).pin_memory()
    info = s.solve_host(fh, uh, tol=1e-10)
    assert info["rel_residual"] <= 1e-10
    hist = s.history()
    assert hist and hist[-1][1] <= 1e-10  # the last batch's history
    got = uh.numpy().reshape(NBATCH * NRHS, pr.ndofs)
    for q in range(NBATCH * NRHS):
        err = np.linalg.norm(got[q] - U[q]) / np.linalg.norm(U[q])
        assert err <= 1e-8, (q, err)
    # the same batches through st_solve on device buffers: identical bits
    for k in range(NBATCH):
        fd = fh[k * s.ndofs:(k + 1) * s.ndofs].cuda()
        ud = torch.zeros_like(fd)
        s.solve(fd, ud, tol=1e-10)
        torch.cuda.synchronize()
        assert torch.equal(ud.cpu(), uh[k * s.ndofs:(k + 1) * s.ndofs]), k
    # pageable buffers give the same result (the copies then block)
    fp, up = fh.clone(), torch.empty_like(fh)
    assert not fp.is_pinned()
    s.solve_host(fp, up, tol=1e-10)
    assert torch.equal(up, uh)
    # guesses are read: starting from the solutions takes fewer steps
    ug = uh.clone().pin_memory()
    ig = s.solve_host(fh, ug, tol=1e-10, use_guess=True)
    assert ig["iterations"] < info["iterations"], (ig, info)
    assert ig["rel_residual"] <= 1e-10
    assert np.abs(ug.numpy() - uh.numpy()).max() <= 1e-8 * np.abs(U).max()
    # one batch is st_solve itself
    one = torch.empty(s.ndofs, dtype=torch.float64).pin_memory()
    s.solve_host(fh[:s.ndofs].clone().pin_memory(), one, tol=1e-10)
    assert torch.equal(one, uh[:s.ndofs])
    s.close()


def test_arguments_rejected(st, problem):
    pr, F, _ = problem
    s = _solver(st)
    fh = torch.tensor(F, dtype=torch.float64)
    uh = torch.empty_like(fh)
    with pytest.raises(ValueError):
        s.solve_host(fh.cuda(), uh)  # device tensors belong to st_solve
    with pytest.raises(ValueError):
        s.solve_host(fh[:-1].clone(), uh[:-1].clone())  # not whole batches
    lib = st.load()
    info = st.StSolveInfo()
    vp = ctypes.c_void_p
    fd = torch.zeros(s.ndofs, dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(fd)
    cases = [
        (0, vp(fh.data_ptr()), 1e-8, vp(uh.data_ptr())),        # nbatch < 1
        (1, None, 1e-8, vp(uh.data_ptr())),                     # null rhs
        (1, vp(fh.data_ptr()), 1e-8, vp(fh.data_ptr())),        # aliased
        (1, vp(fh.data_ptr()), 0.0, vp(uh.data_ptr())),         # tol <= 0
        (1, vp(fd.data_ptr()), 1e-8, vp(ud.data_ptr())),        # device buffers
    ]
    for nb, r, tol, u in cases:
        rc = lib.st_solve_host(s._h, nb, r, tol, u, 0, ctypes.byref(info))
        assert rc == st.ST_ERR_INVALID_ARG, (nb, rc)
    s.close()


def test_failing_batch_ends_the_stream(st, problem):
    pr, F, _ = problem
    # FP64 FGMRES capped at one iteration cannot reach 1e-14
    s = _solver(st, precision="fp64", outer="fgmres", basis="nodal", max_it=1)
    fh = torch.tensor(F, dtype=torch.float64).pin_memory()
    uh = torch.full_like(fh, 7.0).pin_memory()
    r = s.solve_host(fh, uh, tol=1e-14, check=False)
    assert r["rc"] == st.ST_ERR_NO_CONVERGENCE and r["status"] == st.ST_ERR_NO_CONVERGENCE
    assert torch.all(uh == 7.0)  # the failing batch and the later ones are not written
    # the same handle streams again afterwards: a tolerance one iteration
    # reaches writes every batch
    ok = s.solve_host(fh, uh, tol=0.9)
    assert ok["rel_residual"] <= 0.9
    assert not torch.any(uh == 7.0)
    s.close()

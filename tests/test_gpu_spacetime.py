"""GPU parity of space-time coarsening (Sec. 3.1's multigrid coarsens in space
and time) against the CPU oracle, through the C ABI.

The oracle's hierarchy uses Galerkin coarse operators P^T L P; the library
rediscretises (the same operators: nested spaces, pinned in the oracle tests).
Tolerances as for the time-only V-cycle: one V-cycle 1e-11 relative to the
largest entry (FP64); solves reach 1e-8, and solved to 1e-12 (FP64) / 1e-10
(mixed FP32 V-cycle) they match the oracle's exact solution to 1e-10 /
1e-8."""
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


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# (d, spans, p, N, ratio): schedules with space steps first, mixed, and in 3D
CASES = [(1, (64,), 2, 16, 1.0), (2, (16, 16), 2, 16, 1.0), (2, (16, 12), 3, 8, 4.0),
         (3, (8, 8, 8), 1, 8, 2.0), (2, (36, 20), 2, 4, 1.0)]


@pytest.mark.parametrize("d,spans,p,N,ratio", CASES)
def test_space_time_vcycle_parity(st, d, spans, p, N, ratio):
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    H = S.Hierarchy(pr, space_ratio=ratio)
    assert "x" in H.kinds
    s = st.Solver(d, p, spans, N, space_ratio=ratio)
    assert [k for _, _, k in s.level_shapes()[1:]] == H.kinds
    u0 = inputs.uniform_vector(5, pr.ndofs)
    f = inputs.uniform_vector(6, pr.ndofs)
    ref = S.vcycle(H, f, u=u0.copy())
    u = dev(u0)
    s.vcycle(u, dev(f))
    assert relerr(host(u), ref) <= 1e-11
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32", "mixed_tf32"])
def test_space_time_solve(st, precision):
    """FGMRES with the space-time V-cycle reaches 1e-8 and the exact solution,
    in no more iterations than with time-only coarsening (diffusion-dominated
    slabs, tau / h_x^2 = 256)."""
    d, spans, p, N = 1, (64,), 2, 16
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    f = inputs.uniform_vector(9, pr.ndofs)
    ref = S.forward_subst(pr, f)
    its = {}
    for ratio in (0.0, 1.0):
        s = st.Solver(d, p, spans, N, space_ratio=ratio, precision=precision, outer="fgmres")
        u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
        info = s.solve(dev(f), u, tol=1e-8)
        assert info["rel_residual"] <= 1e-8
        its[ratio] = info["iterations"]
        s.close()
    assert its[1.0] <= its[0.0]
    # solved tighter: the oracle's direct solution to 1e-10 (FP64) / 1e-8
    s = st.Solver(d, p, spans, N, space_ratio=1.0, precision=precision, outer="fgmres",
                  max_it=400)
    u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    info = s.solve(dev(f), u, tol=1e-12 if precision == "fp64" else 1e-10)
    assert relerr(host(u), ref) <= (1e-10 if precision == "fp64" else 1e-8), info
    s.close()


def test_space_time_2d_solve_with_minres_smoother(st):
    """Space coarsening combined with the MinRes spatial solves."""
    d, spans, p, N = 2, (16, 16), 2, 16
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    f = inputs.uniform_vector(10, pr.ndofs)
    ref = S.forward_subst(pr, f)
    s = st.Solver(d, p, spans, N, space_ratio=1.0, spatial_solver="minres", outer="fgmres")
    u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    info = s.solve(dev(f), u, tol=1e-12)
    assert info["rel_residual"] <= 1e-12
    assert relerr(host(u), ref) <= 1e-10
    s.close()


def test_space_time_multi_rhs_equals_single(st):
    d, spans, p, N = 2, (16, 16), 2, 8
    pr = A.Problem(d, spans, p, 2, N)
    fs = [inputs.uniform_vector(41 + k, pr.ndofs) for k in range(2)]
    outs = []
    for f in fs:
        s = st.Solver(d, p, spans, N, space_ratio=1.0)
        u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
        s.vcycle(u, dev(f))
        outs.append(host(u))
        s.close()
    s = st.Solver(d, p, spans, N, space_ratio=1.0, nrhs=2)
    u = torch.zeros(2 * pr.ndofs, dtype=torch.float64, device="cuda")
    s.vcycle(u, dev(np.concatenate(fs)))
    both = host(u)
    assert relerr(both[:pr.ndofs], outs[0]) <= 1e-14
    assert relerr(both[pr.ndofs:], outs[1]) <= 1e-14
    s.close()

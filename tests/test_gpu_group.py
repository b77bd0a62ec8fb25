"""st_solve_group: problems of different shapes (dimension, degree, spans,
slabs, right-hand-side count) solved together, one launch per Krylov vector
operation over all their right-hand sides.  Every member's result must have
the bits of its own st_solve and match the oracle's exact solution to the
mixed-precision tolerance (solved to 1e-10: 1e-8, as the mixed parity
tests); the iteration counts are the single-handle ones."""
import numpy as np
import pytest

from oracle import assemble as A
from oracle import solve as S
from paper_1802_09277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (dim, spans, degree, slabs, nrhs, basis)
MIX = [(2, (16, 16), 2, 8, 2, "spectral"), (1, (32,), 3, 16, 1, "spectral"),
       (3, (6, 6, 6), 2, 4, 1, "spectral"), (2, (12, 20), 1, 32, 3, "nodal"),
       (2, (10, 10), 3, 8, 1, "spectral")]
NE = 2


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
def problems():
    """Per member: oracle load vectors of its right-hand sides (concatenated)
    and their exact solutions."""
    out = []
    for i, (d, spans, p, N, R, _) in enumerate(MIX):
        pr = A.Problem(d, spans, p, NE, N, theta=1.0)
        F = [A.load_from_coeffs(pr, inputs.normal_coeffs(700 + 10 * i + r, pr.ndofs))
             for r in range(R)]
        U = [S.forward_subst(pr, f) for f in F]
        out.append((np.concatenate(F), U, pr.ndofs))
    return out


def _solvers(st, **kw):
    return [st.Solver(d, p, spans, N, ne_per_slab=NE, nrhs=R, precision="mixed_tf32",
                      basis=basis, outer="ir", **kw) for d, spans, p, N, R, basis in MIX]


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_group_equals_single_solves_and_oracle(st, problems):
    tol = 1e-10
    ss = _solvers(st)
    fs = [_dev(F) for F, _, _ in problems]
    solo, solo_info = [], []
    for s, f in zip(ss, fs):
        u = torch.zeros_like(f)
        solo_info.append(s.solve(f, u, tol=tol))
        solo.append(u)
    us = [torch.full_like(f, 3.0) for f in fs]  # overwritten (zero initial guess)
    infos = st.solve_group(ss, fs, us, tol=tol)
    torch.cuda.synchronize()
    for k, (s, u, u1, i1, i2) in enumerate(zip(ss, us, solo, solo_info, infos)):
        assert torch.equal(u, u1), (k, MIX[k])
        assert i2["iterations"] == i1["iterations"] and i2["refinements"] == i1["refinements"]
        assert i2["status"] == 0 and i2["rel_residual"] == i1["rel_residual"]
        _, U, n = problems[k]
        got = u.cpu().numpy()
        for r, ud in enumerate(U):
            err = np.linalg.norm(got[r * n:(r + 1) * n] - ud) / np.linalg.norm(ud)
            assert err <= 1e-8, (k, r, err)
        hist = s.history()  # the member's own refinement history
        assert hist and hist[-1][1] == i1["rel_residual"]
    # a different member order and a subset give the same bits
    order = [3, 0, 4]
    us2 = [torch.zeros_like(fs[k]) for k in order]
    st.solve_group([ss[k] for k in order], [fs[k] for k in order], us2, tol=tol)
    for k, u in zip(order, us2):
        assert torch.equal(u, solo[k])
    # initial guesses: starting from the solutions needs no further step
    ug = [u.clone() for u in solo]
    ig = st.solve_group(ss, fs, ug, tol=tol, use_guess=True)
    assert all(i["refinements"] == 0 for i in ig)
    for u, u1 in zip(ug, solo):
        assert torch.equal(u, u1)
    for s in ss:
        s.close()


def test_group_of_one_is_st_solve(st, problems):
    s = _solvers(st)[0]
    f = _dev(problems[0][0])
    u1, u2 = torch.zeros_like(f), torch.zeros_like(f)
    s.solve(f, u1, tol=1e-10)
    st.solve_group([s], [f], [u2], tol=1e-10)
    assert torch.equal(u1, u2)
    s.close()


def test_group_arguments_rejected(st, problems):
    ss = _solvers(st)
    fs = [_dev(F) for F, _, _ in problems]
    us = [torch.zeros_like(f) for f in fs]
    with pytest.raises(st.StError) as e:  # the same handle twice
        st.solve_group([ss[0], ss[0]], [fs[0], fs[0]], [us[0], torch.zeros_like(fs[0])])
    assert e.value.code == st.ST_ERR_INVALID_ARG
    fp64 = st.Solver(2, 2, (8, 8), 4, precision="fp64", outer="fgmres")
    f64 = torch.zeros(fp64.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(st.StError) as e:  # another kind of handle
        st.solve_group([ss[1], fp64], [fs[1], f64], [us[1], torch.zeros_like(f64)])
    assert e.value.code == st.ST_ERR_UNSUPPORTED
    other = st.Solver(1, 2, (16,), 4, nrhs=1, precision="mixed_tf32", basis="spectral",
                      outer="ir", gmres_restart=7)
    fo = torch.ones(other.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(st.StError) as e:  # restart lengths differ
        st.solve_group([ss[1], other], [fs[1], fo], [us[1], torch.zeros_like(fo)])
    assert e.value.code == st.ST_ERR_INVALID_ARG
    big = [st.Solver(1, 2, (16,), 4, nrhs=32, precision="mixed_tf32", basis="spectral",
                     outer="ir")]
    fb = torch.ones(big[0].ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(st.StError) as e:  # more than 32 right-hand sides in all
        st.solve_group([big[0], ss[1]], [fb, fs[1]], [torch.zeros_like(fb), us[1]])
    assert e.value.code == st.ST_ERR_INVALID_ARG
    for s in ss + [fp64, other] + big:
        s.close()

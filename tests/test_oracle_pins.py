"""Pins of the CPU oracle to facts fixed outside the oracle itself: the
paper's printed tables and closed forms, textbook identities, library
routines and convergence rates (arXiv:1802.09277)."""
import os

import numpy as np
import pytest
import scipy.interpolate as si
import scipy.linalg as sl
import scipy.sparse as sp

from oracle import assemble as A
from oracle import bspline as bs
from oracle import solve as S
from paper_1802_09277_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# B-splines (Sec. 2.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_matches_scipy_bspline(p):
    kn = bs.open_knots(0.0, 1.0, 7, p)
    x = np.linspace(0.0, 1.0, 101)
    B = bs.basis(kn, p, x)
    D = bs.basis_deriv(kn, p, x)
    nb = bs.n_basis(kn, p)
    for i in range(nb):
        c = np.zeros(nb)
        c[i] = 1.0
        spl = si.BSpline(kn, c, p, extrapolate=False)
        ref = np.nan_to_num(spl(x))
        ref[-1] = spl(1.0 - 1e-15)  # left limit at the right end
        assert np.allclose(B[:, i], ref, atol=1e-12)
        dref = np.nan_to_num(spl.derivative()(x[:-1]))
        assert np.allclose(D[:-1, i], dref, atol=1e-10)
    assert np.allclose(B.sum(axis=1), 1.0)  # partition of unity


# --------------------------------------------------------------------------
# Space matrices
# --------------------------------------------------------------------------

def test_p1_space_matrices_closed_form():
    """p = 1 hat functions: M1 = h/6 tridiag(1,4,1), K1 = 1/h tridiag(-1,2,-1)."""
    s = 9
    h = 1.0 / s
    M1, K1 = A.space_matrices(s, 1)
    n = s - 1
    T = lambda a, b: (np.diag(np.full(n, a)) + np.diag(np.full(n - 1, b), 1)
                      + np.diag(np.full(n - 1, b), -1))
    assert np.allclose(M1, h / 6 * T(4, 1), atol=1e-15)
    assert np.allclose(K1, T(2, -1) / h, atol=1e-12)


@pytest.mark.parametrize("p", [2, 3])
def test_space_matrices_identities(p):
    """Interior M1, K1 are SPD; the generalized eigenvalues of (K1, M1)
    approximate the Dirichlet Laplacian eigenvalues (k pi)^2."""
    M1, K1 = A.space_matrices(32, p)
    assert np.allclose(M1, M1.T) and np.allclose(K1, K1.T)
    lam = sl.eigh(K1, M1, eigvals_only=True)
    assert lam.min() > 0
    k = np.arange(1, 5)
    assert np.allclose(lam[:4], (k * np.pi) ** 2, rtol=1e-4)
    # mass of the constant: 1^T M1_full 1 = |Omega|, approximated by the
    # interior block plus the two removed boundary functions -> row sums
    # of the interior M1 equal int phi_i for functions away from the ends
    kn = bs.open_knots(0.0, 1.0, 32, p)
    mid = slice(p, 32 + p - 2 - p)
    integral = (kn[p + 1:len(kn)] - kn[:len(kn) - p - 1]) / (p + 1)
    assert np.allclose(M1.sum(axis=1)[mid], integral[1:-1][mid], atol=1e-14)


# --------------------------------------------------------------------------
# Time matrices (Eq. 2.6)
# --------------------------------------------------------------------------

def test_remark_3_2_closed_form():
    """theta = 0, p = 1, uniform: K_t = 1/2 [[1,1],[-1,0,1],...,[-1,1]],
    M_t = C_n tridiag(1,4,1) with corners 2, C_n = h/6 (Remark 3.2)."""
    for ne in (2, 3, 6):
        Kt, Mt = A.time_matrices(1.0, ne, 1, 0.0)
        n = ne + 1
        K = np.diag(np.full(n - 1, 1.0), 1) - np.diag(np.full(n - 1, 1.0), -1)
        K[0, 0] = 1.0
        K[-1, -1] = 1.0
        M = 4 * np.eye(n) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        M[0, 0] = M[-1, -1] = 2.0
        assert np.allclose(Kt, K / 2, atol=1e-14)
        assert np.allclose(Mt, M / (6 * ne), atol=1e-14)


@pytest.mark.parametrize("p,ne,delta", [(1, 3, 0.1), (2, 4, 0.05), (3, 2, 0.3), (4, 5, 0.0)])
def test_lemma_3_1_quadratic_forms(p, ne, delta):
    """Lemma 3.1: v^T K_t v = delta ||v'||^2 + (v(t_n)^2 + v(t_{n-1})^2)/2 and
    v^T M_t v = ||v||^2 + delta (v(t_n)^2 - v(t_{n-1})^2)/2, with the norms
    integrated independently through scipy's BSpline and Gauss quadrature."""
    tau = 0.7
    Kt, Mt = A.time_matrices(tau, ne, p, delta)
    kn = bs.open_knots(0.0, tau, ne, p)
    rng = np.random.default_rng(p * 10 + ne)
    for _ in range(3):
        v = rng.standard_normal(ne + p)
        spl = si.BSpline(kn, v, p)
        dsp = spl.derivative()
        xg, wg = np.polynomial.legendre.leggauss(12)
        br = np.linspace(0.0, tau, ne + 1)
        t = np.concatenate([0.5 * (b - a) * (xg + 1) + a for a, b in zip(br[:-1], br[1:])])
        w = np.concatenate([0.5 * (b - a) * wg for a, b in zip(br[:-1], br[1:])])
        l2 = np.sum(w * spl(t) ** 2)
        h1 = np.sum(w * dsp(t) ** 2)
        v0, v1 = spl(0.0), spl(tau)
        assert np.isclose(v @ Kt @ v, delta * h1 + 0.5 * (v1 ** 2 + v0 ** 2), rtol=1e-12)
        assert np.isclose(v @ Mt @ v, l2 + 0.5 * delta * (v1 ** 2 - v0 ** 2), rtol=1e-12)


def _table2():
    rows = []
    for line in open(os.path.join(GOLDEN, "table2_min_re_eig.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((int(f[1]), float(f[2]), f[3:]))
    return rows


@pytest.mark.parametrize("ne,theta,vals", _table2())
def test_table_2_min_real_part(ne, theta, vals):
    """Table 2 on [0,1]: smallest Re lambda(K_t, M_t); '*' <=> M_t has an
    eigenvalue with negative real part.  h = time element length."""
    for p, printed in zip(range(1, 8), vals):
        Kt, Mt = A.time_matrices(1.0, ne, p, theta / ne)
        mt_neg = np.linalg.eigvals(Mt).real.min() < 0
        if printed == "*":
            assert mt_neg, (ne, theta, p)
            continue
        assert not mt_neg
        val = sl.eigvals(Kt, Mt).real.min()
        ref = float(printed)
        if ref >= 1.0:
            # 1-2 digit print; a few theta >= 1 entries differ by up to 4.5 %
            assert abs(val - ref) <= max(0.1, 0.045 * ref), (ne, theta, p, val, ref)
        else:
            assert 1 / 1.6 <= val / ref <= 1.6, (ne, theta, p, val, ref)


def test_table_1_cond_x():
    """Table 1 (theta = 0.01, slab length 0.1): cond(X) with unit-norm
    eigenvector columns; printed column 'p' = degree p + 1 (see fixture)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_cond_x.txt"))
            if l.strip() and not l.startswith("#")]
    for f in rows:
        ne = int(f[0])
        for label, printed in zip(range(2, 9), f[1:]):
            p = label + 1
            Kt, Mt = A.time_matrices(0.1, ne, p, 0.01 * 0.1 / ne)
            _, X = sl.eig(Kt, Mt)
            X = X / np.linalg.norm(X, axis=0)
            c = np.linalg.cond(X)
            ref = float(printed)
            if "e+" in printed:
                assert 0.5 * ref <= c <= 10 * ref, (ne, label, c, ref)
            else:
                assert abs(c - ref) <= 2e-3 * ref + 1.0, (ne, label, c, ref)


def test_coupling_is_rank_one_corner():
    """Open knots: N_t = e_1 e_{N_t}^T."""
    Nt = A.coupling_matrix(0.3, 3, 2)
    E = np.zeros((5, 5))
    E[0, -1] = 1.0
    assert np.allclose(Nt, E)


# --------------------------------------------------------------------------
# Global system, load vectors, error norm
# --------------------------------------------------------------------------

def test_dg_norm_of_exact_solution_closed_form():
    """With u_h = 0 the dG norm of u = sin(pi x) sin(pi t) on (0,1)^2 is
    pi^2 (1 + delta) / 4 (all jumps and u(T) vanish)."""
    pr = A.Problem(1, (6,), 2, 2, 3, theta=1.0)
    e = A.dg_error_manufactured(pr, np.zeros(pr.ndofs))
    assert np.isclose(e ** 2, np.pi ** 2 * (1 + pr.delta) / 4, rtol=1e-10)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_manufactured_convergence_rate(p):
    """Remark 2.1: ||u - u_h||_dG = O(h^p) under joint refinement."""
    errs = []
    for k in range(3):
        pr = A.Problem(1, (4 * 2 ** k,), p, 2 ** k, 4, theta=1.0)
        uh = S.direct(A.assemble_L(pr), A.manufactured_load(pr))
        errs.append(A.dg_error_manufactured(pr, uh))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p - 0.2, rates


def test_manufactured_2d_error_small():
    pr = A.Problem(2, (8, 8), 2, 2, 4, theta=1.0)
    uh = S.direct(A.assemble_L(pr), A.manufactured_load(pr))
    pr2 = A.Problem(2, (16, 16), 2, 4, 4, theta=1.0)
    uh2 = S.direct(A.assemble_L(pr2), A.manufactured_load(pr2))
    e1 = A.dg_error_manufactured(pr, uh)
    e2 = A.dg_error_manufactured(pr2, uh2)
    assert np.log2(e1 / e2) > 1.7


def test_coercivity():
    """a_h(v,v) > 0 for random v (the lemma after Sec. 2.2)."""
    pr = A.Problem(2, (5, 4), 2, 2, 3, theta=1.0)
    L = A.assemble_L(pr)
    rng = np.random.default_rng(0)
    for _ in range(5):
        v = rng.standard_normal(pr.ndofs)
        assert v @ (L @ v) > 0


def test_system_structure():
    """Eq. 2.4: blocks (n,n) = A, (n,n-1) = -B, zero elsewhere."""
    pr = A.Problem(1, (5,), 2, 2, 4, theta=1.0)
    L = A.assemble_L(pr).toarray()
    Ab, Bb = (m.toarray() for m in A.slab_blocks(pr))
    m = pr.Nt * pr.Nx
    for i in range(pr.N):
        for j in range(pr.N):
            blk = L[i * m:(i + 1) * m, j * m:(j + 1) * m]
            ref = Ab if i == j else (-Bb if j == i - 1 else 0 * Ab)
            assert np.allclose(blk, ref)


@pytest.mark.parametrize("d,spans,p,ne", [(1, (7,), 3, 2), (2, (5, 4), 2, 3),
                                           (3, (5, 4, 6), 2, 2), (3, (4, 6, 5), 1, 4)])
def test_matrix_free_slab_residual_matches_assembled_blocks(d, spans, p, ne):
    """The matrix-free block row of Eq. 2.4 (each Kronecker factor of Eq. 2.5
    along its own axis) equals f - A u + B u_prev with the sparse A, B built
    from the bilinear forms, on grids whose axes all differ (an axis mix-up
    fails) with the non-symmetric SUPG time matrices (a transposed factor
    fails); the first slab has no coupling.  The magnitude form bounds the
    residual and the sparse blocks' absolute terms entry-wise."""
    pr = A.Problem(d, spans, p, ne, 3, theta=1.0)
    Ab, Bb = A.slab_blocks(pr)
    m = pr.Nt * pr.Nx
    rng = np.random.default_rng(11)
    u, up, f = (rng.standard_normal(m) for _ in range(3))
    ref = f - Ab @ u + Bb @ up
    got = A.slab_residual_kron(pr, f, u, up)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    got0 = A.slab_residual_kron(pr, f, u, None)
    assert np.abs(got0 - (f - Ab @ u)).max() <= 1e-13 * np.abs(f - Ab @ u).max()
    mag = A.slab_residual_kron(pr, f, u, up, magnitude=True)
    lower = np.abs(f) + abs(Ab) @ np.abs(u) + abs(Bb) @ np.abs(up)
    assert (mag >= lower * (1 - 1e-13)).all()
    assert (mag >= np.abs(ref)).all()


def test_load_from_coeffs_by_brute_force_quadrature():
    """f = sum c_j phi_j integrated against the test functions
    phi_i + delta d_t phi_i by dense tensor quadrature (1D space)."""
    pr = A.Problem(1, (5,), 2, 2, 2, theta=1.0)
    c = inputs.normal_coeffs(7, pr.ndofs).reshape(pr.N, pr.Nt, pr.Nx)
    f = A.load_from_coeffs(pr, c).reshape(pr.N, pr.Nt, pr.Nx)
    knx = bs.open_knots(0.0, 1.0, 5, 2)
    x, wx = bs.element_quadrature(knx, 6)
    Bx = bs.basis(knx, 2, x)[:, 1:-1]
    for n in range(pr.N):
        knt = bs.open_knots(n * pr.tau, (n + 1) * pr.tau, pr.ne, pr.p)
        t, wt = bs.element_quadrature(knt, 6)
        Bt = bs.basis(knt, 2, t)
        Dt = bs.basis_deriv(knt, 2, t)
        fval = np.einsum('ta,ai,xi->tx', Bt, c[n], Bx)
        test = Bt + pr.delta * Dt
        ref = np.einsum('t,x,tx,ta,xi->ai', wt, wx, fval, test, Bx)
        assert np.allclose(f[n], ref, atol=1e-13)


def test_bumps_load_by_brute_force_quadrature():
    pr = A.Problem(2, (4, 3), 2, 2, 2, theta=1.0)
    cen, wid, amp = inputs.gaussian_bumps(3, count=3, dim=3)
    f = A.bumps_load(pr, cen, wid, amp, npts=12).reshape(pr.N, pr.Nt, pr.n_axis[1], pr.n_axis[0])
    q = 12
    knx = bs.open_knots(0.0, 1.0, 4, 2)
    kny = bs.open_knots(0.0, 1.0, 3, 2)
    x, wx = bs.element_quadrature(knx, q)
    y, wy = bs.element_quadrature(kny, q)
    Bx = bs.basis(knx, 2, x)[:, 1:-1]
    By = bs.basis(kny, 2, y)[:, 1:-1]
    for n in range(pr.N):
        knt = bs.open_knots(n * pr.tau, (n + 1) * pr.tau, pr.ne, pr.p)
        t, wt = bs.element_quadrature(knt, q)
        test = bs.basis(knt, 2, t) + pr.delta * bs.basis_deriv(knt, 2, t)
        T, Y, X = np.meshgrid(t, y, x, indexing="ij")
        fv = sum(a * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (T - c[2]) ** 2) / (2 * w * w))
                 for c, w, a in zip(cen, wid, amp))
        ref = np.einsum('t,y,x,tyx,ta,yj,xi->aji', wt, wy, wx, fv, test, By, Bx)
        assert np.allclose(f[n], ref, rtol=1e-9, atol=1e-12)
    # a subset of slabs, in the order asked for, gives the same rows
    sub = A.bumps_load(pr, cen, wid, amp, npts=12, slabs=[1, 0]).reshape(f.shape)
    assert np.array_equal(sub[0], f[1]) and np.array_equal(sub[1], f[0])


# --------------------------------------------------------------------------
# Solvers (Sec. 3.1)
# --------------------------------------------------------------------------

def test_direct_and_forward_substitution_agree():
    pr = A.Problem(2, (6, 5), 2, 2, 5, theta=1.0)
    f = inputs.normal_coeffs(1, pr.ndofs)
    L = A.assemble_L(pr)
    u1 = S.direct(L, f)
    u2 = S.forward_subst(pr, f)
    assert np.linalg.norm(L @ u1 - f) <= 1e-12 * np.linalg.norm(f)
    assert np.allclose(u1, u2, rtol=0, atol=1e-12 * np.abs(u1).max())


def test_one_slab_exact_smoother_is_direct_solve():
    """With one slab and omega = 1, one block-Jacobi step from u = 0 is the
    direct solve."""
    pr = A.Problem(2, (5, 5), 3, 2, 1, theta=1.0)
    L = A.assemble_L(pr)
    f = inputs.normal_coeffs(2, pr.ndofs)
    lev = S.Level(L, 1, pr.Nt * pr.Nx)
    u = S.jacobi_step(lev, np.zeros(pr.ndofs), f, omega=1.0)
    assert np.allclose(u, S.direct(L, f), atol=1e-12)


def test_exact_solution_is_smoother_fixed_point():
    pr = A.Problem(1, (8,), 2, 2, 4, theta=1.0)
    L = A.assemble_L(pr)
    f = inputs.normal_coeffs(3, pr.ndofs)
    u = S.direct(L, f)
    lev = S.Level(L, pr.N, pr.Nt * pr.Nx)
    assert np.allclose(S.jacobi_step(lev, u, f), u, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_time_prolongation_reproduces_coarse_functions(p):
    """P_t maps coarse coefficients to fine ones that evaluate to the same
    function (brute force at sample points); constants are preserved."""
    tau, ne = 0.25, 3
    Pt = S.time_prolongation(tau, ne, p)
    nt = ne + p
    assert np.allclose(Pt @ np.ones(nt), 1.0)
    kc = bs.open_knots(0.0, 2 * tau, ne, p)
    rng = np.random.default_rng(p)
    c = rng.standard_normal(nt)
    for q in range(2):
        kf = bs.open_knots(q * tau, (q + 1) * tau, ne, p)
        t = np.linspace(q * tau + 1e-9, (q + 1) * tau - 1e-9, 37)
        fine = bs.basis(kf, p, t) @ (Pt[q * nt:(q + 1) * nt] @ c)
        assert np.allclose(fine, bs.basis(kc, p, t) @ c, atol=1e-12)


def test_galerkin_coarse_operator_is_frozen_delta_rediscretisation():
    """P^T L P equals the coarse rediscretisation with theta*h frozen at the
    fine value (two independent routes to the coarse operator)."""
    pr = A.Problem(2, (4, 5), 2, 2, 4, theta=1.0)
    L = A.assemble_L(pr)
    P = S.prolongation(pr)
    Lc = (P.T @ L @ P).toarray()
    Lr = A.assemble_L(pr.coarse()).toarray()
    assert np.abs(Lc - Lr).max() <= 1e-13 * np.abs(Lr).max()


def test_fgmres_on_library_solve():
    """FGMRES with the identity preconditioner on a small well-conditioned
    non-symmetric matrix reproduces numpy.linalg.solve."""
    rng = np.random.default_rng(4)
    M = np.eye(40) * 4 + rng.standard_normal((40, 40)) * 0.3
    b = rng.standard_normal(40)
    u, it, _ = S.fgmres(sp.csr_matrix(M), b, lambda v: v, tol=1e-13, restart=15)
    assert np.allclose(u, np.linalg.solve(M, b), atol=1e-11)


def test_single_slab_multigrid_is_exact():
    pr = A.Problem(2, (6, 6), 2, 2, 1, theta=1.0)
    H = S.Hierarchy(pr)
    f = inputs.normal_coeffs(5, pr.ndofs)
    u, it, _ = S.mg_solve(H, f, tol=1e-12)
    assert it == 1


@pytest.mark.parametrize("d,spans,p,N", [(1, (16,), 2, 8), (2, (8, 8), 3, 8), (1, (10,), 1, 16)])
def test_multigrid_and_fgmres_converge_to_direct(d, spans, p, N):
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    H = S.Hierarchy(pr)
    f = A.load_from_coeffs(pr, inputs.normal_coeffs(6, pr.ndofs))
    ud = S.direct(H.levels[0].L, f)
    u, it, hist = S.mg_solve(H, f, tol=1e-11, maxit=100)
    assert it < 60 and hist[-1] <= 1e-11
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
    u2, it2, _ = S.fgmres(H.levels[0].L, f, lambda v: S.vcycle(H, v), tol=1e-11)
    assert it2 <= it
    assert np.linalg.norm(u2 - ud) <= 1e-9 * np.linalg.norm(ud)


# --------------------------------------------------------------------------
# Space coarsening (Sec. 3.1 coarsens in space and time)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("s", [4, 8, 14])
def test_space_prolongation_reproduces_coarse_functions(p, s):
    """P_x expresses every interior coarse B-spline (s/2 spans) exactly in the
    interior fine ones (s spans): evaluated at random points, B_c = B_f P_x."""
    Px = S.space_prolongation_1d(s, p)
    x = np.random.default_rng(p * 100 + s).uniform(0.0, 1.0, 200)
    Bf = bs.basis(bs.open_knots(0.0, 1.0, s, p), p, x)[:, 1:-1]
    Bc = bs.basis(bs.open_knots(0.0, 1.0, s // 2, p), p, x)[:, 1:-1]
    assert Px.shape == (s + p - 2, s // 2 + p - 2)
    assert np.allclose(Bf @ Px, Bc, atol=1e-12)


@pytest.mark.parametrize("d,spans,p", [(1, (8,), 2), (2, (8, 6), 2), (2, (4, 8), 3), (3, (4, 4, 6), 1)])
def test_galerkin_space_coarse_operator_is_rediscretisation(d, spans, p):
    """Nested spatial spaces: P^T L P with the space prolongation equals L
    assembled on the grid with halved spans (same slabs, same delta)."""
    pr = A.Problem(d, spans, p, 2, 3, theta=1.0)
    P = S.space_prolongation(pr)
    Lc = (P.T @ A.assemble_L(pr) @ P).toarray()
    ref = A.assemble_L(pr.space_coarse()).toarray()
    assert np.abs(Lc - ref).max() <= 1e-12 * np.abs(ref).max()


def test_space_time_hierarchy_rule_and_convergence():
    """Above tau / h^2 = 1 the hierarchy coarsens in space first (diffusion-
    dominated slabs), then in time; the multigrid iteration converges to the
    direct solution, in fewer iterations than with time-only coarsening, and
    its coarsest level is much smaller."""
    pr = A.Problem(1, (64,), 2, 2, 16, theta=1.0)
    assert S.space_time_ratio(pr) == pytest.approx(256.0)
    f = inputs.uniform_vector(4, pr.ndofs)
    ref = S.direct(A.assemble_L(pr), f)
    Ht = S.Hierarchy(pr)
    Hx = S.Hierarchy(pr, space_ratio=1.0)
    assert "".join(Ht.kinds) == "tttt"
    assert "".join(Hx.kinds) == "xxxxtxttt"
    ut, it_t, _ = S.mg_solve(Ht, f, tol=1e-8)
    ux, it_x, _ = S.mg_solve(Hx, f, tol=1e-8)
    assert np.linalg.norm(ux - ref) <= 1e-6 * np.linalg.norm(ref)
    assert it_x < it_t
    assert Hx.levels[-1].L.shape[0] * 10 < Ht.levels[-1].L.shape[0]


# --------------------------------------------------------------------------
# The V-cycle as a linear iteration (Sec. 3.1): one cycle maps the error
# e = u* - u to E e with the multigrid error propagator written densely,
#   two levels:  E_J = S^nu2 (I - P L_c^{-1} P^T L) S^nu1,
#   more levels: E_l = S^nu2 (I - P (I - E_{l+1}) L_{l+1}^{-1} P^T L) S^nu1,
# S = I - omega D^{-1} L, D = blockdiag(A_n) (inverted densely here), and
# the coarsest level solved exactly.  A dropped smoothing loop, a restriction
# of f instead of the residual, a missing coarse correction or a wrong
# damping all change E.
# --------------------------------------------------------------------------

def _dense_propagator(H, lvl, nu1, nu2, omega):
    L = H.levels[lvl].L.toarray()
    n = L.shape[0]
    if lvl == len(H.levels) - 1:
        return np.zeros((n, n))  # exact coarsest solve: no error left
    m = H.levels[lvl].m
    Dinv = np.zeros_like(L)
    for b in range(n // m):
        sl_ = slice(b * m, (b + 1) * m)
        Dinv[sl_, sl_] = np.linalg.inv(L[sl_, sl_])
    Sm = np.eye(n) - omega * Dinv @ L
    P = H.P[lvl].toarray()
    Lc = H.levels[lvl + 1].L.toarray()
    Ec = _dense_propagator(H, lvl + 1, nu1, nu2, omega)
    # one cycle from zero on the coarse level returns (I - E_c) Lc^{-1} r_c
    C = np.eye(n) - P @ (np.eye(Lc.shape[0]) - Ec) @ np.linalg.solve(Lc, P.T @ L)
    return np.linalg.matrix_power(Sm, nu2) @ C @ np.linalg.matrix_power(Sm, nu1)


@pytest.mark.parametrize("N,space_ratio", [(2, 0.0), (4, 0.0), (8, 0.0), (4, 1.0)])
@pytest.mark.parametrize("nu1,nu2", [(1, 1), (2, 1), (0, 1), (1, 0), (2, 2)])
def test_vcycle_is_the_multigrid_error_propagator(N, space_ratio, nu1, nu2):
    pr = A.Problem(1, (8,), 2, 2, N, theta=1.0)
    H = S.Hierarchy(pr, space_ratio=space_ratio)
    assert len(H.levels) >= 2
    if space_ratio > 0:
        assert "x" in H.kinds  # the space-coarsening branch is exercised too
    rng = np.random.default_rng(100 * N + 10 * nu1 + nu2)
    f = rng.standard_normal(pr.ndofs)
    u0 = rng.standard_normal(pr.ndofs)
    ustar = np.linalg.solve(H.levels[0].L.toarray(), f)
    u1 = S.vcycle(H, f, nu1=nu1, nu2=nu2, omega=0.5, u=u0.copy())
    E = _dense_propagator(H, 0, nu1, nu2, 0.5)
    e1 = E @ (ustar - u0)
    assert np.linalg.norm((ustar - u1) - e1) <= 1e-11 * np.linalg.norm(ustar - u0)
    # and the cycle contracts the error (it is a convergent iteration)
    assert np.max(np.abs(np.linalg.eigvals(E))) < 1.0


def test_vcycle_propagator_rejects_planted_mistakes():
    """The propagator check above catches the plausible mistakes: a cycle
    without post-smoothing, one that restricts f instead of the residual,
    and one without the coarse correction all move the error elsewhere."""
    pr = A.Problem(1, (8,), 2, 2, 4, theta=1.0)
    H = S.Hierarchy(pr)
    rng = np.random.default_rng(5)
    f = rng.standard_normal(pr.ndofs)
    u0 = rng.standard_normal(pr.ndofs)
    ustar = np.linalg.solve(H.levels[0].L.toarray(), f)
    e1 = _dense_propagator(H, 0, 1, 1, 0.5) @ (ustar - u0)

    def cycle(lvl, f, u, variant):
        lev = H.levels[lvl]
        if lvl == len(H.levels) - 1:
            return H.coarse_lu.solve(f)
        u = S.jacobi_step(lev, u, f, 0.5)
        r = f - lev.L @ u
        rc = H.P[lvl].T @ (f if variant == "restrict_f" else r)
        if variant != "no_coarse":
            u = u + H.P[lvl] @ cycle(lvl + 1, rc, np.zeros_like(rc), variant)
        if variant != "no_post":
            u = S.jacobi_step(lev, u, f, 0.5)
        return u

    for variant in ("no_post", "restrict_f", "no_coarse"):
        ub = cycle(0, f, u0.copy(), variant)
        assert np.linalg.norm((ustar - ub) - e1) > 1e-3 * np.linalg.norm(ustar - u0), variant

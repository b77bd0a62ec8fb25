"""Pins of the oracle's inexact spatial solves (Sec. 3.3-3.5, Theorems 3.2
and 3.3, Algorithm 1 of arXiv:1802.09277) to facts fixed outside the oracle:
the theorems' spectral bounds, the equivalence of the rescaled block system,
brute-force minimal residuals over explicit Krylov spaces, the two-interval
MinRes convergence bound, and exact sparse-LU slab solves."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import assemble as A
from oracle import minres as MR


def _space(d, spans, p):
    prob = A.Problem(d, spans, p, 2, 1)
    Mx, Kx = A.spatial_operators(prob)
    return Mx, Kx


def _schur_blocks(p, ne, theta, tau=0.1):
    Kt, Mt = A.time_matrices(tau, ne, p, theta * tau / ne)
    T, X, Y, blocks = MR.real_schur_standard(Kt, Mt)
    return Kt, Mt, T, X, Y, blocks


# --------------------------------------------------------------------------
# Real Schur form with standardised blocks (Sec. 3.5)
# --------------------------------------------------------------------------

def test_standardize_2x2_rotation():
    rng = np.random.default_rng(11)
    done = 0
    while done < 20:
        B = rng.standard_normal((2, 2)) * 10
        ev = np.linalg.eigvals(B)
        if abs(ev[0].imag) < 1e-3:
            continue
        G = MR.standardize_2x2(B)
        C = G.T @ B @ G
        assert np.allclose(G.T @ G, np.eye(2), atol=1e-14)
        assert abs(C[0, 0] - C[1, 1]) <= 1e-12 * np.abs(B).max()
        assert C[0, 1] * C[1, 0] < 0  # complex pair: off-diagonals of opposite sign
        got = np.sort_complex(np.linalg.eigvals(C))
        assert np.allclose(got, np.sort_complex(ev), rtol=1e-12)
        # eigenvalues alpha +- i sqrt|beta1 beta2| (Sec. 3.5)
        assert np.isclose(abs(ev[0].imag), np.sqrt(abs(C[0, 1] * C[1, 0])), rtol=1e-12)
        assert np.isclose(ev[0].real, C[0, 0], rtol=1e-12)
        done += 1


@pytest.mark.parametrize("p,ne,theta", [(1, 2, 1.0), (2, 2, 1.0), (2, 4, 0.1), (3, 2, 0.1),
                                        (4, 4, 0.1), (6, 2, 0.1)])
def test_real_schur_standard_factors(p, ne, theta):
    Kt, Mt, T, X, Y, blocks = _schur_blocks(p, ne, theta)
    n = Kt.shape[0]
    assert sum(m for _, m in blocks) == n
    assert np.allclose(X.T @ X, np.eye(n), atol=1e-12)
    S = np.linalg.solve(Mt, Kt)
    assert np.allclose(X @ T @ X.T, S, atol=1e-10 * np.abs(S).max())
    # Eq. 3.1 factors: Y K_t X = T, Y M_t X = I
    assert np.allclose(Y @ Mt @ X, np.eye(n), atol=1e-10)
    assert np.allclose(Y @ Kt @ X, T, atol=1e-9 * np.abs(T).max())
    for (b, m) in blocks:
        assert np.all(T[b + m:, b:b + m] == 0.0)
        if m == 2:
            assert T[b, b] == pytest.approx(T[b + 1, b + 1], rel=1e-12)
            assert T[b, b] > 0 and T[b, b + 1] * T[b + 1, b] < 0
        else:
            assert T[b, b] > 0
    ev = np.sort_complex(np.linalg.eigvals(S))
    mine = []
    for (b, m) in blocks:
        if m == 1:
            mine.append(T[b, b])
        else:
            w = np.sqrt(abs(T[b, b + 1] * T[b + 1, b]))
            mine += [T[b, b] + 1j * w, T[b, b] - 1j * w]
    assert np.allclose(np.sort_complex(np.array(mine)), ev, rtol=1e-10)


# --------------------------------------------------------------------------
# Theorems 3.2 / 3.3: symmetric form and preconditioner
# --------------------------------------------------------------------------

def _block_params():
    """(alpha, beta1, beta2): the time Schur blocks of several degrees and
    theta, random pairs with extreme ratios |beta1|/|beta2|, and complex
    shifts alpha + i beta in Theorem 3.2's form (beta1 = -beta, beta2 = beta)."""
    out = []
    for p, ne, th in [(2, 2, 1.0), (3, 4, 0.1), (4, 2, 0.1)]:
        _, _, T, _, _, blocks = _schur_blocks(p, ne, th)
        out += [(T[b, b], T[b, b + 1], T[b + 1, b]) for b, m in blocks if m == 2]
    rng = np.random.default_rng(5)
    for _ in range(4):
        a = 10 ** rng.uniform(-2, 3)
        b1 = 10 ** rng.uniform(-3, 3)
        b2 = -(10 ** rng.uniform(-3, 3))
        out.append((a, b1, b2) if rng.random() < 0.5 else (a, b2, b1))
    out += [(1.0, -50.0, 50.0), (30.0, -0.5, 0.5)]
    return out


@pytest.mark.parametrize("d,spans,p", [(1, (9,), 2), (2, (4, 5), 2), (2, (3, 4), 3)])
def test_theorem_3_3_spectral_bound(d, spans, p):
    """Generalized eigenvalues of (Abar, P) lie in 1/sqrt2 <= |lambda| <= 1."""
    Mx, Kx = _space(d, spans, p)
    for (a, b1, b2) in _block_params():
        Abar, P, s, _ = MR.block_system(Kx, Mx, a, b1, b2)
        Ad, Pd = Abar.toarray(), P.toarray()
        assert np.allclose(Ad, Ad.T, atol=1e-12 * np.abs(Ad).max())
        lam = sl.eigh(Ad, Pd, eigvals_only=True)
        mag = np.abs(lam)
        assert mag.min() >= 1 / np.sqrt(2) * (1 - 1e-10)
        assert mag.max() <= 1 + 1e-10
        assert mag.max() / mag.min() <= np.sqrt(2) * (1 + 1e-10)  # cond <= sqrt 2


def test_theorem_3_3_bound_needs_its_shift():
    """The shift alpha + sqrt|beta1 beta2| matters: with alpha + max|beta| the
    bound fails for an unbalanced pair (guards the preconditioner's shift)."""
    Mx, Kx = _space(2, (4, 5), 2)
    a, b1, b2 = 5.0, 200.0, -0.5
    Abar, P, s, (a1, a2) = MR.block_system(Kx, Mx, a, b1, b2)
    Pw = sp.block_diag([a1 * (Kx + (a + 200.0) * Mx), a2 * (Kx + (a + 200.0) * Mx)]).toarray()
    lam = np.abs(sl.eigh(Abar.toarray(), Pw, eigvals_only=True))
    assert lam.max() / lam.min() > np.sqrt(2) * 1.5


@pytest.mark.parametrize("a,b1,b2", [(3.0, -7.0, 2.0), (40.0, 100.0, -3.0), (1.0, -0.2, 5.0)])
def test_rescaled_block_system_is_equivalent(a, b1, b2):
    """Abar [x; -y] = [|beta2| f; |beta1| g] has the solution of the original
    non-symmetric 2x2 block system (Sec. 3.5)."""
    Mx, Kx = _space(2, (5, 4), 2)
    rng = np.random.default_rng(3)
    m = Mx.shape[0]
    f, g = rng.standard_normal(m), rng.standard_normal(m)
    Kc = Kx + a * Mx
    orig = sp.bmat([[Kc, b1 * Mx], [b2 * Mx, Kc]]).toarray()
    xy = np.linalg.solve(orig, np.concatenate([f, g]))
    Abar, _, _, (a1, a2) = MR.block_system(Kx, Mx, a, b1, b2)
    w = np.linalg.solve(Abar.toarray(), np.concatenate([a1 * f, a2 * g]))
    assert np.allclose(w[:m], xy[:m], rtol=1e-10, atol=1e-12)
    assert np.allclose(-w[m:], xy[m:], rtol=1e-10, atol=1e-12)


def test_theorem_3_2_is_the_balanced_case():
    """A complex shift alpha + i beta: (K + lambda M)(x + i y) = f + i g
    is the 2x2 block with beta1 = -beta, beta2 = beta, and Theorem 3.3's P is
    |beta| times Theorem 3.2's diag(K + (alpha+|beta|) M)."""
    Mx, Kx = _space(2, (4, 4), 2)
    a, beta = 7.0, -3.0
    rng = np.random.default_rng(8)
    m = Mx.shape[0]
    f, g = rng.standard_normal(m), rng.standard_normal(m)
    z = spla.spsolve(sp.csc_matrix(Kx + (a + 1j * beta) * Mx), f + 1j * g)
    x, y, it = MR.block_solve(Kx, Mx, a, -beta, beta, f, g, tol=1e-13)
    assert np.allclose(x, z.real, rtol=1e-9, atol=1e-11)
    assert np.allclose(y, z.imag, rtol=1e-9, atol=1e-11)
    Abar, P, s, _ = MR.block_system(Kx, Mx, a, -beta, beta)
    P32 = sp.block_diag([Kx + (a + abs(beta)) * Mx] * 2)
    assert np.allclose(P.toarray(), abs(beta) * P32.toarray())
    A32 = sp.bmat([[Kx + a * Mx, beta * Mx], [beta * Mx, -(Kx + a * Mx)]])
    assert np.allclose(Abar.toarray(), abs(beta) * A32.toarray())


# --------------------------------------------------------------------------
# Preconditioned MinRes
# --------------------------------------------------------------------------

def _random_indefinite(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([-rng.uniform(0.5, 3.0, n // 2), rng.uniform(0.2, 4.0, n - n // 2)])
    Am = Q @ np.diag(ev) @ Q.T
    Bm = rng.standard_normal((n, n))
    Pm = Bm @ Bm.T + n * np.eye(n)
    return Am, Pm, rng.standard_normal(n)


def test_pminres_residual_estimate_is_exact():
    """|eta_k| equals the true ||b - A x_k||_{P^{-1}} at every iteration."""
    Am, Pm, b = _random_indefinite(40, 1)
    Pinv = np.linalg.inv(Pm)
    seen = []

    def cb(k, x, eta):
        r = b - Am @ x
        seen.append((eta, np.sqrt(r @ Pinv @ r)))

    MR.pminres(Am, lambda v: np.linalg.solve(Pm, v), b, tol=1e-12, maxit=60, callback=cb)
    assert len(seen) > 10
    for eta, true in seen:
        assert eta == pytest.approx(true, rel=1e-6, abs=1e-12 * seen[0][1])


def test_pminres_is_minimal_residual_bruteforce():
    """The k-th iterate minimises ||b - A x||_{P^{-1}} over the Krylov space
    span{P^{-1} b, (P^{-1} A) P^{-1} b, ...}: least squares on an explicit
    basis of that space gives the same residual norms."""
    Am, Pm, b = _random_indefinite(30, 2)
    Lc = np.linalg.cholesky(Pm)  # ||v||_{P^{-1}} = ||L^{-1} v||
    _, _, hist = MR.pminres(Am, lambda v: np.linalg.solve(Pm, v), b, tol=1e-14, maxit=8)
    v = np.linalg.solve(Pm, b)
    basis = []
    for k in range(1, 8):
        basis.append(v)
        Kb, _ = np.linalg.qr(np.column_stack(basis))
        W = np.linalg.solve(Lc, Am @ Kb)
        c, *_ = np.linalg.lstsq(W, np.linalg.solve(Lc, b), rcond=None)
        best = np.linalg.norm(np.linalg.solve(Lc, b) - W @ c)
        assert hist[k] == pytest.approx(best, rel=1e-7)
        v = np.linalg.solve(Pm, Am @ v)
        v = v / np.linalg.norm(v)


def test_pminres_converges_to_dense_solve():
    Am, Pm, b = _random_indefinite(50, 4)
    x, it, hist = MR.pminres(Am, lambda v: np.linalg.solve(Pm, v), b, tol=1e-12, maxit=200)
    assert hist[-1] <= 1e-12 * hist[0]
    assert np.allclose(x, np.linalg.solve(Am, b), rtol=1e-8, atol=1e-10)


def test_pminres_exact_preconditioner_one_step():
    """P = A SPD: one iteration solves the system exactly (beta_2 = 0)."""
    rng = np.random.default_rng(6)
    Bm = rng.standard_normal((20, 20))
    Am = Bm @ Bm.T + 20 * np.eye(20)
    b = rng.standard_normal(20)
    x, it, hist = MR.pminres(Am, lambda v: np.linalg.solve(Am, v), b, tol=1e-14)
    assert it == 1
    assert np.allclose(x, np.linalg.solve(Am, b), rtol=1e-12)


def test_minres_bound_iterations_closed_form():
    # q = (sqrt2 - 1)/(sqrt2 + 1) = 3 - 2 sqrt2; 2 q^7 = 1.0e-5.4... : k for 1e-10 is 28
    assert MR.minres_bound_iterations(1e-10) == 28
    assert MR.minres_bound_iterations(1e-4) == 12
    q = 3 - 2 * np.sqrt(2)
    k = MR.minres_bound_iterations(1e-6)
    assert 2 * q ** (k // 2) <= 1e-6 < 2 * q ** (k // 2 - 1)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_table_3_shape_iterations_bounded(p):
    """Table 3's experiment on the unit square: MinRes iterations for the
    2x2 blocks of the real Schur form and for the complex shifts (Theorem 3.2
    form), theta = 0.1, zero initial guess, reduction 1e-10, under uniform
    refinement in x and t.  The count stays below the two-interval bound for
    cond <= sqrt 2 (28) and levels off under refinement (18-26 here; the
    paper's Table 3 prints 18-27 on its multi-patch domain)."""
    rng = np.random.default_rng(p)
    counts = []
    for ref in range(4):
        nel = 2 * 2 ** ref
        Kt, Mt = A.time_matrices(0.1, nel, p, 0.1 * 0.1 / nel)
        T, X, Y, blocks = MR.real_schur_standard(Kt, Mt)
        Mx, Kx = _space(2, (4 * 2 ** ref, 4 * 2 ** ref), p)
        m = Mx.shape[0]
        its_r, its_c = [], []
        for (b, sz) in blocks:
            if sz != 2:
                continue
            a, b1, b2 = T[b, b], T[b, b + 1], T[b + 1, b]
            f, g = rng.standard_normal(m), rng.standard_normal(m)
            its_r.append(MR.block_solve(Kx, Mx, a, b1, b2, f, g, tol=1e-10)[2])
            w = np.sqrt(abs(b1 * b2))
            its_c.append(MR.block_solve(Kx, Mx, a, -w, w, f, g, tol=1e-10)[2])
        counts.append((max(its_r), max(its_c)))
    bound = MR.minres_bound_iterations(1e-10)
    for r, c in counts:
        assert 4 <= r <= bound and 4 <= c <= bound
    assert abs(counts[-1][0] - counts[-2][0]) <= 2 and abs(counts[-1][1] - counts[-2][1]) <= 2


# --------------------------------------------------------------------------
# Slab solve by Eq. 3.1 + Algorithm 1 with MinRes blocks
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d,spans,p,ne,theta", [(1, (12,), 2, 2, 1.0), (2, (6, 5), 2, 2, 1.0),
                                                (2, (5, 4), 3, 2, 0.1), (2, (4, 4), 1, 4, 0.1)])
def test_slab_solve_minres_matches_lu(d, spans, p, ne, theta):
    prob = A.Problem(d, spans, p, ne, 4, theta=theta)
    _, _, _, _, _, blocks = _schur_blocks(p, ne, theta, tau=prob.tau)
    assert any(m == 2 for _, m in blocks)
    Ab, _ = A.slab_blocks(prob)
    r = np.random.default_rng(9).standard_normal(prob.Nt * prob.Nx)
    exact = spla.spsolve(sp.csc_matrix(Ab), r)
    got, it = MR.slab_solve_minres(prob, r, tol=1e-13)
    assert np.linalg.norm(got - exact) <= 1e-9 * np.linalg.norm(exact)
    assert it >= 2


def test_slab_solve_minres_inexact_error_scales_with_tolerance():
    """At the smoother's inner tolerance the slab inverse is approximate; its
    error shrinks with the tolerance (about linearly)."""
    prob = A.Problem(2, (6, 6), 2, 2, 4, theta=1.0)
    Ab, _ = A.slab_blocks(prob)
    r = np.random.default_rng(10).standard_normal(prob.Nt * prob.Nx)
    exact = spla.spsolve(sp.csc_matrix(Ab), r)
    errs = []
    for tol in (1e-2, 1e-4, 1e-6):
        got, _ = MR.slab_solve_minres(prob, r, tol=tol)
        errs.append(np.linalg.norm(got - exact) / np.linalg.norm(exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] <= 1e-2 and errs[2] <= 1e-4


def test_jacobi_step_minres_tight_tolerance_is_exact_step():
    """With a tight inner tolerance the inexact smoother is the exact damped
    block-Jacobi step of Sec. 3.1 (sparse-LU slab solves)."""
    from oracle import solve as S
    prob = A.Problem(2, (8, 6), 3, 2, 5, theta=1.0)
    L = A.assemble_L(prob)
    lev = S.Level(L, prob.N, prob.Nt * prob.Nx)
    rng = np.random.default_rng(12)
    u0, f = rng.standard_normal(prob.ndofs), rng.standard_normal(prob.ndofs)
    ref = S.jacobi_step(lev, u0, f, 0.5)
    got, it = MR.jacobi_step_minres(prob, u0, f, 0.5, tol=1e-13)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    got4, it4 = MR.jacobi_step_minres(prob, u0, f, 0.5, tol=1e-4)
    err = np.abs(got4 - ref).max() / np.abs(ref).max()
    assert 1e-8 < err < 1e-3
    assert it4 <= MR.minres_bound_iterations(1e-4) < it


@pytest.mark.parametrize("variant", ["eig", "cschur"])
@pytest.mark.parametrize("d,spans,p,ne,theta", [(1, (12,), 2, 2, 1.0), (2, (6, 5), 2, 2, 1.0),
                                                (2, (5, 4), 3, 2, 0.1)])
def test_complex_slab_solve_minres_matches_lu(variant, d, spans, p, ne, theta):
    """Eq. 3.1 with the diagonalisation / complex Schur factors and Theorem
    3.2's MinRes for every complex shift equals the sparse-LU slab solve at a
    tight tolerance; the factors satisfy K_t X = M_t X T, Y M_t X = I."""
    prob = A.Problem(d, spans, p, ne, 4, theta=theta)
    Kt, Mt = A.time_matrices(prob.tau, prob.ne, prob.p, prob.delta)
    T, X, Y = MR.complex_factors(Kt, Mt, variant)
    n = Kt.shape[0]
    assert np.allclose(Kt @ X, Mt @ X @ T, atol=1e-10 * np.abs(Kt).max())
    assert np.allclose(Y @ Mt @ X, np.eye(n), atol=1e-9)
    assert np.allclose(np.tril(T, -1), 0.0)
    if variant == "cschur":
        assert np.allclose(X.conj().T @ X, np.eye(n), atol=1e-12)
    else:
        assert np.allclose(T, np.diag(np.diag(T)))
    assert np.any(np.abs(np.diag(T).imag) > 1e-3)
    Ab, _ = A.slab_blocks(prob)
    r = np.random.default_rng(13).standard_normal(prob.Nt * prob.Nx)
    exact = spla.spsolve(sp.csc_matrix(Ab), r)
    got, it = MR.slab_solve_minres_complex(prob, r, variant, tol=1e-13)
    assert np.linalg.norm(got - exact) <= 1e-9 * np.linalg.norm(exact)
    assert it >= 2
    got4, _ = MR.slab_solve_minres_complex(prob, r, variant, tol=1e-4)
    err = np.linalg.norm(got4 - exact) / np.linalg.norm(exact)
    assert 1e-9 < err < 1e-2

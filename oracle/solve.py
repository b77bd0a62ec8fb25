"""Oracle solvers for L_h u = f (Sec. 3.1 of arXiv:1802.09277).

Test infrastructure only (see ``oracle/__init__.py``).

* ``direct``           -- sparse LU of the whole L_h (the exact solution).
* ``forward_subst``    -- exact block forward substitution: L_h is block
  lower bidiagonal, so u_n = A_n^{-1} (f_n + B_n u_{n-1}).
* ``jacobi_step``      -- one damped block-Jacobi step
  u <- u + omega D^{-1} (f - L u), D = blockdiag(A_n), slab solves by LU.
* ``time_prolongation``-- P_t: a coarse slab (two fine slabs merged, same
  number of elements) expressed in the two fine slabs' bases.  The coarse
  spline space is nested in the broken fine space, so the L2 projection onto
  each fine slab reproduces it exactly.
* ``space_prolongation_1d``, ``space_prolongation`` -- P_x: the coarse
  spatial B-splines (spans halved) in the fine basis (knot insertion).
* ``Hierarchy``        -- levels with Galerkin coarse operators P^T L P,
  coarsening in time (slab pairs) or, above a parabolic ratio tau / h^2, in
  space.
* ``vcycle``, ``mg_solve``, ``fgmres`` -- the V-cycle, the plain multigrid
  iteration and right-preconditioned flexible GMRES.

The multigrid details are not in this paper (it defers them to the
Gander-Neumueller reference); the reading adopted: time-only coarsening by
slab pairs, restriction R = P^T, Galerkin coarse operators, nu1 = nu2 = 1
damped block-Jacobi steps with omega = 1/2, exact solve on the coarsest
level.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble, bspline


def direct(L, f):
    """Exact solution of L u = f by sparse LU (SuperLU)."""
    return spla.splu(sp.csc_matrix(L)).solve(np.asarray(f, dtype=float))


def forward_subst(prob, f):
    """Exact solve by block forward substitution over the slabs."""
    A, B = assemble.slab_blocks(prob)
    lu = spla.splu(sp.csc_matrix(A))
    m = prob.Nt * prob.Nx
    f = np.asarray(f, dtype=float).reshape(prob.N, m)
    u = np.zeros_like(f)
    for n in range(prob.N):
        rhs = f[n] + (B @ u[n - 1] if n > 0 else 0.0)
        u[n] = lu.solve(rhs)
    return u.reshape(-1)


class Level:
    """One multigrid level: its system matrix and the LU of every diagonal
    block (all equal on the finest level, but taken from L itself so that
    Galerkin coarse levels are handled the same way)."""

    def __init__(self, L, nslabs, m):
        self.L = sp.csr_matrix(L)
        self.N = nslabs
        self.m = m  # unknowns per slab
        self.lu = []
        for n in range(nslabs):
            blk = self.L[n * m:(n + 1) * m, n * m:(n + 1) * m]
            self.lu.append(spla.splu(sp.csc_matrix(blk)))

    def block_solve(self, r):
        r = r.reshape(self.N, self.m)
        return np.stack([self.lu[n].solve(r[n]) for n in range(self.N)]).reshape(-1)


def jacobi_step(level, u, f, omega=0.5):
    """u + omega * D^{-1} (f - L u)  (the smoother of Sec. 3.1)."""
    r = f - level.L @ u
    return u + omega * level.block_solve(r)


def time_prolongation(tau, ne, p):
    """P_t of shape (2 Nt, Nt): coarse slab [0, 2 tau] with ne elements of
    length 2 tau/ne, fine slabs [0, tau] and [tau, 2 tau] with ne elements
    each.  Rows: first fine slab's coefficients, then the second's."""
    kc = bspline.open_knots(0.0, 2 * tau, ne, p)
    blocks = []
    for q in range(2):
        kf = bspline.open_knots(q * tau, (q + 1) * tau, ne, p)
        x, w = bspline.element_quadrature(kf, p + 2)
        Bf = bspline.basis(kf, p, x)
        Bc = bspline.basis(kc, p, x)
        Mff = Bf.T @ (w[:, None] * Bf)
        Mfc = Bf.T @ (w[:, None] * Bc)
        blocks.append(np.linalg.solve(Mff, Mfc))
    return np.vstack(blocks)


def prolongation(prob):
    """P = blockdiag over coarse slabs of (P_t (x) I_x): maps a level with
    N/2 slabs to the level with N slabs (prob is the fine level)."""
    Pt = time_prolongation(prob.tau, prob.ne, prob.p)
    blk = sp.kron(sp.csr_matrix(Pt), sp.identity(prob.Nx, format="csr"))
    return sp.block_diag([blk] * (prob.N // 2), format="csr")


def space_prolongation_1d(s, p):
    """P_x of shape (n_f, n_c): the interior B-splines of s/2 spans on (0,1)
    expressed in the interior B-splines of s spans.  The coarse space is
    nested in the fine one (the fine knots are the coarse knots plus the
    midpoints), so the L2 projection with the fine mass matrix reproduces it
    exactly; the fine quadrature integrates the products exactly."""
    assert s % 2 == 0
    kf = bspline.open_knots(0.0, 1.0, s, p)
    kc = bspline.open_knots(0.0, 1.0, s // 2, p)
    x, w = bspline.element_quadrature(kf, p + 2)
    Bf = bspline.basis(kf, p, x)[:, 1:-1]
    Bc = bspline.basis(kc, p, x)[:, 1:-1]
    Mff = Bf.T @ (w[:, None] * Bf)
    Mfc = Bf.T @ (w[:, None] * Bc)
    return np.linalg.solve(Mff, Mfc)


def space_prolongation(prob):
    """P = I_{N N_t} (x) P_z (x) P_y (x) P_x: maps the level with every
    axis' spans halved (same slabs) to prob's level (space coarsening)."""
    mats = [space_prolongation_1d(s, prob.p) for s in prob.spans]
    Px = assemble._kron_all(mats)
    return sp.kron(sp.identity(prob.N * prob.Nt, format="csr"), Px, format="csr")


def space_time_ratio(prob):
    """tau / h_x^2 with h_x the largest spatial element size (the parabolic
    ratio that decides between coarsening in time and in space)."""
    return prob.tau * min(prob.spans) ** 2


class Hierarchy:
    """Levels 0 (finest) .. J with Galerkin operators.  Each coarsening step
    merges slab pairs (time), or -- when space_ratio > 0 and the level's
    tau / h_x^2 exceeds it (diffusion-dominated slabs) -- halves every spatial
    axis' spans (space; Sec. 3.1's multigrid coarsens in space and time, the
    rule is not given in the paper; the coarse level keeps at least min_spans
    spans per axis); it stops at one slab or when neither applies.  kinds[l]
    is "t" or "x" for the step from level l to l + 1."""

    def __init__(self, prob, min_slabs=1, space_ratio=0.0, min_spans=2):
        self.probs = [prob]
        self.levels = []
        self.P = []
        self.kinds = []
        L = assemble.assemble_L(prob)
        while True:
            pr = self.probs[-1]
            self.levels.append(Level(L, pr.N, pr.Nt * pr.Nx))
            space_ok = all(s % 2 == 0 and s // 2 >= min_spans for s in pr.spans)
            if space_ratio > 0 and space_time_ratio(pr) > space_ratio and space_ok:
                P = space_prolongation(pr)
                nxt = pr.space_coarse()
                self.kinds.append("x")
            elif pr.N > min_slabs and pr.N % 2 == 0:
                P = prolongation(pr)
                nxt = pr.coarse()
                self.kinds.append("t")
            else:
                break
            self.P.append(P)
            L = (P.T @ L @ P).tocsr()
            self.probs.append(nxt)
        self.coarse_lu = spla.splu(sp.csc_matrix(self.levels[-1].L))


def vcycle(H, f, lvl=0, nu1=1, nu2=1, omega=0.5, u=None):
    """One V-cycle for L_lvl u = f starting from u (zero if None)."""
    level = H.levels[lvl]
    if u is None:
        u = np.zeros_like(f)
    if lvl == len(H.levels) - 1:
        return H.coarse_lu.solve(f)
    for _ in range(nu1):
        u = jacobi_step(level, u, f, omega)
    r = f - level.L @ u
    P = H.P[lvl]
    ec = vcycle(H, P.T @ r, lvl + 1, nu1, nu2, omega)
    u = u + P @ ec
    for _ in range(nu2):
        u = jacobi_step(level, u, f, omega)
    return u


def mg_solve(H, f, tol=1e-8, maxit=200, **kw):
    """Multigrid iteration u <- u + V(f - L u) from u = 0 until
    ||f - L u||_2 <= tol ||f||_2.  Returns (u, iterations, history)."""
    L = H.levels[0].L
    u = np.zeros_like(f)
    nf = np.linalg.norm(f)
    hist = [1.0]
    for it in range(1, maxit + 1):
        u = vcycle(H, f, u=u, **kw)
        rel = np.linalg.norm(f - L @ u) / nf
        hist.append(rel)
        if rel <= tol:
            return u, it, hist
    return u, maxit, hist


def fgmres(L, f, precond, tol=1e-8, restart=30, maxit=300):
    """Right-preconditioned flexible GMRES (modified Gram-Schmidt, Givens
    rotations), zero initial guess, stop at ||f - L u||_2 <= tol ||f||_2.
    Returns (u, iterations, history)."""
    n = f.shape[0]
    u = np.zeros(n)
    nf = np.linalg.norm(f)
    hist = [1.0]
    total = 0
    while total < maxit:
        r = f - L @ u
        beta = np.linalg.norm(r)
        if beta <= tol * nf:
            break
        V = [r / beta]
        Z = []
        Hm = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k = 0
        for j in range(restart):
            z = precond(V[j])
            Z.append(z)
            w = L @ z
            for i in range(j + 1):
                Hm[i, j] = np.dot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hm[j + 1, j] if Hm[j + 1, j] > 0 else w)
            for i in range(j):
                a, b = Hm[i, j], Hm[i + 1, j]
                Hm[i, j] = cs[i] * a + sn[i] * b
                Hm[i + 1, j] = -sn[i] * a + cs[i] * b
            a, b = Hm[j, j], Hm[j + 1, j]
            rad = np.hypot(a, b)
            cs[j], sn[j] = a / rad, b / rad
            Hm[j, j] = rad
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            total += 1
            hist.append(abs(g[j + 1]) / nf)
            if abs(g[j + 1]) <= tol * nf or total >= maxit:
                break
        y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
        for i in range(k):
            u = u + y[i] * Z[i]
        if np.linalg.norm(f - L @ u) <= tol * nf:
            break
    return u, total, hist

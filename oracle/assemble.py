"""Oracle assembly of the space-time dG-IgA system (Sec. 2.2-2.3 of
arXiv:1802.09277).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper adopted here (each also listed in the design notes):

* ``h_n`` in the SUPG weight ``theta_n h_n`` is the length of one time
  element inside slab n (this reproduces Table 2).
* On coarse multigrid levels the product ``delta = theta * h`` stays at its
  finest-level value (this is what the Galerkin coarse operator gives).
* The spatial domain is the unit interval / square / cube with homogeneous
  Dirichlet data: the first and last B-spline of every axis are removed.
* Every slab has the same number ``ne`` of time elements and all slabs have
  the same length, so all diagonal blocks A_n are equal.

Vector layout: u[slab][t][z][y][x] (time outer, space inner, x fastest),
matching the Kronecker order ``K_t (x) M_x`` of Eq. 2.5.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import bspline


@dataclass
class Problem:
    """Uniform space-time problem on (0,1)^d x (0,T).

    d: space dimension; spans: knot spans per axis (x, y, z order);
    p: degree in space and time; ne: time elements per slab; N: slabs;
    theta: SUPG parameter; T: final time.
    """
    d: int
    spans: tuple
    p: int
    ne: int
    N: int
    theta: float = 1.0
    T: float = 1.0
    delta: float = field(default=None)  # SUPG weight theta*h, frozen if given

    def __post_init__(self):
        self.spans = tuple(int(s) for s in self.spans)
        assert len(self.spans) == self.d
        if self.delta is None:
            self.delta = self.theta * self.h

    @property
    def tau(self):
        """Slab length t_n - t_{n-1}."""
        return self.T / self.N

    @property
    def h(self):
        """Time element length (the reading of h_n)."""
        return self.tau / self.ne

    @property
    def n_axis(self):
        """Interior spatial dofs per axis (x first)."""
        return tuple(s + self.p - 2 for s in self.spans)

    @property
    def Nx(self):
        return int(np.prod(self.n_axis))

    @property
    def Nt(self):
        return self.ne + self.p

    @property
    def ndofs(self):
        return self.N * self.Nt * self.Nx

    def coarse(self):
        """The next coarser level: slab pairs merged, same ne, delta frozen."""
        assert self.N % 2 == 0
        return Problem(self.d, self.spans, self.p, self.ne, self.N // 2,
                       self.theta, self.T, self.delta)

    def space_coarse(self):
        """The next coarser level in space: every axis' spans halved, the
        same slabs and time discretisation."""
        assert all(s % 2 == 0 for s in self.spans)
        return Problem(self.d, tuple(s // 2 for s in self.spans), self.p, self.ne, self.N,
                       self.theta, self.T, self.delta)


# ----------------------------------------------------------------------------
# 1D matrices
# ----------------------------------------------------------------------------

def space_matrices(s, p):
    """Mass M1[i,j] = int phi_j phi_i and stiffness K1[i,j] = int phi_j' phi_i'
    on (0,1) (the 1D factors of M_x, K_x after Eq. 2.5), Dirichlet functions
    removed.  Dense arrays of size (s+p-2)^2."""
    kn = bspline.open_knots(0.0, 1.0, s, p)
    x, w = bspline.element_quadrature(kn, p + 2)
    B = bspline.basis(kn, p, x)[:, 1:-1]
    D = bspline.basis_deriv(kn, p, x)[:, 1:-1]
    M1 = B.T @ (w[:, None] * B)
    K1 = D.T @ (w[:, None] * D)
    return M1, K1


def time_matrices(tau, ne, p, delta):
    """K_t and M_t of Eq. 2.6 on one slab [0, tau] with ne elements:

        K_t[i,j] = int psi_j' (psi_i + delta psi_i') dt + psi_j(0) psi_i(0)
        M_t[i,j] = int psi_j  (psi_i + delta psi_i') dt

    where delta = theta_n h_n.  Row index i is the test function."""
    kn = bspline.open_knots(0.0, tau, ne, p)
    t, w = bspline.element_quadrature(kn, p + 2)
    B = bspline.basis(kn, p, t)
    D = bspline.basis_deriv(kn, p, t)
    W = B + delta * D                    # test functions, one column each
    Kt = W.T @ (w[:, None] * D)
    Mt = W.T @ (w[:, None] * B)
    b0 = bspline.basis(kn, p, [0.0])[0]
    Kt += np.outer(b0, b0)
    return Kt, Mt


def coupling_matrix(tau, ne, p):
    """N_t[i,k] = psi_k^{n-1}(t_{n-1}) psi_i^n(t_{n-1}) (after Eq. 2.6): the
    previous slab's basis at its end times this slab's basis at its start."""
    kn = bspline.open_knots(0.0, tau, ne, p)
    start = bspline.basis(kn, p, [0.0])[0]
    end = bspline.basis(kn, p, [tau])[0]
    return np.outer(start, end)


def _kron_all(mats):
    """mats in x, y, z order -> kron(z, y, x) (x fastest)."""
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(sp.csr_matrix(m), out, format="csr")
    return out


def spatial_operators(prob):
    """M_x = tensor product of M1, K_x = sum over axes of K1 in one slot
    (the Laplacian stiffness of the tensor-product basis)."""
    facs = [space_matrices(s, prob.p) for s in prob.spans]
    Mx = _kron_all([f[0] for f in facs])
    Kx = None
    for a in range(prob.d):
        mats = [facs[b][1] if b == a else facs[b][0] for b in range(prob.d)]
        term = _kron_all(mats)
        Kx = term if Kx is None else Kx + term
    return Mx.tocsr(), Kx.tocsr()


def slab_blocks(prob):
    """A_n = K_t (x) M_x + M_t (x) K_x (Eq. 2.5), B_n = N_t (x) M_x."""
    Mx, Kx = spatial_operators(prob)
    Kt, Mt = time_matrices(prob.tau, prob.ne, prob.p, prob.delta)
    Nt = coupling_matrix(prob.tau, prob.ne, prob.p)
    A = (sp.kron(sp.csr_matrix(Kt), Mx) + sp.kron(sp.csr_matrix(Mt), Kx)).tocsr()
    B = sp.kron(sp.csr_matrix(Nt), Mx).tocsr()
    return A, B


def _apply_axis(mat, v, axis):
    """Apply a dense 1D matrix along one axis of v (shape (N_t, n_z, n_y, n_x)
    trimmed to the problem's dimension; spatial axis 0 is x, the last)."""
    ax = v.ndim - 1 - axis
    return np.moveaxis(np.tensordot(mat, v, axes=([1], [ax])), 0, ax)


def slab_residual_kron(prob, f_n, u_n, u_prev, magnitude=False):
    """One block row of Eq. 2.4 without assembling it: the slab residual
    r_n = f_n - (K_t (x) M_x + M_t (x) K_x) u_n + (N_t (x) M_x) u_{n-1}
    (Eq. 2.5), each Kronecker factor applied along its own axis, M_x as the
    product of the 1D mass matrices and K_x as the sum over axes of the 1D
    stiffness in one slot.  u_prev = None for the first slab (no coupling).

    With magnitude=True every factor and vector is replaced by its entry-wise
    absolute value and the three terms are added: the size of the terms the
    residual sums, |f_n| + (|K_t| (x) |M_x| + |M_t| (x) |K_x|) |u_n| +
    (|N_t| (x) |M_x|) |u_{n-1}|, the scale of a rounding-error bound."""
    facs = [space_matrices(s, prob.p) for s in prob.spans]
    Kt, Mt = time_matrices(prob.tau, prob.ne, prob.p, prob.delta)
    Nt = coupling_matrix(prob.tau, prob.ne, prob.p)
    ab = np.abs if magnitude else (lambda a: a)
    shape = (prob.Nt,) + tuple(reversed(prob.n_axis))

    def mass(v):
        for a in range(prob.d):
            v = _apply_axis(ab(facs[a][0]), v, a)
        return v

    def stiff(v):
        out = 0.0
        for a in range(prob.d):
            w = v
            for b in range(prob.d):
                w = _apply_axis(ab(facs[b][1] if b == a else facs[b][0]), w, b)
            out = out + w
        return out

    def time(mat, v):
        return np.tensordot(ab(mat), v, axes=([1], [0]))

    u = ab(np.asarray(u_n, dtype=np.float64).reshape(shape))
    Lu = time(Kt, mass(u)) + time(Mt, stiff(u))
    f = ab(np.asarray(f_n, dtype=np.float64).reshape(shape))
    if magnitude:
        r = f + Lu
    else:
        r = f - Lu
    if u_prev is not None:
        c = time(Nt, mass(ab(np.asarray(u_prev, dtype=np.float64).reshape(shape))))
        r = r + c
    return r.reshape(-1)


def assemble_L(prob):
    """The block lower-bidiagonal system matrix of Eq. 2.4: A on the
    diagonal, -B on the first sub-diagonal."""
    A, B = slab_blocks(prob)
    N = prob.N
    blocks = [[None] * N for _ in range(N)]
    for n in range(N):
        blocks[n][n] = A
        if n > 0:
            blocks[n][n - 1] = -B
    return sp.bmat(blocks, format="csr")


# ----------------------------------------------------------------------------
# Load vectors  f_n[i] = l_h(phi_i^n)  (Sec. 2.3), u0 = 0
# ----------------------------------------------------------------------------

def load_from_coeffs(prob, c):
    """f = sum_j c_j phi_j over the interior trial basis of every slab.  Then
    l_h(phi_i) = int f (phi_i + delta d_t phi_i) = ((M_t (x) M_x) c)_i
    exactly.  c: [N, Nt, Nx] (or flat)."""
    Mx, _ = spatial_operators(prob)
    _, Mt = time_matrices(prob.tau, prob.ne, prob.p, prob.delta)
    S = sp.kron(sp.csr_matrix(Mt), Mx).tocsr()
    c = np.asarray(c, dtype=float).reshape(prob.N, prob.Nt * prob.Nx)
    return np.stack([S @ c[n] for n in range(prob.N)]).reshape(-1)


def _space_load_1d(s, p, func, npts):
    """g[i] = int_0^1 func(x) phi_i(x) dx over the interior basis."""
    kn = bspline.open_knots(0.0, 1.0, s, p)
    x, w = bspline.element_quadrature(kn, npts)
    B = bspline.basis(kn, p, x)[:, 1:-1]
    return B.T @ (w * func(x))


def _time_load(prob, n, func, npts):
    """g[a] = int_{t_{n-1}}^{t_n} func(t) (psi_a + delta psi_a') dt."""
    t0 = n * prob.tau
    kn = bspline.open_knots(t0, t0 + prob.tau, prob.ne, prob.p)
    t, w = bspline.element_quadrature(kn, npts)
    W = bspline.basis(kn, prob.p, t) + prob.delta * bspline.basis_deriv(kn, prob.p, t)
    return W.T @ (w * func(t))


def _separable_load(prob, space_funcs, time_func, npts, slabs=None):
    """Load vector of f(x,t) = prod_a space_funcs[a](x_a) * time_func(t),
    on the slabs listed in `slabs` (all slabs if None), in that order."""
    gx = None
    for a in range(prob.d):
        g = _space_load_1d(prob.spans[a], prob.p, space_funcs[a], npts)
        gx = g if gx is None else np.kron(g, gx)
    slabs = range(prob.N) if slabs is None else list(slabs)
    out = np.zeros((len(slabs), prob.Nt, prob.Nx))
    for i, n in enumerate(slabs):
        out[i] = np.outer(_time_load(prob, n, time_func, npts), gx)
    return out.reshape(-1)


def manufactured_load(prob):
    """Load vector for u = prod_a sin(pi x_a) * sin(pi t), i.e. the source
    f = prod sin(pi x_a) * (pi cos(pi t) + d pi^2 sin(pi t)), u0 = 0,
    quadrature with 2p+4 points per element."""
    d = prob.d
    sx = [lambda x: np.sin(np.pi * x)] * d
    ft = lambda t: np.pi * np.cos(np.pi * t) + d * np.pi ** 2 * np.sin(np.pi * t)
    return _separable_load(prob, sx, ft, 2 * prob.p + 4)


def bumps_load(prob, centers, widths, amps, npts=None, slabs=None):
    """Load vector of f(x,t) = sum_k a_k exp(-|(x,t) - c_k|^2 / (2 w_k^2)),
    space-time Gaussian bumps (centers [K, d+1] in (x, y, z, t) order),
    Gauss-Legendre quadrature with npts (default 2p+4) points per element;
    only the slabs listed in `slabs` (all if None), in that order."""
    npts = 2 * prob.p + 4 if npts is None else npts
    ns = prob.N if slabs is None else len(list(slabs))
    out = np.zeros(ns * prob.Nt * prob.Nx)
    for c, wk, a in zip(centers, widths, amps):
        sfun = [(lambda x, cc=c[i], ww=wk: np.exp(-(x - cc) ** 2 / (2 * ww * ww)))
                for i in range(prob.d)]
        tfun = lambda t, cc=c[prob.d], ww=wk: a * np.exp(-(t - cc) ** 2 / (2 * ww * ww))
        out += _separable_load(prob, sfun, tfun, npts, slabs)
    return out


# ----------------------------------------------------------------------------
# dG norm of the error for the manufactured solution (after Eq. 2.3)
# ----------------------------------------------------------------------------

def dg_error_manufactured(prob, uh):
    """||u - u_h||_dG for u = prod sin(pi x_a) sin(pi t), d = 1 or 2, by
    tensor Gauss quadrature with p+3 points per element:

      sum_n ( ||grad_x e||^2_{Q_n} + delta ||d_t e||^2_{Q_n}
              + 1/2 ||[[e]]^{n-1}||^2 ) + 1/2 ||e(T)||^2,

    with [[e]]^0 = e(0^+) (u0 = 0) and, u being continuous,
    [[e]]^{n-1} = -(u_h(t_{n-1}^+) - u_h(t_{n-1}^-)) for n > 1."""
    d, p = prob.d, prob.p
    assert d in (1, 2)
    q = p + 3
    ax = []
    for a in range(d):
        kn = bspline.open_knots(0.0, 1.0, prob.spans[a], p)
        x, w = bspline.element_quadrature(kn, q)
        ax.append((x, w, bspline.basis(kn, p, x)[:, 1:-1],
                   bspline.basis_deriv(kn, p, x)[:, 1:-1]))
    U = uh.reshape(prob.N, prob.Nt, *reversed(prob.n_axis))
    sx = [np.sin(np.pi * a[0]) for a in ax]
    cx = [np.pi * np.cos(np.pi * a[0]) for a in ax]

    if d == 1:
        wsp = ax[0][1]
        def ev(Tt, coef, dx):            # -> [t, x]
            Bx = ax[0][3] if dx[0] else ax[0][2]
            return np.einsum('ta,ai,xi->tx', Tt, coef, Bx)
        def ex_space(dx):
            return cx[0] if dx[0] else sx[0]
    else:
        wsp = np.outer(ax[1][1], ax[0][1])   # [y, x]
        def ev(Tt, coef, dx):            # -> [t, y, x]
            Bx = ax[0][3] if dx[0] else ax[0][2]
            By = ax[1][3] if dx[1] else ax[1][2]
            return np.einsum('ta,aji,yj,xi->tyx', Tt, coef, By, Bx)
        def ex_space(dx):
            fx = cx[0] if dx[0] else sx[0]
            fy = cx[1] if dx[1] else sx[1]
            return np.outer(fy, fx)

    def integ(vals_t_space, wt):
        wt_b = wt.reshape((-1,) + (1,) * d)
        return float(np.sum(wt_b * vals_t_space * wsp))

    total = 0.0
    prev_end = None
    for n in range(prob.N):
        t0 = n * prob.tau
        kn = bspline.open_knots(t0, t0 + prob.tau, prob.ne, p)
        t, wt = bspline.element_quadrature(kn, q)
        Bt = bspline.basis(kn, p, t)
        Dt = bspline.basis_deriv(kn, p, t)
        coef = U[n]
        for a in range(d):
            dx = [b == a for b in range(d)]
            e = np.multiply.outer(np.sin(np.pi * t), ex_space(dx)) - ev(Bt, coef, dx)
            total += integ(e ** 2, wt)
        dx0 = [False] * d
        e = np.multiply.outer(np.pi * np.cos(np.pi * t), ex_space(dx0)) - ev(Dt, coef, dx0)
        total += prob.delta * integ(e ** 2, wt)
        b0 = bspline.basis(kn, p, [t0])
        b1 = bspline.basis(kn, p, [t0 + prob.tau])
        start = ev(b0, coef, dx0)[0]
        end = ev(b1, coef, dx0)[0]
        if n == 0:
            jump = start - np.sin(0.0) * ex_space(dx0)
        else:
            jump = start - prev_end
        total += 0.5 * float(np.sum(jump ** 2 * wsp))
        prev_end = end
    eT = np.sin(np.pi * prob.T) * ex_space([False] * d) - prev_end
    total += 0.5 * float(np.sum(eT ** 2 * wsp))
    return float(np.sqrt(total))

"""Oracle for the inexact spatial solves of Sec. 3.3-3.5 of arXiv:1802.09277.

Test infrastructure only (see ``oracle/__init__.py``).

The slab inverse of Eq. 3.1 needs, for every diagonal block of the (real)
Schur form of M_t^{-1} K_t, a spatial solve.  For a 2x2 block
[[alpha, beta1], [beta2, alpha]] (complex pair alpha +- i sqrt|beta1 beta2|)
the spatial system is

    [[K_x + alpha M_x, beta1 M_x], [beta2 M_x, K_x + alpha M_x]] [x; y] = [f; g].

Sec. 3.5 rescales it to a symmetric indefinite matrix Abar acting on
[x; -y] and Theorem 3.3 gives a block-diagonal preconditioner P with
cond(P^{-1} Abar) <= sqrt 2; Theorem 3.2 (a complex shift alpha + i beta,
Sec. 3.3/3.4) is the special case beta1 = -beta, beta2 = beta up to the
common factor |beta|.  The systems are solved by MinRes preconditioned by P.

* ``standardize_2x2``      -- the rotation of Sec. 3.5 that gives a 2x2 block
  equal diagonal entries.
* ``real_schur_standard``  -- real Schur form of M_t^{-1} K_t with standardised
  2x2 blocks, and the factors X = Q, Y = (M_t X)^{-1} of Eq. 3.1.
* ``block_system``         -- Abar, P and the right-hand-side scaling of
  Theorem 3.3.
* ``pminres``              -- textbook preconditioned MinRes (Lanczos in the
  inner product of P^{-1}, QR of the tridiagonal matrix by Givens rotations).
* ``block_solve``          -- one 2x2 block system by ``pminres``.
* ``slab_solve_minres``    -- A_n^{-1} r by Eq. 3.1: time transform Y, the
  block back substitution of Algorithm 1 over the real Schur form (each
  block's spatial system by MinRes, the 1x1 blocks, which are SPD with P
  equal to the matrix itself, by one solve with P), time transform X.
* ``complex_factors``, ``slab_solve_minres_complex`` -- the same with the
  diagonalisation (Sec. 3.3) or the complex Schur form (Sec. 3.4): complex
  time transforms, complex shifts solved in Theorem 3.2's form.
* ``jacobi_step_minres``   -- the damped block-Jacobi step with these slab
  solves.

P is applied here by a sparse LU of K_x + s M_x; the tolerance is a reduction
of the P^{-1}-norm of the residual, the quantity MinRes minimises.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble


def standardize_2x2(B):
    """Rotation G = [[c, -s], [s, c]] such that G^T B G has equal diagonal
    entries (Sec. 3.5).  With B = [[a, b], [c, d]] the difference of the two
    diagonal entries of G^T B G is cos(2t) (a - d) + sin(2t) (b + c), which
    vanishes for 2t = atan2(d - a, b + c)."""
    a, b = B[0, 0], B[0, 1]
    c, d = B[1, 0], B[1, 1]
    t = 0.5 * np.arctan2(d - a, b + c)
    cs, sn = np.cos(t), np.sin(t)
    return np.array([[cs, -sn], [sn, cs]])


def real_schur_standard(Kt, Mt):
    """Q^T (M_t^{-1} K_t) Q = T, Q orthogonal, T upper quasi-triangular with
    every 2x2 block of the form [[alpha, beta1], [beta2, alpha]].  Returns
    (T, X, Y, blocks) with X = Q, Y = (M_t X)^{-1} (Eq. 3.1) and blocks the
    list of (first row, size) of the diagonal blocks."""
    A = np.linalg.solve(Mt, Kt)
    T, Q = sla.schur(A, output="real")
    n = A.shape[0]
    blocks = []
    i = 0
    while i < n:
        if i + 1 < n and T[i + 1, i] != 0.0:
            G = np.eye(n)
            G[i:i + 2, i:i + 2] = standardize_2x2(T[i:i + 2, i:i + 2])
            T = G.T @ T @ G
            Q = Q @ G
            blocks.append((i, 2))
            i += 2
        else:
            blocks.append((i, 1))
            i += 1
    # zero what lies below the diagonal blocks (rounding of the rotations)
    for (b, m) in blocks:
        T[b + m:, b:b + m] = 0.0
    X = Q
    Y = np.linalg.inv(Mt @ X)
    return T, X, Y, blocks


def block_system(Kx, Mx, alpha, beta1, beta2):
    """Theorem 3.3.  With Kc = K_x + alpha M_x:

        Abar = [[|beta2| Kc, -beta1 |beta2| M_x], [|beta1| beta2 M_x, -|beta1| Kc]]
        P    = diag(|beta2| (K_x + s M_x), |beta1| (K_x + s M_x)),  s = alpha + sqrt|beta1 beta2|

    and [[Kc, beta1 M_x], [beta2 M_x, Kc]] [x; y] = [f; g] is equivalent to
    Abar [x; -y] = [|beta2| f; |beta1| g].  Returns (Abar, P, s, (|beta2|, |beta1|))."""
    Kx = sp.csr_matrix(Kx)
    Mx = sp.csr_matrix(Mx)
    Kc = Kx + alpha * Mx
    a1, a2 = abs(beta2), abs(beta1)
    Abar = sp.bmat([[a1 * Kc, -beta1 * a1 * Mx],
                    [a2 * beta2 * Mx, -a2 * Kc]], format="csr")
    s = alpha + np.sqrt(abs(beta1 * beta2))
    Ps = Kx + s * Mx
    P = sp.bmat([[a1 * Ps, None], [None, a2 * Ps]], format="csr")
    return Abar, P, s, (a1, a2)


def pminres(A, Psolve, b, tol=1e-10, maxit=500, x0=None, callback=None):
    """MinRes for the symmetric matrix A preconditioned by the SPD matrix P
    (Psolve(v) = P^{-1} v).  Zero initial guess unless x0 is given; stops when
    ||r_k||_{P^{-1}} <= tol ||r_0||_{P^{-1}}.

    Lanczos in the P^{-1} inner product: q_1 = r_0 / beta_1, p_j = P^{-1} q_j,
    A p_j = beta_j q_{j-1} + alpha_j q_j + beta_{j+1} q_{j+1}.  The iterate
    minimises ||beta_1 e_1 - T_{k+1,k} y||_2 = ||r_k||_{P^{-1}} over
    x_0 + span(p_1..p_k); T_{k+1,k} is reduced by Givens rotations and the
    search directions d_k = (p_k - delta_k d_{k-1} - eps_k d_{k-2}) / rho_k
    hold the columns of P_k R_k^{-1}.

    callback(k, x_k, |eta_k|) is called after every iteration (|eta_k| is the
    recurrence's value of ||r_k||_{P^{-1}}).

    Returns (x, iterations, history of ||r_k||_{P^{-1}} for k = 0..iterations)."""
    b = np.asarray(b, dtype=float)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    r = b - A @ x
    z = Psolve(r)
    beta = np.sqrt(max(float(r @ z), 0.0))
    hist = [beta]
    if beta == 0.0:
        return x, 0, hist
    beta1 = beta
    q_prev = np.zeros(n)
    q = r / beta
    p = z / beta
    d1 = np.zeros(n)       # d_{k-1}
    d2 = np.zeros(n)       # d_{k-2}
    c1, s1 = 1.0, 0.0      # rotation k-1
    c2, s2 = 1.0, 0.0      # rotation k-2
    eta = beta1
    beta_k = 0.0           # beta_k (beta_1 q_0 = 0)
    k = 0
    while k < maxit:
        k += 1
        t = A @ p
        alpha = float(p @ t)
        qh = t - alpha * q - beta_k * q_prev
        zh = Psolve(qh)
        beta_next = np.sqrt(max(float(qh @ zh), 0.0))
        # new column of T_{k+1,k}: (beta_k, alpha_k, beta_{k+1}) in rows k-1..k+1
        eps = s2 * beta_k
        dbar = c2 * beta_k
        delta = c1 * dbar + s1 * alpha
        gbar = -s1 * dbar + c1 * alpha
        rho = np.hypot(gbar, beta_next)
        c, s = gbar / rho, beta_next / rho
        d = (p - delta * d1 - eps * d2) / rho
        x = x + c * eta * d
        eta = -s * eta
        hist.append(abs(eta))
        if callback is not None:
            callback(k, x, abs(eta))
        if abs(eta) <= tol * beta1 or beta_next == 0.0:
            break
        d2, d1 = d1, d
        c2, s2, c1, s1 = c1, s1, c, s
        q_prev, q = q, qh / beta_next
        p = zh / beta_next
        beta_k = beta_next
    return x, k, hist


def block_solve(Kx, Mx, alpha, beta1, beta2, f, g, tol=1e-10, maxit=500):
    """[[K_x + alpha M_x, beta1 M_x], [beta2 M_x, K_x + alpha M_x]] [x; y] = [f; g]
    by MinRes on Theorem 3.3's symmetric form.  Returns (x, y, iterations)."""
    Abar, P, s, (a1, a2) = block_system(Kx, Mx, alpha, beta1, beta2)
    lu = spla.splu(sp.csc_matrix(sp.csr_matrix(Kx) + s * sp.csr_matrix(Mx)))
    m = np.asarray(f).size

    def Psolve(v):
        return np.concatenate([lu.solve(v[:m]) / a1, lu.solve(v[m:]) / a2])

    rhs = np.concatenate([a1 * np.asarray(f, float), a2 * np.asarray(g, float)])
    w, it, _ = pminres(Abar, Psolve, rhs, tol=tol, maxit=maxit)
    return w[:m], -w[m:], it


def slab_solve_minres(prob, r, tol=1e-4, maxit=500):
    """A_n^{-1} r for one slab vector r (length Nt * Nx) by Eq. 3.1 with the
    standardised real Schur form: w = (Y (x) I) r, then Algorithm 1 from the
    last diagonal block to the first on (T (x) M_x + I (x) K_x) z = w:

        g_B = w_B - sum_{j beyond block B} T_{B j} M_x z_j,

    a 1x1 block solved exactly (K_x + T_ii M_x is its own preconditioner),
    a 2x2 block by ``block_solve`` to the relative tolerance tol; finally
    (X (x) I) z.  Returns (A_n^{-1} r approximately, max MinRes iterations)."""
    Mx, Kx = assemble.spatial_operators(prob)
    Kt, Mt = assemble.time_matrices(prob.tau, prob.ne, prob.p, prob.delta)
    T, X, Y, blocks = real_schur_standard(Kt, Mt)
    nt, m = prob.Nt, prob.Nx
    w = (Y @ np.asarray(r, float).reshape(nt, m))
    z = np.zeros((nt, m))
    itmax = 0
    for (b, size) in reversed(blocks):
        g = w[b:b + size].copy()
        for i in range(b, b + size):
            for j in range(b + size, nt):
                g[i - b] -= T[i, j] * (Mx @ z[j])
        if size == 1:
            lu = spla.splu(sp.csc_matrix(Kx + T[b, b] * Mx))
            z[b] = lu.solve(g[0])
        else:
            alpha = T[b, b]
            x, y, it = block_solve(Kx, Mx, alpha, T[b, b + 1], T[b + 1, b], g[0], g[1],
                                   tol=tol, maxit=maxit)
            z[b], z[b + 1] = x, y
            itmax = max(itmax, it)
    return (X @ z).reshape(-1), itmax


def minres_bound_iterations(tol, kappa=np.sqrt(2.0)):
    """Iterations after which the MinRes bound for a spectrum inside
    [-1, -1/kappa] u [1/kappa, 1],
        ||r_k|| <= 2 ((kappa - 1)/(kappa + 1))^floor(k/2) ||r_0||,
    is at most tol (the two-interval Chebyshev bound)."""
    q = (kappa - 1.0) / (kappa + 1.0)
    return 2 * int(np.ceil(np.log(tol / 2.0) / np.log(q)))


def complex_factors(Kt, Mt, variant):
    """Complex factors of Eq. 3.1, K_t X = M_t X T, Y = (M_t X)^{-1}:
    variant "eig" (Sec. 3.3): T = diag(lambda), X the eigenvectors of the
    pencil (K_t, M_t); variant "cschur" (Sec. 3.4): the complex Schur form
    M_t^{-1} K_t = Q T Q^H, X = Q unitary, T upper triangular."""
    if variant == "eig":
        lam, X = sla.eig(Kt, Mt)
        T = np.diag(lam)
    elif variant == "cschur":
        T, X = sla.schur(np.linalg.solve(Mt, Kt).astype(complex), output="complex")
    else:
        raise ValueError(variant)
    Y = np.linalg.inv(Mt @ X)
    return T, X, Y


def slab_solve_minres_complex(prob, r, variant, tol=1e-4, maxit=500):
    """A_n^{-1} r by Eq. 3.1 with complex factors (``complex_factors``):
    w = (Y (x) I) r, then Algorithm 1 from the last row to the first,

        g_i = w_i - sum_{j > i} T_ij M_x z_j,   (K_x + lambda_i M_x) z_i = g_i,

    each complex shift lambda_i = alpha + i beta solved by MinRes in Theorem
    3.2's form (the 2x2 real block with beta1 = -beta, beta2 = beta); a real
    eigenvalue (|beta| <= 1e-13 |lambda|) by a direct solve of its real and
    imaginary parts.  The diagonalisation has no back substitution (T is
    diagonal).  Returns (Re (X (x) I) z, max MinRes iterations)."""
    Mx, Kx = assemble.spatial_operators(prob)
    Kt, Mt = assemble.time_matrices(prob.tau, prob.ne, prob.p, prob.delta)
    T, X, Y = complex_factors(Kt, Mt, variant)
    nt, m = prob.Nt, prob.Nx
    w = Y @ np.asarray(r, float).reshape(nt, m)
    z = np.zeros((nt, m), dtype=complex)
    itmax = 0
    for i in reversed(range(nt)):
        g = w[i].copy()
        for j in range(i + 1, nt):
            g -= T[i, j] * (Mx @ z[j])
        lam = T[i, i]
        if abs(lam.imag) <= 1e-13 * abs(lam):
            lu = spla.splu(sp.csc_matrix(Kx + lam.real * Mx))
            z[i] = lu.solve(g.real) + 1j * lu.solve(g.imag)
        else:
            x, y, it = block_solve(Kx, Mx, lam.real, -lam.imag, lam.imag, g.real, g.imag,
                                   tol=tol, maxit=maxit)
            z[i] = x + 1j * y
            itmax = max(itmax, it)
    return (X @ z).real.reshape(-1), itmax


def jacobi_step_minres(prob, u, f, omega=0.5, tol=1e-4, variant="rschur"):
    """One damped block-Jacobi step of Sec. 3.1, u + omega D^{-1} (f - L u),
    with every slab inverse applied by ``slab_solve_minres`` (variant
    "rschur") or ``slab_solve_minres_complex`` ("eig", "cschur") -- inexact,
    the smoothers of the paper's multigrid runs with MinRes block solves
    (Table 4).  Returns (new u, max MinRes iterations over the slabs)."""
    L = assemble.assemble_L(prob)
    r = (np.asarray(f, float) - L @ u).reshape(prob.N, -1)
    out = np.array(u, dtype=float).reshape(prob.N, -1).copy()
    itmax = 0
    for n in range(prob.N):
        if variant == "rschur":
            z, it = slab_solve_minres(prob, r[n], tol=tol)
        else:
            z, it = slab_solve_minres_complex(prob, r[n], variant, tol=tol)
        out[n] += omega * z
        itmax = max(itmax, it)
    return out.reshape(-1), itmax

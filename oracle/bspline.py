"""B-spline bases for the oracle (Sec. 2.1 of arXiv:1802.09277).

Test infrastructure only (see ``oracle/__init__.py``).

The paper builds its discrete spaces from B-splines defined by the Cox-de Boor
recursion on an open knot vector over [0, 1] (tensor products in d
dimensions).  Its knot-count formula is garbled; the reading used here is the
standard open uniform knot vector with ``s`` spans: the end knots repeated
``p + 1`` times, ``s - 1`` simple interior knots, hence ``s + p`` basis
functions of maximal smoothness C^{p-1}.
"""
import numpy as np


def open_knots(a, b, nel, p):
    """Open uniform knot vector on [a, b] with ``nel`` elements, degree ``p``."""
    inner = np.linspace(a, b, nel + 1)
    return np.concatenate([np.full(p, float(a)), inner, np.full(p, float(b))])


def n_basis(knots, p):
    return len(knots) - p - 1


def _degree0(knots, x):
    """Indicator functions of the knot spans [t_i, t_{i+1}); the right end
    point b belongs to the last non-empty span so that the basis is
    evaluated as a left limit there."""
    m = len(knots) - 1
    out = np.zeros((len(x), m))
    for i in range(m):
        if knots[i] < knots[i + 1]:
            out[:, i] = (knots[i] <= x) & (x < knots[i + 1])
    last = max(i for i in range(m) if knots[i] < knots[i + 1])
    out[x == knots[-1], last] = 1.0
    return out


def _raise_degree(knots, vals, k, x):
    """One Cox-de Boor step: degree k-1 values -> degree k values."""
    m = vals.shape[1] - 1
    out = np.zeros((len(x), m))
    for i in range(m):
        d1 = knots[i + k] - knots[i]
        d2 = knots[i + k + 1] - knots[i + 1]
        if d1 > 0:
            out[:, i] += (x - knots[i]) / d1 * vals[:, i]
        if d2 > 0:
            out[:, i] += (knots[i + k + 1] - x) / d2 * vals[:, i + 1]
    return out


def basis(knots, p, x):
    """Values of all degree-p B-splines at points x: array [len(x), n_basis]."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    knots = np.asarray(knots, dtype=float)
    vals = _degree0(knots, x)
    for k in range(1, p + 1):
        vals = _raise_degree(knots, vals, k, x)
    return vals


def basis_deriv(knots, p, x):
    """First derivatives of all degree-p B-splines at x, from the standard
    derivative formula N'_{i,p} = p/(t_{i+p}-t_i) N_{i,p-1}
    - p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    knots = np.asarray(knots, dtype=float)
    nb = n_basis(knots, p)
    if p == 0:
        return np.zeros((len(x), nb))
    low = basis(knots, p - 1, x)  # nb + 1 functions
    out = np.zeros((len(x), nb))
    for i in range(nb):
        d1 = knots[i + p] - knots[i]
        d2 = knots[i + p + 1] - knots[i + 1]
        if d1 > 0:
            out[:, i] += p / d1 * low[:, i]
        if d2 > 0:
            out[:, i] -= p / d2 * low[:, i + 1]
    return out


def element_quadrature(knots, npts):
    """Gauss-Legendre points/weights on every non-empty knot span."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    brk = np.unique(knots)
    pts, wts = [], []
    for a, b in zip(brk[:-1], brk[1:]):
        pts.append(0.5 * (b - a) * xg + 0.5 * (b + a))
        wts.append(0.5 * (b - a) * wg)
    return np.concatenate(pts), np.concatenate(wts)

// Host-side FP64 setup of the space-time multigrid (no CUDA).
//
// Everything here runs once per handle on the host: Gauss-Legendre rules,
// B-spline bases on open uniform knot vectors (Sec. 2.1 of arXiv:1802.09277),
// the 1D space matrices M1, K1 and the SUPG-weighted time matrices K_t, M_t
// (Eq. 2.6), the generalized symmetric eigenproblem K1 U = M1 U Lambda that
// drives the spatial fast diagonalisation, the real Schur form
// M_t^{-1} K_t = Q T Q^T of Sec. 3.5 and the time prolongation P_t of two
// slabs onto one (Sec. 3.1).  Matrices are dense row-major std::vector.
#pragma once
#include <string>
#include <vector>

namespace st {
namespace host {

using Mat = std::vector<double>;  // row-major, size rows*cols

// Gauss-Legendre nodes/weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);

// Open uniform knot vector on [a, b]: a, b repeated p+1 times, nel elements.
std::vector<double> open_knots(double a, double b, int nel, int p);

// Values and first derivatives of ALL nb = knots.size()-p-1 B-splines of
// degree p at x (zero outside their support).  At x == b the left limit is
// used (the last non-empty span).
void eval_basis(const std::vector<double> &knots, int p, double x,
                std::vector<double> &val, std::vector<double> &der);

// M1[i][j] = int phi_j phi_i, K1[i][j] = int phi_j' phi_i' on (0,1) with s
// spans, degree p, first and last basis function removed: n = s + p - 2.
void space_matrices(int s, int p, Mat &M1, Mat &K1);

// Px (n_f x n_c, row-major): the interior B-splines of s/2 spans on (0,1)
// in the interior B-splines of s spans (s even; nested spaces, so exact).
void space_prolongation(int s, int p, Mat &Px);

// K_t, M_t (Eq. 2.6) on one slab of length tau with ne elements, SUPG
// weight delta = theta*h: nt = ne + p.
void time_matrices(double tau, int ne, int p, double delta, Mat &Kt, Mat &Mt);

// P_t (2nt x nt): coarse slab [0, 2tau] (ne elements) expressed in the two
// fine slabs [0,tau], [tau,2tau] (ne elements each), by collocation at the
// fine bases' Greville abscissae.
void time_prolongation(double tau, int ne, int p, Mat &Pt);

// Solve A X = B (n x n, n x m) by Gaussian elimination with partial
// pivoting; returns false if A is singular to working precision.
bool lu_solve(int n, int m, Mat A, Mat &B);

// Generalized symmetric-definite eigenproblem K U = M U diag(lam), with
// U^T M U = I, eigenvalues ascending.  Cholesky of M + cyclic Jacobi.
bool sym_gen_eig(int n, const Mat &K, const Mat &M, Mat &U, std::vector<double> &lam,
                 std::string &err);

// Real Schur form A = Q T Q^T (Householder-Hessenberg + Francis double-shift
// QR), T quasi upper triangular with 1x1 blocks for real eigenvalues and 2x2
// blocks only for complex-conjugate pairs.  blk[i] = 1 if row i is the
// second row of a 2x2 block, else 0.
bool real_schur(int n, const Mat &A, Mat &Q, Mat &T, std::vector<int> &blk, std::string &err);

// Rotate every 2x2 block of a real Schur form (Q, T) to the standard form
// [[alpha, beta1], [beta2, alpha]] (Sec. 3.5): T <- G^T T G, Q <- Q G with G
// the rotation by t = atan2(d - a, b + c) / 2 for the block [[a, b], [c, d]]
// (the diagonal difference of G^T B G is cos 2t (a - d) + sin 2t (b + c)).
void standardize_schur(int n, Mat &Q, Mat &T, const std::vector<int> &blk);

// Eigen-decomposition A X = X diag(lam) from the real Schur form A = Q T Q^T
// (blk as returned by real_schur): eigenvectors of T by back substitution
// (complex for the 2x2 blocks), X = Q V, columns scaled to unit 2-norm.
// Re/Im parts returned separately (row-major n x n).
bool schur_eigvecs(int n, const Mat &Q, const Mat &T, const std::vector<int> &blk,
                   std::vector<double> &lam_re, std::vector<double> &lam_im, Mat &Xre, Mat &Xim,
                   std::string &err);

// Complex Schur form A = Q_c T_c Q_c^H (Sec. 3.4) from the real Schur form
// A = Q T Q^T: every 2x2 block is triangularised by a 2x2 unitary rotation.
// T_c is upper triangular with the eigenvalues on its diagonal.
bool complex_schur(int n, const Mat &Q, const Mat &T, const std::vector<int> &blk, Mat &Qre,
                   Mat &Qim, Mat &Tre, Mat &Tim, std::string &err);

// Inverse of the complex matrix (A_re + i A_im) by Gauss-Jordan with partial
// pivoting; false if singular.
bool complex_inverse(int n, const Mat &Are, const Mat &Aim, Mat &Bre, Mat &Bim);

// 2-norm condition number of a complex matrix (power iteration on M^H M and
// on its inverse).
double complex_cond2(int n, const Mat &Are, const Mat &Aim);

// g[i] = int_a^b func(x) (phi_i(x) + delta phi_i'(x)) dx over the B-splines of
// an open knot vector on [a, b] with nel elements (first/last removed if
// interior_only), Gauss-Legendre with npts points per element.
template <typename F>
std::vector<double> load_1d(double a, double b, int nel, int p, double delta, bool interior_only,
                            int npts, F func) {
    const std::vector<double> t = open_knots(a, b, nel, p);
    const int nb = nel + p;
    std::vector<double> g(nb, 0.0), gx, gw, v, d;
    gauss_legendre(npts, gx, gw);
    for (int e = 0; e < nel; ++e) {
        const double lo = a + (b - a) * e / nel, hi = a + (b - a) * (e + 1) / nel;
        for (int q = 0; q < npts; ++q) {
            const double x = 0.5 * (hi - lo) * (gx[q] + 1.0) + lo, w = 0.5 * (hi - lo) * gw[q];
            eval_basis(t, p, x, v, d);
            const double fx = func(x);
            for (int i = 0; i < nb; ++i) g[i] += w * fx * (v[i] + delta * d[i]);
        }
    }
    if (interior_only) return std::vector<double>(g.begin() + 1, g.end() - 1);
    return g;
}

// Frobenius norm of A*B - C (n x n), helper for the residual checks.
double resid_norm(int n, const Mat &A, const Mat &B, const Mat &C);
double frob(const Mat &A);
Mat matmul(int n, const Mat &A, const Mat &B);

}  // namespace host
}  // namespace st

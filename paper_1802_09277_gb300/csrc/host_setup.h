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

// Frobenius norm of A*B - C (n x n), helper for the residual checks.
double resid_norm(int n, const Mat &A, const Mat &B, const Mat &C);
double frob(const Mat &A);
Mat matmul(int n, const Mat &A, const Mat &B);

}  // namespace host
}  // namespace st

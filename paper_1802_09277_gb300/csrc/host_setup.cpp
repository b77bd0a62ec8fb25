// Host-side FP64 setup: see host_setup.h.
#include "host_setup.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>

namespace st {
namespace host {

static const double kPi = 3.14159265358979323846;

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        // initial guess for the i-th root (descending), Newton on P_n
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {  // three-term recurrence
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

std::vector<double> open_knots(double a, double b, int nel, int p) {
    std::vector<double> k;
    for (int i = 0; i < p; ++i) k.push_back(a);
    for (int e = 0; e <= nel; ++e) k.push_back(a + (b - a) * e / nel);
    k.back() = b;
    for (int i = 0; i < p; ++i) k.push_back(b);
    return k;
}

// index s of the span [t_s, t_{s+1}) holding x (p <= s < nb); the right end
// belongs to the last non-empty span
static int find_span(const std::vector<double> &t, int p, double x) {
    const int nb = (int)t.size() - p - 1;
    if (x >= t[nb]) {
        int s = nb - 1;
        while (s > p && t[s] == t[s + 1]) --s;
        return s;
    }
    int s = p;
    while (s < nb - 1 && x >= t[s + 1]) ++s;
    return s;
}

void eval_basis(const std::vector<double> &t, int p, double x, std::vector<double> &val,
                std::vector<double> &der) {
    const int nb = (int)t.size() - p - 1;
    val.assign(nb, 0.0);
    der.assign(nb, 0.0);
    const int s = find_span(t, p, x);
    // tri[k][r] = N_{s-k+r, k}(x), r = 0..k: the degree-k functions that do
    // not vanish on span s, raised one degree at a time
    double tri[16][16] = {{0.0}};
    tri[0][0] = 1.0;
    for (int k = 1; k <= p; ++k) {
        for (int r = 0; r <= k; ++r) {
            const int i = s - k + r;
            double v = 0.0;
            if (r >= 1) {  // N_{i,k-1} = tri[k-1][r-1]
                const double den = t[i + k] - t[i];
                if (den > 0.0) v += (x - t[i]) / den * tri[k - 1][r - 1];
            }
            if (r <= k - 1) {  // N_{i+1,k-1} = tri[k-1][r]
                const double den = t[i + k + 1] - t[i + 1];
                if (den > 0.0) v += (t[i + k + 1] - x) / den * tri[k - 1][r];
            }
            tri[k][r] = v;
        }
    }
    for (int r = 0; r <= p; ++r) {
        const int i = s - p + r;
        val[i] = tri[p][r];
        if (p == 0) continue;
        double d = 0.0;
        if (r >= 1) {
            const double den = t[i + p] - t[i];
            if (den > 0.0) d += p / den * tri[p - 1][r - 1];
        }
        if (r <= p - 1) {
            const double den = t[i + p + 1] - t[i + 1];
            if (den > 0.0) d -= p / den * tri[p - 1][r];
        }
        der[i] = d;
    }
}

void space_matrices(int s, int p, Mat &M1, Mat &K1) {
    const std::vector<double> t = open_knots(0.0, 1.0, s, p);
    const int nb = s + p, n = nb - 2;
    Mat Mf(nb * nb, 0.0), Kf(nb * nb, 0.0);
    std::vector<double> gx, gw, v, d;
    gauss_legendre(p + 2, gx, gw);
    for (int e = 0; e < s; ++e) {
        const double a = (double)e / s, b = (double)(e + 1) / s;
        for (size_t q = 0; q < gx.size(); ++q) {
            const double x = 0.5 * (b - a) * (gx[q] + 1.0) + a, w = 0.5 * (b - a) * gw[q];
            eval_basis(t, p, x, v, d);
            for (int i = 0; i < nb; ++i) {
                if (v[i] == 0.0 && d[i] == 0.0) continue;
                for (int j = 0; j < nb; ++j) {
                    Mf[i * nb + j] += w * v[i] * v[j];
                    Kf[i * nb + j] += w * d[i] * d[j];
                }
            }
        }
    }
    M1.assign(n * n, 0.0);
    K1.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            M1[i * n + j] = Mf[(i + 1) * nb + j + 1];
            K1[i * n + j] = Kf[(i + 1) * nb + j + 1];
        }
}

void space_prolongation(int s, int p, Mat &Px) {
    // interior functions: fine n_f = s + p - 2 on s spans, coarse n_c on s/2;
    // a coarse interior B-spline vanishes at both ends, so it is a combination
    // of the fine interior ones; collocation at their Greville abscissae
    // (Schoenberg-Whitney: the collocation matrix is nonsingular) finds it
    const std::vector<double> tf = open_knots(0.0, 1.0, s, p);
    const std::vector<double> tc = open_knots(0.0, 1.0, s / 2, p);
    const int nf = s + p - 2, nc = s / 2 + p - 2;
    Mat Bf((size_t)nf * nf), Bc((size_t)nf * nc);
    std::vector<double> v, d;
    for (int m = 0; m < nf; ++m) {
        double g = 0.0;  // Greville abscissa of fine function m + 1
        for (int k = 1; k <= p; ++k) g += tf[m + 1 + k];
        g = (p > 0) ? g / p : tf[m + 1];
        eval_basis(tf, p, g, v, d);
        for (int a = 0; a < nf; ++a) Bf[(size_t)m * nf + a] = v[a + 1];
        eval_basis(tc, p, g, v, d);
        for (int b = 0; b < nc; ++b) Bc[(size_t)m * nc + b] = v[b + 1];
    }
    lu_solve(nf, nc, Bf, Bc);
    Px = Bc;
}

void time_matrices(double tau, int ne, int p, double delta, Mat &Kt, Mat &Mt) {
    const std::vector<double> t = open_knots(0.0, tau, ne, p);
    const int nt = ne + p;
    Kt.assign(nt * nt, 0.0);
    Mt.assign(nt * nt, 0.0);
    std::vector<double> gx, gw, v, d;
    gauss_legendre(p + 2, gx, gw);
    for (int e = 0; e < ne; ++e) {
        const double a = tau * e / ne, b = tau * (e + 1) / ne;
        for (size_t q = 0; q < gx.size(); ++q) {
            const double x = 0.5 * (b - a) * (gx[q] + 1.0) + a, w = 0.5 * (b - a) * gw[q];
            eval_basis(t, p, x, v, d);
            for (int i = 0; i < nt; ++i) {
                const double test = v[i] + delta * d[i];  // psi_i + theta h psi_i'
                for (int j = 0; j < nt; ++j) {
                    Kt[i * nt + j] += w * d[j] * test;
                    Mt[i * nt + j] += w * v[j] * test;
                }
            }
        }
    }
    eval_basis(t, p, 0.0, v, d);  // upwind term psi_j(t_{n-1}) psi_i(t_{n-1})
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nt; ++j) Kt[i * nt + j] += v[j] * v[i];
}

void time_prolongation(double tau, int ne, int p, Mat &Pt) {
    const int nt = ne + p;
    const std::vector<double> tc = open_knots(0.0, 2.0 * tau, ne, p);
    Pt.assign(2 * nt * nt, 0.0);
    std::vector<double> v, d;
    for (int q = 0; q < 2; ++q) {
        const std::vector<double> tf = open_knots(q * tau, (q + 1) * tau, ne, p);
        Mat Bf(nt * nt), Bc(nt * nt);
        for (int m = 0; m < nt; ++m) {
            double g = 0.0;  // Greville abscissa of fine function m
            for (int k = 1; k <= p; ++k) g += tf[m + k];
            g = (p > 0) ? g / p : tf[m];
            eval_basis(tf, p, g, v, d);
            for (int a = 0; a < nt; ++a) Bf[m * nt + a] = v[a];
            eval_basis(tc, p, g, v, d);
            for (int b = 0; b < nt; ++b) Bc[m * nt + b] = v[b];
        }
        lu_solve(nt, nt, Bf, Bc);
        for (int a = 0; a < nt; ++a)
            for (int b = 0; b < nt; ++b) Pt[(q * nt + a) * nt + b] = Bc[a * nt + b];
    }
}

bool lu_solve(int n, int m, Mat A, Mat &B) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A[i * n + k]) > std::fabs(A[piv * n + k])) piv = i;
        if (A[piv * n + k] == 0.0) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
            for (int j = 0; j < m; ++j) std::swap(B[k * m + j], B[piv * m + j]);
        }
        for (int i = k + 1; i < n; ++i) {
            const double l = A[i * n + k] / A[k * n + k];
            if (l == 0.0) continue;
            for (int j = k; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
            for (int j = 0; j < m; ++j) B[i * m + j] -= l * B[k * m + j];
        }
    }
    for (int i = n - 1; i >= 0; --i)
        for (int j = 0; j < m; ++j) {
            double s = B[i * m + j];
            for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * B[k * m + j];
            B[i * m + j] = s / A[i * n + i];
        }
    return true;
}

double frob(const Mat &A) {
    double s = 0.0;
    for (double a : A) s += a * a;
    return std::sqrt(s);
}

Mat matmul(int n, const Mat &A, const Mat &B) {
    Mat C(n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double a = A[i * n + k];
            for (int j = 0; j < n; ++j) C[i * n + j] += a * B[k * n + j];
        }
    return C;
}

double resid_norm(int n, const Mat &A, const Mat &B, const Mat &C) {
    Mat P = matmul(n, A, B);
    double s = 0.0;
    for (int i = 0; i < n * n; ++i) s += (P[i] - C[i]) * (P[i] - C[i]);
    return std::sqrt(s);
}

bool sym_gen_eig(int n, const Mat &K, const Mat &M, Mat &U, std::vector<double> &lam,
                 std::string &err) {
    // Cholesky M = L L^T (L lower)
    Mat L(n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = M[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) {
            err = "space mass matrix is not positive definite";
            return false;
        }
        L[j * n + j] = std::sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = M[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    // C = L^{-1} K L^{-T}: first W = L^{-1} K (forward substitution per column)
    Mat W(K);
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double s = W[i * n + c];
            for (int k = 0; k < i; ++k) s -= L[i * n + k] * W[k * n + c];
            W[i * n + c] = s / L[i * n + i];
        }
    // C^T = L^{-1} W^T, and C is symmetric
    Mat C(n * n);
    for (int r = 0; r < n; ++r)
        for (int i = 0; i < n; ++i) {
            double s = W[r * n + i];
            for (int k = 0; k < i; ++k) s -= L[i * n + k] * C[r * n + k];
            C[r * n + i] = s / L[i * n + i];
        }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double a = 0.5 * (C[i * n + j] + C[j * n + i]);
            C[i * n + j] = C[j * n + i] = a;
        }
    // cyclic Jacobi: C <- J^T C J until off-diagonal mass is negligible
    Mat V(n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    const double cnorm = frob(C);
    bool converged = (n == 1);
    for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += C[i * n + j] * C[i * n + j];
        if (std::sqrt(2.0 * off) <= 1e-17 * cnorm) {
            converged = true;
            break;
        }
        for (int pi = 0; pi < n - 1; ++pi)
            for (int qi = pi + 1; qi < n; ++qi) {
                const double apq = C[pi * n + qi];
                if (std::fabs(apq) < 1e-300) continue;
                const double app = C[pi * n + pi], aqq = C[qi * n + qi];
                const double th = (aqq - app) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double ckp = C[k * n + pi], ckq = C[k * n + qi];
                    C[k * n + pi] = c * ckp - s * ckq;
                    C[k * n + qi] = s * ckp + c * ckq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double cpk = C[pi * n + k], cqk = C[qi * n + k];
                    C[pi * n + k] = c * cpk - s * cqk;
                    C[qi * n + k] = s * cpk + c * cqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + pi], vkq = V[k * n + qi];
                    V[k * n + pi] = c * vkp - s * vkq;
                    V[k * n + qi] = s * vkp + c * vkq;
                }
            }
    }
    if (!converged) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += C[i * n + j] * C[i * n + j];
        if (std::sqrt(2.0 * off) > 1e-13 * cnorm) {
            err = "Jacobi eigensolver did not converge";
            return false;
        }
    }
    // sort ascending, U = L^{-T} V
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return C[a * n + a] < C[b * n + b]; });
    lam.resize(n);
    U.assign(n * n, 0.0);
    for (int c = 0; c < n; ++c) {
        lam[c] = C[idx[c] * n + idx[c]];
        for (int i = n - 1; i >= 0; --i) {  // back substitution with L^T
            double s = V[i * n + idx[c]];
            for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * U[k * n + c];
            U[i * n + c] = s / L[i * n + i];
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Real Schur form
// ---------------------------------------------------------------------------

// Apply the reflector I - beta v v^T (v of length m, rows/cols k..k+m-1).
static void reflect_rows(int n, Mat &H, int k, int m, const double *v, double beta, int c0, int c1) {
    for (int j = c0; j <= c1; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += v[i] * H[(k + i) * n + j];
        s *= beta;
        for (int i = 0; i < m; ++i) H[(k + i) * n + j] -= s * v[i];
    }
}
static void reflect_cols(int n, Mat &H, int k, int m, const double *v, double beta, int r0, int r1) {
    for (int i = r0; i <= r1; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += H[i * n + k + j] * v[j];
        s *= beta;
        for (int j = 0; j < m; ++j) H[i * n + k + j] -= s * v[j];
    }
}
// v, beta with (I - beta v v^T) x = -sign(x0) ||x|| e1; returns false if x = 0
static bool householder(int m, const double *x, double *v, double &beta) {
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return false;
    const double alpha = (x[0] >= 0.0) ? -nrm : nrm;
    for (int i = 0; i < m; ++i) v[i] = x[i];
    v[0] -= alpha;
    double vv = 0.0;
    for (int i = 0; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) return false;
    beta = 2.0 / vv;
    return true;
}

// Rotate rows/cols k, k+1 by G = [[c, -s], [s, c]] : H <- G^T H G, Q <- Q G
static void rotate(int n, Mat &H, Mat &Q, int k, double c, double s) {
    for (int j = 0; j < n; ++j) {
        const double a = H[k * n + j], b = H[(k + 1) * n + j];
        H[k * n + j] = c * a + s * b;
        H[(k + 1) * n + j] = -s * a + c * b;
    }
    for (int i = 0; i < n; ++i) {
        const double a = H[i * n + k], b = H[i * n + k + 1];
        H[i * n + k] = c * a + s * b;
        H[i * n + k + 1] = -s * a + c * b;
        const double qa = Q[i * n + k], qb = Q[i * n + k + 1];
        Q[i * n + k] = c * qa + s * qb;
        Q[i * n + k + 1] = -s * qa + c * qb;
    }
}

bool real_schur(int n, const Mat &A, Mat &Q, Mat &T, std::vector<int> &blk, std::string &err) {
    Mat H(A);
    Q.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
    double v[16], x[16], beta;
    // 1. Householder reduction to upper Hessenberg form
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        for (int i = 0; i < m; ++i) x[i] = H[(k + 1 + i) * n + k];
        if (!householder(m, x, v, beta)) continue;
        reflect_rows(n, H, k + 1, m, v, beta, 0, n - 1);
        reflect_cols(n, H, k + 1, m, v, beta, 0, n - 1);
        reflect_cols(n, Q, k + 1, m, v, beta, 0, n - 1);
        for (int i = k + 2; i < n; ++i) H[i * n + k] = 0.0;
    }
    // 2. Francis double-shift QR with deflation
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0;
    while (hi >= 0) {
        if (iter > 60 * n) {
            err = "Francis QR iteration did not converge";
            return false;
        }
        int lo = hi;  // start of the unreduced block ending at hi
        while (lo > 0) {
            const double sub = std::fabs(H[lo * n + lo - 1]);
            double scale = std::fabs(H[(lo - 1) * n + lo - 1]) + std::fabs(H[lo * n + lo]);
            if (scale == 0.0) scale = frob(H);
            if (sub <= eps * scale) {
                H[lo * n + lo - 1] = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {  // 1x1 block converged
            --hi;
            iter = 0;
            continue;
        }
        if (lo == hi - 1) {  // 2x2 block: split it if its eigenvalues are real
            const int k = lo;
            const double a = H[k * n + k], b = H[k * n + k + 1];
            const double c = H[(k + 1) * n + k], d = H[(k + 1) * n + k + 1];
            const double hd = 0.5 * (a - d), disc = hd * hd + b * c;
            if (disc >= 0.0) {
                const double r = std::sqrt(disc);
                const double l1 = 0.5 * (a + d) + (hd >= 0 ? r : -r);  // larger |.| root
                // eigenvector of [[a,b],[c,d]] for l1 as first rotation column
                double e0 = b, e1 = l1 - a;
                if (std::fabs(l1 - d) + std::fabs(c) > std::fabs(e0) + std::fabs(e1)) {
                    e0 = l1 - d;
                    e1 = c;
                }
                const double nr = std::hypot(e0, e1);
                if (nr > 0.0) {
                    rotate(n, H, Q, k, e0 / nr, e1 / nr);
                    H[(k + 1) * n + k] = 0.0;
                }
            }
            hi -= 2;
            iter = 0;
            continue;
        }
        // Francis double-shift step on the window lo..hi
        ++iter;
        double s = H[(hi - 1) * n + hi - 1] + H[hi * n + hi];
        double t = H[(hi - 1) * n + hi - 1] * H[hi * n + hi] - H[(hi - 1) * n + hi] * H[hi * n + hi - 1];
        if (iter % 11 == 0) {  // exceptional shift
            const double w = std::fabs(H[hi * n + hi - 1]) + std::fabs(H[(hi - 1) * n + hi - 2]);
            s = 1.5 * w;
            t = w * w;
        }
        double X0 = H[lo * n + lo] * H[lo * n + lo] + H[lo * n + lo + 1] * H[(lo + 1) * n + lo] -
                    s * H[lo * n + lo] + t;
        double X1 = H[(lo + 1) * n + lo] * (H[lo * n + lo] + H[(lo + 1) * n + lo + 1] - s);
        double X2 = H[(lo + 1) * n + lo] * H[(lo + 2) * n + lo + 1];
        for (int k = lo; k <= hi - 2; ++k) {
            x[0] = X0;
            x[1] = X1;
            x[2] = X2;
            if (householder(3, x, v, beta)) {
                const int r = std::max(lo, k - 1);
                reflect_rows(n, H, k, 3, v, beta, r, n - 1);
                const int rr = std::min(k + 3, hi);
                reflect_cols(n, H, k, 3, v, beta, 0, rr);
                reflect_cols(n, Q, k, 3, v, beta, 0, n - 1);
            }
            X0 = H[(k + 1) * n + k];
            X1 = H[(k + 2) * n + k];
            if (k < hi - 2) X2 = H[(k + 3) * n + k];
        }
        x[0] = X0;
        x[1] = X1;
        if (householder(2, x, v, beta)) {
            reflect_rows(n, H, hi - 1, 2, v, beta, hi - 2, n - 1);
            reflect_cols(n, H, hi - 1, 2, v, beta, 0, hi);
            reflect_cols(n, Q, hi - 1, 2, v, beta, 0, n - 1);
        }
        for (int i = lo + 2; i <= hi; ++i)
            for (int j = lo; j < i - 1; ++j) H[i * n + j] = 0.0;
    }
    T = H;
    blk.assign(n, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i > j + 1) T[i * n + j] = 0.0;
    for (int i = 1; i < n; ++i)
        if (T[i * n + i - 1] != 0.0) blk[i] = 1;
    for (int i = 1; i < n; ++i)
        if (blk[i] && i >= 2 && blk[i - 1]) {
            err = "Schur form has overlapping 2x2 blocks";
            return false;
        }
    // residual check ||A Q - Q T|| <= tol ||A||
    const double r = std::sqrt(std::pow(resid_norm(n, A, Q, matmul(n, Q, T)), 2));
    if (!(r <= 1e-12 * std::max(1.0, frob(A)))) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "Schur residual %.3e too large", r);
        err = buf;
        return false;
    }
    return true;
}

void standardize_schur(int n, Mat &Q, Mat &T, const std::vector<int> &blk) {
    for (int k = 0; k + 1 < n; ++k) {
        if (!blk[k + 1]) continue;
        const double a = T[k * n + k], b = T[k * n + k + 1];
        const double c = T[(k + 1) * n + k], d = T[(k + 1) * n + k + 1];
        const double t = 0.5 * std::atan2(d - a, b + c);
        rotate(n, T, Q, k, std::cos(t), std::sin(t));
        const double al = 0.5 * (T[k * n + k] + T[(k + 1) * n + k + 1]);
        T[k * n + k] = T[(k + 1) * n + k + 1] = al;
        // rows below the block stay zero up to rounding of the rotation
        for (int i = k + 2; i < n; ++i) T[i * n + k] = T[i * n + k + 1] = 0.0;
        ++k;
    }
}

using cd = std::complex<double>;

bool schur_eigvecs(int n, const Mat &Q, const Mat &T, const std::vector<int> &blk,
                   std::vector<double> &lam_re, std::vector<double> &lam_im, Mat &Xre, Mat &Xim,
                   std::string &err) {
    lam_re.assign(n, 0.0);
    lam_im.assign(n, 0.0);
    // eigenvalues from the diagonal blocks
    for (int i = 0; i < n; ++i) {
        if (i + 1 < n && blk[i + 1]) {
            const double a = T[i * n + i], b = T[i * n + i + 1];
            const double c = T[(i + 1) * n + i], d = T[(i + 1) * n + i + 1];
            const double hd = 0.5 * (a - d), disc = hd * hd + b * c;
            const double im = std::sqrt(std::max(-disc, 0.0));
            lam_re[i] = lam_re[i + 1] = 0.5 * (a + d);
            lam_im[i] = im;
            lam_im[i + 1] = -im;
            ++i;
        } else {
            lam_re[i] = T[i * n + i];
        }
    }
    // eigenvectors of T: (T - lam I) v = 0, v zero below the eigenvalue's block
    std::vector<cd> V(n * n, cd(0.0, 0.0));
    for (int k = 0; k < n; ++k) {
        const cd lam(lam_re[k], lam_im[k]);
        std::vector<cd> v(n, cd(0.0, 0.0));
        int top;  // first row of the eigenvalue's block
        if (k + 1 < n && blk[k + 1]) {  // first of a conjugate pair
            const double a = T[k * n + k], b = T[k * n + k + 1];
            v[k] = cd(b, 0.0);
            v[k + 1] = lam - a;
            top = k;
        } else if (blk[k]) {  // second of the pair: conjugate of the first
            for (int i = 0; i < n; ++i) V[i * n + k] = std::conj(V[i * n + k - 1]);
            continue;
        } else {
            v[k] = cd(1.0, 0.0);
            top = k;
        }
        // back substitution for rows above the block, block by block
        for (int i = top - 1; i >= 0; --i) {
            if (i >= 1 && blk[i]) {  // 2x2 block on rows i-1, i
                cd g1(0.0, 0.0), g2(0.0, 0.0);
                for (int j = i + 1; j < n; ++j) {
                    g1 -= T[(i - 1) * n + j] * v[j];
                    g2 -= T[i * n + j] * v[j];
                }
                const cd a = T[(i - 1) * n + i - 1] - lam, b = T[(i - 1) * n + i];
                const cd c = T[i * n + i - 1], d = T[i * n + i] - lam;
                const cd det = a * d - b * c;
                if (std::abs(det) == 0.0) {
                    err = "defective eigenvalue (repeated)";
                    return false;
                }
                v[i - 1] = (d * g1 - b * g2) / det;
                v[i] = (a * g2 - c * g1) / det;
                --i;
            } else {
                cd g(0.0, 0.0);
                for (int j = i + 1; j < n; ++j) g -= T[i * n + j] * v[j];
                const cd den = T[i * n + i] - lam;
                if (std::abs(den) == 0.0) {
                    err = "defective eigenvalue (repeated)";
                    return false;
                }
                v[i] = g / den;
            }
        }
        for (int i = 0; i < n; ++i) V[i * n + k] = v[i];
    }
    // X = Q V, unit 2-norm columns
    Xre.assign(n * n, 0.0);
    Xim.assign(n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        std::vector<cd> col(n, cd(0.0, 0.0));
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) col[i] += Q[i * n + j] * V[j * n + k];
            nrm += std::norm(col[i]);
        }
        nrm = std::sqrt(nrm);
        if (!(nrm > 0)) {
            err = "zero eigenvector";
            return false;
        }
        for (int i = 0; i < n; ++i) {
            Xre[i * n + k] = col[i].real() / nrm;
            Xim[i * n + k] = col[i].imag() / nrm;
        }
    }
    return true;
}

bool complex_inverse(int n, const Mat &Are, const Mat &Aim, Mat &Bre, Mat &Bim) {
    std::vector<cd> A(n * n), B(n * n, cd(0.0, 0.0));
    for (int i = 0; i < n * n; ++i) A[i] = cd(Are[i], Aim[i]);
    for (int i = 0; i < n; ++i) B[i * n + i] = cd(1.0, 0.0);
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(A[i * n + k]) > std::abs(A[piv * n + k])) piv = i;
        if (std::abs(A[piv * n + k]) == 0.0) return false;
        if (piv != k)
            for (int j = 0; j < n; ++j) {
                std::swap(A[k * n + j], A[piv * n + j]);
                std::swap(B[k * n + j], B[piv * n + j]);
            }
        const cd inv = 1.0 / A[k * n + k];
        for (int j = 0; j < n; ++j) {
            A[k * n + j] *= inv;
            B[k * n + j] *= inv;
        }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            const cd l = A[i * n + k];
            if (std::abs(l) == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[i * n + j] -= l * A[k * n + j];
                B[i * n + j] -= l * B[k * n + j];
            }
        }
    }
    Bre.resize(n * n);
    Bim.resize(n * n);
    for (int i = 0; i < n * n; ++i) {
        Bre[i] = B[i].real();
        Bim[i] = B[i].imag();
    }
    return true;
}

static double complex_norm2(int n, const std::vector<cd> &M) {
    // largest singular value: power iteration on M^H M
    std::vector<cd> x(n, cd(1.0, 0.0)), y(n), z(n);
    double s = 0.0;
    for (int it = 0; it < 500; ++it) {
        for (int i = 0; i < n; ++i) {
            y[i] = 0.0;
            for (int j = 0; j < n; ++j) y[i] += M[i * n + j] * x[j];
        }
        for (int j = 0; j < n; ++j) {
            z[j] = 0.0;
            for (int i = 0; i < n; ++i) z[j] += std::conj(M[i * n + j]) * y[i];
        }
        double nz = 0.0;
        for (int j = 0; j < n; ++j) nz += std::norm(z[j]);
        nz = std::sqrt(nz);
        if (!(nz > 0)) return 0.0;
        const double snew = std::sqrt(nz);
        for (int j = 0; j < n; ++j) x[j] = z[j] / nz;
        if (std::fabs(snew - s) <= 1e-13 * snew) {
            s = snew;
            break;
        }
        s = snew;
    }
    return s;
}

double complex_cond2(int n, const Mat &Are, const Mat &Aim) {
    Mat Bre, Bim;
    if (!complex_inverse(n, Are, Aim, Bre, Bim)) return INFINITY;
    std::vector<cd> A(n * n), B(n * n);
    for (int i = 0; i < n * n; ++i) {
        A[i] = cd(Are[i], Aim[i]);
        B[i] = cd(Bre[i], Bim[i]);
    }
    return complex_norm2(n, A) * complex_norm2(n, B);
}

// Complex Schur form from the real one: each 2x2 block B of T (a complex pair
// lambda, conj(lambda)) is made upper triangular by the unitary 2x2 matrix
// G = [g, g_perp] whose first column is the unit eigenvector g of B for
// lambda; T <- G^H T G and Q <- Q G on the two rows / columns of the block.
// The blocks are disjoint, so the updates commute.  A = Q T Q^H with T
// complex upper triangular (diagonal = the eigenvalues) and Q unitary.
bool complex_schur(int n, const Mat &Q, const Mat &T, const std::vector<int> &blk, Mat &Qre,
                   Mat &Qim, Mat &Tre, Mat &Tim, std::string &err) {
    using C = std::complex<double>;
    std::vector<C> q(n * n), t(n * n);
    for (int i = 0; i < n * n; ++i) {
        q[i] = Q[i];
        t[i] = T[i];
    }
    for (int i = 1; i < n; ++i) {
        if (!blk[i]) continue;
        const int r0 = i - 1, r1 = i;
        const double a = T[r0 * n + r0], b = T[r0 * n + r1], c = T[r1 * n + r0], d = T[r1 * n + r1];
        const double disc = (a - d) * (a - d) + 4.0 * b * c;
        if (!(disc < 0)) {
            err = "2x2 Schur block with real eigenvalues";
            return false;
        }
        const C lam(0.5 * (a + d), 0.5 * std::sqrt(-disc));
        // (B - lambda I) v = 0: v = (b, lambda - a), or (lambda - d, c)
        C v0(b, 0.0), v1 = lam - a;
        if (std::abs(v0) + std::abs(v1) < std::abs(lam - d) + std::abs(c)) {
            v0 = lam - d;
            v1 = C(c, 0.0);
        }
        const double nv = std::sqrt(std::norm(v0) + std::norm(v1));
        if (!(nv > 0)) {
            err = "degenerate 2x2 Schur block";
            return false;
        }
        v0 /= nv;
        v1 /= nv;
        // G = [[v0, -conj(v1)], [v1, conj(v0)]]
        const C g00 = v0, g01 = -std::conj(v1), g10 = v1, g11 = std::conj(v0);
        for (int row = 0; row < n; ++row) {  // columns r0, r1 of T and Q times G
            const C t0 = t[row * n + r0], t1 = t[row * n + r1];
            t[row * n + r0] = t0 * g00 + t1 * g10;
            t[row * n + r1] = t0 * g01 + t1 * g11;
            const C q0 = q[row * n + r0], q1 = q[row * n + r1];
            q[row * n + r0] = q0 * g00 + q1 * g10;
            q[row * n + r1] = q0 * g01 + q1 * g11;
        }
        for (int col = 0; col < n; ++col) {  // rows r0, r1 of T times G^H
            const C t0 = t[r0 * n + col], t1 = t[r1 * n + col];
            t[r0 * n + col] = std::conj(g00) * t0 + std::conj(g10) * t1;
            t[r1 * n + col] = std::conj(g01) * t0 + std::conj(g11) * t1;
        }
        t[r1 * n + r0] = 0.0;  // eliminated (rounding residue)
    }
    Qre.assign(n * n, 0.0);
    Qim.assign(n * n, 0.0);
    Tre.assign(n * n, 0.0);
    Tim.assign(n * n, 0.0);
    for (int i = 0; i < n * n; ++i) {
        Qre[i] = q[i].real();
        Qim[i] = q[i].imag();
        Tre[i] = t[i].real();
        Tim[i] = t[i].imag();
    }
    return true;
}

}  // namespace host
}  // namespace st

// Inexact spatial solves of the slab inverse (Sec. 3.3-3.5 of
// arXiv:1802.09277): preconditioned MinRes on batches of the 2x2 block
// spatial systems of a real Schur (or complex-shift) block, with the
// block-diagonal preconditioner of Theorem 3.3 (Theorem 3.2 for a complex
// shift) applied by fast diagonalisation.
//
// A batch holds nsys systems of c components (c = 1 or 2) of m spatial dofs
// each, laid out [sys][comp][m].  Element kernels run on a 2D grid:
// blockIdx.y is the system (or the system's component plane), blockIdx.x
// strides over its elements, so per-system scalars are read once per thread
// and no division by the system length is needed.  Scalars of the iteration
// (Lanczos coefficients, Givens rotations, the residual norm) live in one
// MrState per system on the device (two buffers, swapped every step), so the
// whole iteration runs without host synchronisation.
#include "st_internal.h"

namespace st {
namespace {

constexpr int MR_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// fixed-order sum of the chunk partials of system `sys`
__device__ __forceinline__ double part_sum(const double *part, int chunks, int sys) {
    double s = 0.0;
    for (int i = 0; i < chunks; ++i) s += part[(long long)sys * chunks + i];
    return s;
}

// part[sys][blockIdx.x] = partial sum of a[sys][e] * b[sys][e] over this CTA's
// elements (per-thread sums in T, the CTA reduction in FP64)
template <typename T>
__global__ void __launch_bounds__(MR_THREADS)
    k_seg_dot(const T *__restrict__ a, const T *__restrict__ b, double *__restrict__ part,
              long long len) {
    __shared__ double red[MR_THREADS / 32];
    const long long off = (long long)blockIdx.y * len;
    T acc = T(0);
    for (long long e = (long long)blockIdx.x * MR_THREADS + threadIdx.x; e < len;
         e += (long long)gridDim.x * MR_THREADS)
        acc += a[off + e] * b[off + e];
    double v = warp_sum((double)acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = (lane < MR_THREADS / 32) ? red[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = v;
    }
}

// beta_1 = ||r_0||_{P^{-1}} = sqrt(r_0 . P^{-1} r_0); initial rotations
__global__ void k_mr_init(const double *__restrict__ partB, int chunks, MrState *__restrict__ st,
                          int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const double b2 = part_sum(partB, chunks, s);
    const double beta = b2 > 0.0 ? sqrt(b2) : 0.0;
    MrState q;
    q.beta1 = beta;
    q.eta = beta;
    q.bk = 0.0;
    q.c1 = q.c2 = 1.0;
    q.s1 = q.s2 = 0.0;
    q.cd = q.cdel = q.ceps = q.cx = 0.0;
    q.invb = beta > 0.0 ? 1.0 / beta : 0.0;
    q.relres = beta > 0.0 ? 1.0 : 0.0;
    q.active = beta > 0.0 ? 1 : 0;
    q.upd = 0;
    q.iters = 0;
    q.pad = 0;
    st[s] = q;
}

// q_1 = r_0 / beta_1 (in place), p_1 = P^{-1} r_0 / beta_1; q_0 = d_0 = d_{-1} = x = 0
template <typename T>
__global__ void __launch_bounds__(MR_THREADS)
    k_mr_init_vec(T *__restrict__ q, T *__restrict__ p, const T *__restrict__ z,
                  T *__restrict__ qp, T *__restrict__ d1, T *__restrict__ d2, T *__restrict__ x,
                  const MrState *__restrict__ st, long long len) {
    const T ib = (T)st[blockIdx.y].invb;
    const long long off = (long long)blockIdx.y * len;
    for (long long e = (long long)blockIdx.x * MR_THREADS + threadIdx.x; e < len;
         e += (long long)gridDim.x * MR_THREADS) {
        const long long i = off + e;
        q[i] *= ib;
        p[i] = z[i] * ib;
        qp[i] = T(0);
        d1[i] = T(0);
        d2[i] = T(0);
        x[i] = T(0);
    }
}

// Lanczos step: t <- A p_k - alpha_k q_k - beta_k q_{k-1}, alpha_k = p_k . A p_k
template <typename T>
__global__ void __launch_bounds__(MR_THREADS)
    k_mr_lanczos(T *__restrict__ t, const T *__restrict__ q, const T *__restrict__ qp,
                 const double *__restrict__ partA, int chunks, const MrState *__restrict__ st,
                 long long len) {
    const int sys = blockIdx.y;
    if (!st[sys].active) return;
    const T al = (T)part_sum(partA, chunks, sys);
    const T bk = (T)st[sys].bk;
    const long long off = (long long)sys * len;
    for (long long e = (long long)blockIdx.x * MR_THREADS + threadIdx.x; e < len;
         e += (long long)gridDim.x * MR_THREADS) {
        const long long i = off + e;
        t[i] = t[i] - al * q[i] - bk * qp[i];
    }
}

// New column (beta_k, alpha_k, beta_{k+1}) of the tridiagonal matrix: apply
// the two previous rotations, choose the one that annihilates beta_{k+1},
// and record the coefficients of the direction and iterate updates
// (alpha = p_k . A p_k, b2 = beta_{k+1}^2).
__device__ MrState mr_rotate(MrState q, double alpha, double b2, double tol) {
    q.upd = 0;
    if (!q.active) return q;
    const double bn = b2 > 0.0 ? sqrt(b2) : 0.0;
    const double eps = q.s2 * q.bk;
    const double dbar = q.c2 * q.bk;
    const double delta = q.c1 * dbar + q.s1 * alpha;
    const double gbar = -q.s1 * dbar + q.c1 * alpha;
    const double rho = hypot(gbar, bn);
    if (!(rho > 0.0)) {  // breakdown: keep the current iterate
        q.active = 0;
        return q;
    }
    const double c = gbar / rho, sn = bn / rho;
    q.cd = 1.0 / rho;
    q.cdel = delta;
    q.ceps = eps;
    q.cx = c * q.eta;
    q.eta = -sn * q.eta;
    q.iters += 1;
    q.upd = 1;
    q.relres = fabs(q.eta) / q.beta1;
    if (fabs(q.eta) <= tol * q.beta1 || bn == 0.0) {
        q.active = 0;
        q.invb = 0.0;
    } else {
        q.invb = 1.0 / bn;
    }
    q.c2 = q.c1;
    q.s2 = q.s1;
    q.c1 = c;
    q.s1 = sn;
    q.bk = bn;
    return q;
}

// One MinRes step's rotation and vector update.  Thread 0 of every CTA of a
// system forms the new state from st_in and the chunk partials (the same
// fixed-order sums in every CTA); CTA 0 stores it in st_out (a second state
// buffer, so no CTA reads a state another one has already replaced).  Then
// d_k = (p_k - delta d_{k-1} - eps d_{k-2}) / rho (written over d_{k-2}),
// x += c eta d_k; if the system goes on: q_{k+1} = t / beta_{k+1} (in place),
// p_{k+1} = P^{-1} t / beta_{k+1} (over p_k).
template <typename T>
__global__ void __launch_bounds__(MR_THREADS)
    k_mr_step(T *__restrict__ p, const T *__restrict__ z, T *__restrict__ t,
              const T *__restrict__ d1, T *__restrict__ d2, T *__restrict__ x,
              const double *__restrict__ partA, const double *__restrict__ partB, int chunks,
              const MrState *__restrict__ st_in, MrState *__restrict__ st_out, double tol,
              long long len) {
    __shared__ MrState sh;
    const int sys = blockIdx.y;
    if (threadIdx.x == 0) {
        const MrState q = mr_rotate(st_in[sys], part_sum(partA, chunks, sys),
                                    part_sum(partB, chunks, sys), tol);
        sh = q;
        if (blockIdx.x == 0) st_out[sys] = q;
    }
    __syncthreads();
    if (!sh.upd) return;
    const T cd = (T)sh.cd, cdel = (T)sh.cdel, ceps = (T)sh.ceps;
    const T cx = (T)sh.cx, ib = (T)sh.invb;
    const bool go_on = sh.active != 0;
    const long long off = (long long)sys * len;
    for (long long e = (long long)blockIdx.x * MR_THREADS + threadIdx.x; e < len;
         e += (long long)gridDim.x * MR_THREADS) {
        const long long i = off + e;
        const T dn = (p[i] - cdel * d1[i] - ceps * d2[i]) * cd;
        d2[i] = dn;
        x[i] += cx * dn;
        if (go_on) {
            t[i] *= ib;
            p[i] = z[i] * ib;
        }
    }
}

// In the spatial eigenbasis: w[plane][k] /= pw_comp (mu_k + shift), the
// inverse of pw (K_x + shift M_x); plane = sys * c + comp
template <typename T>
__global__ void __launch_bounds__(MR_THREADS)
    k_fd_scale(T *__restrict__ w, const T *__restrict__ mu, T shift, T ipw0, T ipw1, int c,
               long long m) {
    const int plane = blockIdx.y;
    const T ipw = (plane % c == 0) ? ipw0 : ipw1;
    T *wp = w + (long long)plane * m;
    for (long long e = (long long)blockIdx.x * MR_THREADS + threadIdx.x; e < m;
         e += (long long)gridDim.x * MR_THREADS)
        wp[e] = ipw * wp[e] / (mu[e] + shift);
}

// dst[sys][comp][:] = scale_comp * src_comp[sys][row_comp][:]  (sources: nt
// planes per slab; component 1 may come from another vector or row)
template <typename T>
__global__ void __launch_bounds__(MR_THREADS)
    k_mr_gather(const T *__restrict__ src0, int row0, const T *__restrict__ src1, int row1,
                T *__restrict__ dst, int c, int nt, long long m, T sc0, T sc1) {
    const int plane = blockIdx.y;
    const int sys = plane / c, comp = plane - sys * c;
    const T sc = comp == 0 ? sc0 : sc1;
    const T *sp = (comp == 0 ? src0 : src1) + ((long long)sys * nt + (comp == 0 ? row0 : row1)) * m;
    T *dp = dst + (long long)plane * m;
    for (long long e = (long long)blockIdx.x * MR_THREADS + threadIdx.x; e < m;
         e += (long long)gridDim.x * MR_THREADS)
        dp[e] = sc * sp[e];
}

// dst_comp[sys][row_comp][:] = sign_comp * src[sys][comp][:]
template <typename T>
__global__ void __launch_bounds__(MR_THREADS)
    k_mr_scatter(const T *__restrict__ src, T *__restrict__ dst0, int row0, T *__restrict__ dst1,
                 int row1, int c, int nt, long long m, T sg0, T sg1) {
    const int plane = blockIdx.y;
    const int sys = plane / c, comp = plane - sys * c;
    const T sg = comp == 0 ? sg0 : sg1;
    const T *sp = src + (long long)plane * m;
    T *dp = (comp == 0 ? dst0 : dst1) + ((long long)sys * nt + (comp == 0 ? row0 : row1)) * m;
    for (long long e = (long long)blockIdx.x * MR_THREADS + threadIdx.x; e < m;
         e += (long long)gridDim.x * MR_THREADS)
        dp[e] = sg * sp[e];
}

// number of systems still iterating
__global__ void k_mr_count(const MrState *__restrict__ st, int nsys, int *__restrict__ out) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int mine = 0;
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) mine += st[s].active ? 1 : 0;
    atomicAdd(&cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) *out = cnt;
}

inline unsigned grid_x(long long len, int cap) {
    long long g = (len + MR_THREADS - 1) / MR_THREADS;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

inline bool grid_y_ok(long long planes) { return planes >= 1 && planes <= 65535; }

}  // namespace

int mr_dot_chunks(long long len) {
    long long c = (len + 4095) / 4096;
    if (c < 1) c = 1;
    if (c > MR_MAX_CHUNKS) c = MR_MAX_CHUNKS;
    return (int)c;
}

template <typename T>
cudaError_t launch_seg_dot(const T *a, const T *b, double *part, long long len, int nsys,
                           cudaStream_t s) {
    if (nsys <= 0 || len <= 0) return cudaSuccess;
    if (!grid_y_ok(nsys)) return cudaErrorInvalidValue;
    dim3 grid((unsigned)mr_dot_chunks(len), (unsigned)nsys);
    k_seg_dot<T><<<grid, MR_THREADS, 0, s>>>(a, b, part, len);
    return cudaGetLastError();
}

cudaError_t launch_mr_init(const double *partB, int chunks, MrState *st, int nsys, cudaStream_t s) {
    if (nsys <= 0) return cudaSuccess;
    k_mr_init<<<(nsys + 127) / 128, 128, 0, s>>>(partB, chunks, st, nsys);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mr_init_vec(T *q, T *p, const T *z, T *qp, T *d1, T *d2, T *x,
                               const MrState *st, long long len, int nsys, cudaStream_t s) {
    if (nsys <= 0 || len <= 0) return cudaSuccess;
    if (!grid_y_ok(nsys)) return cudaErrorInvalidValue;
    dim3 grid(grid_x(len, 64), (unsigned)nsys);
    k_mr_init_vec<T><<<grid, MR_THREADS, 0, s>>>(q, p, z, qp, d1, d2, x, st, len);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mr_lanczos(T *t, const T *q, const T *qp, const double *partA, int chunks,
                              const MrState *st, long long len, int nsys, cudaStream_t s) {
    if (nsys <= 0 || len <= 0) return cudaSuccess;
    if (!grid_y_ok(nsys)) return cudaErrorInvalidValue;
    dim3 grid(grid_x(len, 64), (unsigned)nsys);
    k_mr_lanczos<T><<<grid, MR_THREADS, 0, s>>>(t, q, qp, partA, chunks, st, len);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mr_step(T *p, const T *z, T *t, const T *d1, T *d2, T *x, const double *partA,
                           const double *partB, int chunks, const MrState *st_in, MrState *st_out,
                           double tol, long long len, int nsys, cudaStream_t s) {
    if (nsys <= 0 || len <= 0) return cudaSuccess;
    if (!grid_y_ok(nsys) || st_in == st_out) return cudaErrorInvalidValue;
    dim3 grid(grid_x(len, 64), (unsigned)nsys);
    k_mr_step<T><<<grid, MR_THREADS, 0, s>>>(p, z, t, d1, d2, x, partA, partB, chunks, st_in,
                                             st_out, tol, len);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fd_scale(T *w, const T *mu, double shift, double pw0, double pw1, int c,
                            long long m, int nsys, cudaStream_t s) {
    if (nsys <= 0 || m <= 0) return cudaSuccess;
    if (c < 1 || c > 2 || !grid_y_ok((long long)nsys * c) || !(pw0 > 0) || !(pw1 > 0))
        return cudaErrorInvalidValue;
    dim3 grid(grid_x(m, 64), (unsigned)(nsys * c));
    k_fd_scale<T><<<grid, MR_THREADS, 0, s>>>(w, mu, (T)shift, (T)(1.0 / pw0), (T)(1.0 / pw1), c,
                                              m);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mr_gather(const T *src0, int row0, const T *src1, int row1, T *dst, int c,
                             int nt, long long m, double sc0, double sc1, int nsys,
                             cudaStream_t s) {
    if (nsys <= 0 || m <= 0) return cudaSuccess;
    if (c < 1 || c > 2 || row0 < 0 || row0 >= nt || (c == 2 && (row1 < 0 || row1 >= nt)) ||
        !grid_y_ok((long long)nsys * c))
        return cudaErrorInvalidValue;
    dim3 grid(grid_x(m, 64), (unsigned)(nsys * c));
    k_mr_gather<T><<<grid, MR_THREADS, 0, s>>>(src0, row0, c == 2 ? src1 : src0, row1, dst, c, nt,
                                               m, (T)sc0, (T)sc1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mr_scatter(const T *src, T *dst0, int row0, T *dst1, int row1, int c, int nt,
                              long long m, double sg0, double sg1, int nsys, cudaStream_t s) {
    if (nsys <= 0 || m <= 0) return cudaSuccess;
    if (c < 1 || c > 2 || row0 < 0 || row0 >= nt || (c == 2 && (row1 < 0 || row1 >= nt)) ||
        !grid_y_ok((long long)nsys * c))
        return cudaErrorInvalidValue;
    dim3 grid(grid_x(m, 64), (unsigned)(nsys * c));
    k_mr_scatter<T><<<grid, MR_THREADS, 0, s>>>(src, dst0, row0, c == 2 ? dst1 : dst0, row1, c, nt,
                                                m, (T)sg0, (T)sg1);
    return cudaGetLastError();
}

cudaError_t launch_mr_count(const MrState *st, int nsys, int *count, cudaStream_t s) {
    k_mr_count<<<1, 256, 0, s>>>(st, nsys, count);
    return cudaGetLastError();
}

#define ST_MR_INST(T)                                                                           \
    template cudaError_t launch_seg_dot<T>(const T *, const T *, double *, long long, int,       \
                                           cudaStream_t);                                       \
    template cudaError_t launch_mr_init_vec<T>(T *, T *, const T *, T *, T *, T *, T *,          \
                                               const MrState *, long long, int, cudaStream_t);  \
    template cudaError_t launch_mr_lanczos<T>(T *, const T *, const T *, const double *, int,    \
                                              const MrState *, long long, int, cudaStream_t);   \
    template cudaError_t launch_mr_step<T>(T *, const T *, T *, const T *, T *, T *,             \
                                           const double *, const double *, int, const MrState *, \
                                           MrState *, double, long long, int, cudaStream_t);    \
    template cudaError_t launch_fd_scale<T>(T *, const T *, double, double, double, int,         \
                                            long long, int, cudaStream_t);                      \
    template cudaError_t launch_mr_gather<T>(const T *, int, const T *, int, T *, int, int,      \
                                             long long, double, double, int, cudaStream_t);     \
    template cudaError_t launch_mr_scatter<T>(const T *, T *, int, T *, int, int, int, long long, \
                                              double, double, int, cudaStream_t);
ST_MR_INST(double)
ST_MR_INST(float)
#undef ST_MR_INST

}  // namespace st

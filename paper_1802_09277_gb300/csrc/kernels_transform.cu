// Slab-inverse pieces of the damped block-Jacobi smoother (Sec. 3.1-3.5 of
// arXiv:1802.09277) and the time-multigrid transfers, CUDA-core versions
// (FP64 and FP32).
//
// A^{-1} = (X (x) U) (Z (x) I + I (x) Lambda)^{-1} (Y (x) U^T)   (Eq. 3.1 with
// the spatial problems diagonalised: U^T M_x U = I, U^T K_x U = Lambda)
//
//  * strided GEMM      : one mode product with U^T (forward) or U (inverse)
//                        along one spatial axis, batched over the others
//  * shift solve       : per spatial mode k, (Z + mu_k I) z = w by back
//                        substitution over the quasi-triangular real Schur
//                        factor (Algorithm 1 in the eigenbasis, 2x2 blocks
//                        solved in closed form, Sec. 3.5)
//  * update            : u += omega X z (backward time transform + damping)
//  * restrict/prolong  : R = P^T, P = P_t (x) I on slab pairs (Sec. 3.1)
#include "st_internal.h"

namespace st {

// ---------------------------------------------------------------------------
// Strided batched GEMM (SIMT), 64x64 tiles, 16-deep k slices, 4x4 per thread
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16;

template <typename T>
__global__ void __launch_bounds__(256)
    k_gemm_strided(int M, int N, int K, int tiles_m, int tiles_n, const T *__restrict__ A,
                   long long sAb, long long sAm, long long sAk, const T *__restrict__ B,
                   long long sBb, long long sBk, long long sBn, T *__restrict__ C, long long sCb,
                   long long sCm, long long sCn) {
    __shared__ T As[GBK][GBM + 1];
    __shared__ T Bs[GBK][GBN + 1];
    const long long t = blockIdx.x;
    const int tn_i = (int)(t % tiles_n);
    const int tm_i = (int)((t / tiles_n) % tiles_m);
    const long long b = t / ((long long)tiles_n * tiles_m);
    const int m0 = tm_i * GBM, n0 = tn_i * GBN;
    A += b * sAb;
    B += b * sBb;
    C += b * sCb;
    const int tid = threadIdx.x;
    const int tm = tid / 16, tn = tid % 16;
    T c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[i][j] = T(0);
    const bool a_krow = (sAk == 1);
    const bool b_nrow = (sBn == 1);
    for (int k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            int m, k;
            if (a_krow) {
                m = e / GBK;
                k = e % GBK;
            } else {
                m = e % GBM;
                k = e / GBM;
            }
            const int gm = m0 + m, gk = k0 + k;
            As[k][m] = (gm < M && gk < K) ? A[gm * sAm + gk * sAk] : T(0);
            int kb, n;
            if (b_nrow) {
                kb = e / GBN;
                n = e % GBN;
            } else {
                kb = e % GBK;
                n = e / GBK;
            }
            const int gn = n0 + n, gkb = k0 + kb;
            Bs[kb][n] = (gn < N && gkb < K) ? B[gkb * sBk + gn * sBn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tn + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) c[i][j] += a[i] * bb[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tm + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tn + 16 * j;
            if (gn < N) C[gm * sCm + gn * sCn] = c[i][j];
        }
    }
}

template <typename T>
cudaError_t launch_gemm_strided(int batch, int M, int N, int K, const T *A, long long sAb,
                                long long sAm, long long sAk, const T *B, long long sBb,
                                long long sBk, long long sBn, T *C, long long sCb, long long sCm,
                                long long sCn, cudaStream_t s) {
    const int tm = (M + GBM - 1) / GBM, tn = (N + GBN - 1) / GBN;
    const long long blocks = (long long)tm * tn * batch;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_gemm_strided<T><<<(unsigned)blocks, 256, 0, s>>>(M, N, K, tm, tn, A, sAb, sAm, sAk, B, sBb,
                                                       sBk, sBn, C, sCb, sCm, sCn);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shift solve in the spatial eigenbasis
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_shift_solve(T *__restrict__ w, const T *__restrict__ lam0,
                              const T *__restrict__ lam1, const T *__restrict__ lam2, Grid g,
                              const __grid_constant__ SchurCoefs<T> sc, long long nslabs) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = nslabs * g.nxyz;
    if (idx >= total) return;
    const long long slab = idx / g.nxyz, k = idx % g.nxyz;
    const int kx = (int)(k % g.nx), ky = (int)((k / g.nx) % g.ny), kz = (int)(k / ((long long)g.nx * g.ny));
    T mu = lam0[kx];
    if (g.dim >= 2) mu += lam1[ky];
    if (g.dim >= 3) mu += lam2[kz];
    const int nt = sc.nt;
    T *base = w + slab * nt * g.nxyz + k;
    T r[NTMAX], z[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        r[i] = (i < nt) ? base[(long long)i * g.nxyz] : T(0);
        z[i] = T(0);
    }
    bool skip = false;
#pragma unroll
    for (int i = NTMAX - 1; i >= 0; --i) {
        if (i >= nt) continue;
        if (skip) {
            skip = false;
            continue;
        }
        if (i >= 1 && sc.blk[i]) {  // 2x2 block on rows i-1, i
            T g1 = r[i - 1], g2 = r[i];
#pragma unroll
            for (int j = i + 1; j < NTMAX; ++j)
                if (j < nt) {
                    g1 -= sc.Z[(i - 1) * NTMAX + j] * z[j];
                    g2 -= sc.Z[i * NTMAX + j] * z[j];
                }
            const T a = sc.Z[(i - 1) * NTMAX + i - 1] + mu, b = sc.Z[(i - 1) * NTMAX + i];
            const T c = sc.Z[i * NTMAX + i - 1], d = sc.Z[i * NTMAX + i] + mu;
            const T det = a * d - b * c;
            z[i - 1] = (d * g1 - b * g2) / det;
            z[i] = (a * g2 - c * g1) / det;
            skip = true;
        } else {
            T gg = r[i];
#pragma unroll
            for (int j = i + 1; j < NTMAX; ++j)
                if (j < nt) gg -= sc.Z[i * NTMAX + j] * z[j];
            z[i] = gg / (sc.Z[i * NTMAX + i] + mu);
        }
    }
#pragma unroll
    for (int i = 0; i < NTMAX; ++i)
        if (i < nt) base[(long long)i * g.nxyz] = z[i];
}

template <typename T>
cudaError_t launch_shift_solve(T *w, const T *lam0, const T *lam1, const T *lam2, const Grid &g,
                               const SchurCoefs<T> &sc, long long nslabs, cudaStream_t s) {
    const long long total = nslabs * g.nxyz;
    if (total <= 0) return cudaSuccess;
    const int bs = 256;
    k_shift_solve<T><<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(w, lam0, lam1, lam2, g, sc,
                                                                     nslabs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// u (+)= omega X z  (backward time transform fused with the damped update)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_update(T *__restrict__ u, const T *__restrict__ z,
                         const __grid_constant__ SchurCoefs<T> sc, T omega, long long nxyz,
                         long long nslabs, int overwrite) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nslabs * nxyz) return;
    const long long slab = idx / nxyz, k = idx % nxyz;
    const int nt = sc.nt;
    const long long base = slab * nt * nxyz + k;
    T zz[NTMAX];
#pragma unroll
    for (int j = 0; j < NTMAX; ++j) zz[j] = (j < nt) ? z[base + (long long)j * nxyz] : T(0);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        if (i >= nt) break;
        T v = T(0);
#pragma unroll
        for (int j = 0; j < NTMAX; ++j)
            if (j < nt) v += sc.X[i * NTMAX + j] * zz[j];
        const long long o = base + (long long)i * nxyz;
        u[o] = overwrite ? omega * v : u[o] + omega * v;
    }
}

// y += x (the space prolongation's correction)
template <typename T>
__global__ void k_add(T *__restrict__ y, const T *__restrict__ x, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

template <typename T>
cudaError_t launch_add(T *y, const T *x, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_add<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, x, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(T *u, const T *z, const SchurCoefs<T> &sc, T omega, const Grid &g,
                          long long nslabs, int overwrite, cudaStream_t s) {
    const long long total = nslabs * g.nxyz;
    if (total <= 0) return cudaSuccess;
    const int bs = 256;
    k_update<T><<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(u, z, sc, omega, g.nxyz, nslabs,
                                                                overwrite);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Time transfers between slab pairs and their merged coarse slab
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_restrict(const T *__restrict__ rf, T *__restrict__ fc,
                           const __grid_constant__ ProlongCoefs<T> pc, long long nxyz,
                           long long ncoarse) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncoarse * nxyz) return;
    const long long m = idx / nxyz, k = idx % nxyz;
    const int nt = pc.nt;
    T r[2 * NTMAX];
#pragma unroll
    for (int j = 0; j < 2 * NTMAX; ++j) {
        const int q = j / NTMAX, jj = j % NTMAX;
        r[j] = (jj < nt) ? rf[((2 * m + q) * nt + jj) * nxyz + k] : T(0);
    }
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        if (i >= nt) break;
        T v = T(0);
#pragma unroll
        for (int j = 0; j < 2 * NTMAX; ++j) {
            const int q = j / NTMAX, jj = j % NTMAX;
            if (jj < nt) v += pc.P[((q * nt) + jj) * NTMAX + i] * r[j];
        }
        fc[(m * nt + i) * nxyz + k] = v;
    }
}

template <typename T>
__global__ void k_prolong_add(const T *__restrict__ ec, T *__restrict__ uf,
                              const __grid_constant__ ProlongCoefs<T> pc, long long nxyz,
                              long long ncoarse) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncoarse * nxyz) return;
    const long long m = idx / nxyz, k = idx % nxyz;
    const int nt = pc.nt;
    T e[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) e[i] = (i < nt) ? ec[(m * nt + i) * nxyz + k] : T(0);
#pragma unroll
    for (int j = 0; j < 2 * NTMAX; ++j) {
        const int q = j / NTMAX, jj = j % NTMAX;
        if (jj >= nt) continue;
        T v = T(0);
#pragma unroll
        for (int i = 0; i < NTMAX; ++i)
            if (i < nt) v += pc.P[((q * nt) + jj) * NTMAX + i] * e[i];
        const long long o = ((2 * m + q) * nt + jj) * nxyz + k;
        uf[o] += v;
    }
}

template <typename T>
cudaError_t launch_restrict(const T *rf, T *fc, const ProlongCoefs<T> &pc, const Grid &g,
                            long long ncoarse, cudaStream_t s) {
    const long long total = ncoarse * g.nxyz;
    if (total <= 0) return cudaSuccess;
    k_restrict<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(rf, fc, pc, g.nxyz, ncoarse);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const T *ec, T *uf, const ProlongCoefs<T> &pc, const Grid &g,
                               long long ncoarse, cudaStream_t s) {
    const long long total = ncoarse * g.nxyz;
    if (total <= 0) return cudaSuccess;
    k_prolong_add<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ec, uf, pc, g.nxyz, ncoarse);
    return cudaGetLastError();
}

#define ST_INST(T)                                                                              \
    template cudaError_t launch_gemm_strided<T>(int, int, int, int, const T *, long long,       \
                                                long long, long long, const T *, long long,     \
                                                long long, long long, T *, long long, long long, \
                                                long long, cudaStream_t);                       \
    template cudaError_t launch_shift_solve<T>(T *, const T *, const T *, const T *,            \
                                               const Grid &, const SchurCoefs<T> &, long long,  \
                                               cudaStream_t);                                   \
    template cudaError_t launch_update<T>(T *, const T *, const SchurCoefs<T> &, T, const Grid &, \
                                          long long, int, cudaStream_t);                        \
    template cudaError_t launch_restrict<T>(const T *, T *, const ProlongCoefs<T> &,            \
                                            const Grid &, long long, cudaStream_t);             \
    template cudaError_t launch_prolong_add<T>(const T *, T *, const ProlongCoefs<T> &,         \
                                               const Grid &, long long, cudaStream_t);         \
    template cudaError_t launch_add<T>(T *, const T *, long long, cudaStream_t);
ST_INST(double)
ST_INST(float)
#undef ST_INST

}  // namespace st

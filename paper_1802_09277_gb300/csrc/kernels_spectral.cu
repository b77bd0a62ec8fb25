// The time-multigrid V-cycle in the spatial eigenbasis (arXiv:1802.09277,
// Sec. 3.1 smoother with A_n^{-1} from Eq. 3.1).
//
// With U^T M_x U = I and U^T K_x U = Lambda (U = U_z (x) U_y (x) U_x) the
// slab operator becomes A^ = K_t (x) I + M_t (x) Lambda and the coupling
// B^ = N_t (x) I: every spatial mode k (shift mu_k = sum over axes of the 1D
// eigenvalues) carries an independent block lower-bidiagonal time problem
// with diagonal blocks K_t + mu_k M_t = Y^{-1} (Z + mu_k I) X^{-1}.  Time
// coarsening (P = P_t (x) I) and block Jacobi commute with the spatial
// transform, so the V-cycle of the original basis equals
// (I (x) U) V^(r^) with r^ = (I (x) U^T) r.
//
// This file: the per-mode block solve of the B-spline-basis smoother in the
// diagonalisation variant (k_mode_solve) and the whole eigenbasis V-cycle in
// one shared-memory kernel (k_spec_vcycle, opt.fused_vcycle).  The level-wise
// eigenbasis kernels are in kernels_modes.cu.
#include <cstring>

#include "spec_common.cuh"

namespace st {

template <typename T>
__global__ void __launch_bounds__(256)
    k_mode_solve(T *__restrict__ w, const T *__restrict__ mu_tab, Grid g, const __grid_constant__ SpecCoefs<T> c,
                 long long nslabs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long slab = slab_index();
    if (k >= g.nxyz || slab >= nslabs) return;
    const int nt = c.nt;
    const long long base = slab * nt * g.nxyz + k;
    const T mu = mu_tab[k];
    T r[NTMAX], v[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) r[i] = (i < nt) ? w[base + (long long)i * g.nxyz] : T(0);
    spec_block_solve(c, mu, r, v);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i)
        if (i < nt) w[base + (long long)i * g.nxyz] = v[i];
}

template <typename T>
cudaError_t launch_mode_solve(T *w, const T *mu, const Grid &g, const SpecCoefs<T> &c,
                              long long nslabs, cudaStream_t s) {
    if (nslabs <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, nslabs);
    k_mode_solve<T><<<L.grid, L.block, 0, s>>>(w, mu, g,
                                                                    c, nslabs);
    return cudaGetLastError();
}

// The eigenbasis operator L^ = blockbidiag(K_t + mu M_t, -N_t):
// res = 1: out = f - L^ u, else out = L^ u  (pointwise per (slab, mode))
// ---------------------------------------------------------------------------
// The whole eigenbasis V-cycle in shared memory.  CTA (problem r, mode block
// b) owns modes k0 .. k0 + MB - 1 of problem r on every slab of every level:
// per level l it keeps u_l and f_l as [nt][N_l][MB] (mode fastest, so a
// warp's 32 consecutive (slab, mode) items hit 32 consecutive words), plus
// one level-0 sized scratch array for the out-of-place Jacobi steps.  All
// levels' time coefficients arrive as one __grid_constant__ parameter block
// (constant-bank operands).  HBM is touched twice: f^ read once, u^ written
// once.  The steps of the level-wise V-cycle (kernels_modes.cu), with the
// Schur-form block solve in place of the per-mode inverses.
// ---------------------------------------------------------------------------
template <typename T>
struct FusedParams {
    // levels that fit the 32 KB kernel-parameter space
    static constexpr int LMAX = sizeof(T) == 4 ? 12 : 6;
    SpecCoefs<T> lv[LMAX];
    ProlongCoefs<T> pc;
};

template <typename T>
__global__ void __launch_bounds__(256)
    k_spec_vcycle(const T *__restrict__ fin, T *__restrict__ uout,
                  const __grid_constant__ FusedParams<T> P, const T *__restrict__ mu_tab, Grid g, int nlev, int N,
                  int MB, int nu1, int nu2, T omega) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int nt = P.pc.nt;
    const long long nmodes = g.nxyz;
    const int nblk = (int)((nmodes + MB - 1) / MB);
    const int r = blockIdx.x / nblk;
    const long long k0 = (long long)(blockIdx.x % nblk) * MB;
    const int tid = threadIdx.x, NTH = blockDim.x;
    // layout: mu[MB] | U_0 F_0 U_1 F_1 ... | TMP, each [nt][N_l][MB]
    T *mu = sm;
    T *lev = sm + MB;
    auto U = [&](int l) {
        long long off = 0;
        for (int q = 0; q < l; ++q) off += 2LL * (N >> q) * nt * MB;
        return lev + off;
    };
    auto F = [&](int l) { return U(l) + (long long)(N >> l) * nt * MB; };
    T *TMP = U(nlev);
    // element (i, n, kk) of a level with Nl slabs
#define SV_IDX(i, n, kk, Nl) (((long long)(i) * (Nl) + (n)) * MB + (kk))
    for (int kk = tid; kk < MB; kk += NTH)
        mu[kk] = (k0 + kk < nmodes) ? mu_tab[k0 + kk] : T(0);
    {  // load f^ of this problem's mode block
        T *F0 = F(0);
        const long long base = (long long)r * N * nt * nmodes;
        for (long long e = tid; e < (long long)N * nt * MB; e += NTH) {
            const long long row = e / MB;  // n * nt + i in global order
            const int kk = (int)(e % MB), n = (int)(row / nt), i = (int)(row % nt);
            F0[SV_IDX(i, n, kk, N)] = (k0 + kk < nmodes) ? fin[base + row * nmodes + k0 + kk] : T(0);
        }
    }
    __syncthreads();

    // one damped block-Jacobi step on level l: TMP = smooth(u), then u = TMP
    auto smooth = [&](int l, bool zero) {
        const SpecCoefs<T> &c = P.lv[l];
        const int Nl = N >> l;
        T *u = U(l);
        const T *f = F(l);
        for (int it = tid; it < Nl * MB; it += NTH) {
            const int n = it / MB, kk = it % MB;
            T uu[NTMAX], rr[NTMAX], v[NTMAX];
#pragma unroll
            for (int i = 0; i < NTMAX; ++i) {
                uu[i] = (i < nt && !zero) ? u[SV_IDX(i, n, kk, Nl)] : T(0);
                rr[i] = (i < nt) ? f[SV_IDX(i, n, kk, Nl)] : T(0);
            }
            const T up = (!zero && n > 0) ? u[SV_IDX(nt - 1, n - 1, kk, Nl)] : T(0);
            spec_residual(c, mu[kk], uu, up, rr);
            spec_block_solve(c, mu[kk], rr, v);
#pragma unroll
            for (int i = 0; i < NTMAX; ++i)
                if (i < nt) TMP[SV_IDX(i, n, kk, Nl)] = uu[i] + omega * v[i];
        }
        __syncthreads();
        for (long long e = tid; e < (long long)Nl * nt * MB; e += NTH) u[e] = TMP[e];
        __syncthreads();
    };

    for (int l = 0; l < nlev - 1; ++l) {
        for (int sidx = 0; sidx < nu1; ++sidx) smooth(l, sidx == 0);
        if (nu1 == 0)
            for (long long e = tid; e < (long long)(N >> l) * nt * MB; e += NTH) U(l)[e] = T(0);
        __syncthreads();
        // residual of slab pairs, restricted to level l + 1
        const SpecCoefs<T> &c = P.lv[l];
        const int Nl = N >> l, Nc = N >> (l + 1);
        const T *u = U(l), *f = F(l);
        T *fc = F(l + 1), *uc = U(l + 1);
        for (int it = tid; it < Nc * MB; it += NTH) {
            const int m = it / MB, kk = it % MB, a = 2 * m;
            T ua[NTMAX], ub[NTMAX], ra[NTMAX], rb[NTMAX];
#pragma unroll
            for (int i = 0; i < NTMAX; ++i) {
                const bool in = i < nt;
                ua[i] = in ? u[SV_IDX(i, a, kk, Nl)] : T(0);
                ub[i] = in ? u[SV_IDX(i, a + 1, kk, Nl)] : T(0);
                ra[i] = in ? f[SV_IDX(i, a, kk, Nl)] : T(0);
                rb[i] = in ? f[SV_IDX(i, a + 1, kk, Nl)] : T(0);
            }
            const T up = (a > 0) ? u[SV_IDX(nt - 1, a - 1, kk, Nl)] : T(0);
            T ualast = T(0);
            ualast = last_of(ua, nt);
            spec_residual(c, mu[kk], ua, up, ra);
            spec_residual(c, mu[kk], ub, ualast, rb);
#pragma unroll
            for (int i = 0; i < NTMAX; ++i) {
                if (i >= nt) break;
                T sacc = T(0);
#pragma unroll
                for (int j = 0; j < NTMAX; ++j)
                    if (j < nt)
                        sacc += P.pc.P[j * NTMAX + i] * ra[j] + P.pc.P[(nt + j) * NTMAX + i] * rb[j];
                fc[SV_IDX(i, m, kk, Nc)] = sacc;
                uc[SV_IDX(i, m, kk, Nc)] = T(0);
            }
        }
        __syncthreads();
    }
    {  // coarsest level: exact forward substitution over its slabs, per mode
        const int l = nlev - 1, Nl = N >> l;
        const SpecCoefs<T> &c = P.lv[l];
        T *u = U(l);
        const T *f = F(l);
        for (int kk = tid; kk < MB; kk += NTH) {
            T prev = T(0);
            for (int n = 0; n < Nl; ++n) {
                T rr[NTMAX], v[NTMAX];
#pragma unroll
                for (int i = 0; i < NTMAX; ++i) rr[i] = (i < nt) ? f[SV_IDX(i, n, kk, Nl)] : T(0);
                rr[0] += prev;
                spec_block_solve(c, mu[kk], rr, v);
#pragma unroll
                for (int i = 0; i < NTMAX; ++i)
                    if (i < nt) u[SV_IDX(i, n, kk, Nl)] = v[i];
                prev = last_of(v, nt);
            }
        }
        __syncthreads();
    }
    for (int l = nlev - 2; l >= 0; --l) {
        // prolongation of the coarse correction
        const int Nl = N >> l, Nc = N >> (l + 1);
        T *u = U(l);
        const T *uc = U(l + 1);
        for (int it = tid; it < Nc * MB; it += NTH) {
            const int m = it / MB, kk = it % MB;
            T e[NTMAX];
#pragma unroll
            for (int i = 0; i < NTMAX; ++i) e[i] = (i < nt) ? uc[SV_IDX(i, m, kk, Nc)] : T(0);
#pragma unroll
            for (int j = 0; j < 2 * NTMAX; ++j) {
                const int q = j / NTMAX, jj = j % NTMAX;
                if (jj >= nt) continue;
                T sacc = T(0);
#pragma unroll
                for (int i = 0; i < NTMAX; ++i)
                    if (i < nt) sacc += P.pc.P[((q * nt) + jj) * NTMAX + i] * e[i];
                u[SV_IDX(jj, 2 * m + q, kk, Nl)] += sacc;
            }
        }
        __syncthreads();
        for (int sidx = 0; sidx < nu2; ++sidx) smooth(l, false);
    }
    {  // store u^
        const T *U0 = U(0);
        const long long base = (long long)r * N * nt * nmodes;
        for (long long e = tid; e < (long long)N * nt * MB; e += NTH) {
            const long long row = e / MB;
            const int kk = (int)(e % MB), n = (int)(row / nt), i = (int)(row % nt);
            if (k0 + kk < nmodes) uout[base + row * nmodes + k0 + kk] = U0[SV_IDX(i, n, kk, N)];
        }
    }
#undef SV_IDX
}

// Shared memory (elements) of k_spec_vcycle for a mode block of MB modes.
static long long spec_vcycle_elems(int nlev, int N, int nt, int MB) {
    long long e = MB;
    for (int l = 0; l < nlev; ++l) e += 2LL * (N >> l) * nt * MB;
    return e + (long long)N * nt * MB;
}

template <typename T>
cudaError_t launch_spec_vcycle(const T *fin, T *uout, const SpecCoefs<T> *lvc_host,
                               const T *mu, const Grid &g, const ProlongCoefs<T> &pc,
                               int nlev, int N, int nrhs, int nu1, int nu2, T omega, int max_smem,
                               int nsm, cudaStream_t s) {
    if (nlev > FusedParams<T>::LMAX) return cudaErrorNotSupported;
    // the mode block: at most 32 modes, small enough for two CTAs per SM
    // when there are enough blocks to fill the GPU
    int MB = 32;
    const long long cap2 = (long long)(max_smem / 2 - 1024);
    while (MB > 1 && (spec_vcycle_elems(nlev, N, pc.nt, MB) * (long long)sizeof(T) > cap2 ||
                      (g.nxyz + MB - 1) / MB * nrhs < 2LL * nsm))
        MB /= 2;
    long long bytes = spec_vcycle_elems(nlev, N, pc.nt, MB) * (long long)sizeof(T);
    if (bytes > max_smem) return cudaErrorNotSupported;
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e = smem_attr_once((const void *)k_spec_vcycle<T>, max_smem, attr);
        if (e != cudaSuccess) return e;
    }
    FusedParams<T> P;
    memset(&P, 0, sizeof P);
    for (int l = 0; l < nlev; ++l) P.lv[l] = lvc_host[l];
    P.pc = pc;
    const long long nblk = (g.nxyz + MB - 1) / MB;
    const long long grid = nblk * nrhs;
    if (grid <= 0) return cudaSuccess;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_spec_vcycle<T><<<(unsigned)grid, 256, (size_t)bytes, s>>>(fin, uout, P, mu,
                                                               g, nlev, N, MB, nu1, nu2, omega);
    return cudaGetLastError();
}

// grid over (problem, mode); sequential over the level's slabs
#define ST_INST(T)                                                                             \
    template cudaError_t launch_mode_solve<T>(T *, const T *, const Grid &,                     \
                                              const SpecCoefs<T> &, long long, cudaStream_t);     \
    template cudaError_t launch_spec_vcycle<T>(const T *, T *, const SpecCoefs<T> *,            \
                                               const T *, const Grid &,                         \
                                               const ProlongCoefs<T> &, int, int, int, int, int, \
                                               T, int, int, cudaStream_t);
ST_INST(double)
ST_INST(float)
#undef ST_INST

}  // namespace st

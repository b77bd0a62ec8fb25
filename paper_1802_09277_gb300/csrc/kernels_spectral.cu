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
// (I (x) U) V^(r^) with r^ = (I (x) U^T) r.  Here every kernel is pointwise in
// the spatial mode; one thread owns one (slab, mode) pair and its N_t
// coefficients, reading them with stride nxyz (coalesced across threads).
//
//  k_spec_smooth        one damped block-Jacobi step, out-of-place (Jacobi:
//                       every slab sees the previous iterate of its
//                       predecessor): r = f - A^ u + B^ u_prev,
//                       u_out = u + omega X (Z + mu I)^{-1} Y r
//  k_spec_res_restrict  residual of two fine slabs and their restriction
//                       P_t^T onto the merged coarse slab
//  k_spec_down          the last pre-smoothing step, the residual and its
//                       restriction in one pass
//  k_spec_up            prolongation of the coarse correction and the first
//                       post-smoothing step in one pass
//  k_spec_coarse        exact solve of a level by forward substitution over
//                       its slabs: u_n = A^{-1} (f_n + B^ u_{n-1})
#include <cstring>

#include "st_internal.h"

namespace st {

// r = f - (Kt + mu Mt) u + e_0 uprev  (in place into f's copy)
template <typename T>
__device__ __forceinline__ void spec_residual(const SpecCoefs<T> &c, T mu, const T *u, T uprev,
                                              T *r) {
    const int nt = c.nt;
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        if (i >= nt) break;
        T a = r[i];
#pragma unroll
        for (int j = 0; j < NTMAX; ++j)
            if (j < nt) a -= (c.Kt[i * NTMAX + j] + mu * c.Mt[i * NTMAX + j]) * u[j];
        if (i == 0) a += uprev;
        r[i] = a;
    }
}

// 1 / x for the divisions of the block solve: the quotient becomes a
// reciprocal and a multiply (two roundings instead of one); in FP32 the
// correctly rounded reciprocal intrinsic avoids the longer IEEE division
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// v = X (Z + mu I)^{-1} Y r  =  (K_t + mu M_t)^{-1} r   (Eq. 3.1 per mode)
template <typename T>
__device__ __forceinline__ void spec_block_solve(const SpecCoefs<T> &c, T mu, const T *r, T *v) {
    const int nt = c.nt;
    if (c.variant == 1) {  // diagonalisation (Sec. 3.3): complex shifts lambda_i + mu
        T zr[NTMAX], zi[NTMAX];
#pragma unroll
        for (int i = 0; i < NTMAX; ++i) {
            T ar = T(0), ai = T(0);
#pragma unroll
            for (int j = 0; j < NTMAX; ++j)
                if (j < nt) {
                    ar += c.Y[i * NTMAX + j] * r[j];
                    ai += c.Yi[i * NTMAX + j] * r[j];
                }
            const T dr = c.lre[i] + mu, di = c.lim[i];
            const T den = dr * dr + di * di;
            const T rden = recip(den);
            zr[i] = (i < nt) ? (ar * dr + ai * di) * rden : T(0);
            zi[i] = (i < nt) ? (ai * dr - ar * di) * rden : T(0);
        }
#pragma unroll
        for (int i = 0; i < NTMAX; ++i) {
            T a = T(0);
#pragma unroll
            for (int j = 0; j < NTMAX; ++j)
                if (j < nt) a += c.X[i * NTMAX + j] * zr[j] - c.Xi[i * NTMAX + j] * zi[j];
            v[i] = a;
        }
        return;
    }
    T w[NTMAX], z[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        T a = T(0);
#pragma unroll
        for (int j = 0; j < NTMAX; ++j)
            if (j < nt) a += c.Y[i * NTMAX + j] * r[j];
        w[i] = a;
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
        if (i >= 1 && c.blk[i]) {
            T g1 = w[i - 1], g2 = w[i];
#pragma unroll
            for (int j = i + 1; j < NTMAX; ++j)
                if (j < nt) {
                    g1 -= c.Z[(i - 1) * NTMAX + j] * z[j];
                    g2 -= c.Z[i * NTMAX + j] * z[j];
                }
            const T a = c.Z[(i - 1) * NTMAX + i - 1] + mu, b = c.Z[(i - 1) * NTMAX + i];
            const T cc = c.Z[i * NTMAX + i - 1], d = c.Z[i * NTMAX + i] + mu;
            const T rdet = recip(a * d - b * cc);
            z[i - 1] = (d * g1 - b * g2) * rdet;
            z[i] = (a * g2 - cc * g1) * rdet;
            skip = true;
        } else {
            T gg = w[i];
#pragma unroll
            for (int j = i + 1; j < NTMAX; ++j)
                if (j < nt) gg -= c.Z[i * NTMAX + j] * z[j];
            z[i] = gg * recip(c.Z[i * NTMAX + i] + mu);
        }
    }
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        T a = T(0);
#pragma unroll
        for (int j = 0; j < NTMAX; ++j)
            if (j < nt) a += c.X[i * NTMAX + j] * z[j];
        v[i] = a;
    }
}

// a[nt - 1] without a run-time index (a select loop over a register array
// can be rewritten into an indexed load, which moves the array to local
// memory; the masked sum keeps every access static)
template <typename T>
__device__ __forceinline__ T last_of(const T *a, int nt) {
    T x = T(0);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) x = fma(a[i], (i == nt - 1) ? T(1) : T(0), x);
    return x;
}

// One thread per spatial mode k (x) and slab or slab pair (y, z: slab =
// z * gridDim.y + y): no integer division in the index arithmetic.
__device__ __forceinline__ long long slab_index() {
    return (long long)blockIdx.z * gridDim.y + blockIdx.y;
}

struct ModeLaunch {
    dim3 grid, block;
};

static ModeLaunch mode_launch(long long nmodes, long long nslabs) {
    ModeLaunch L;
    const int th = nmodes >= 256 ? 256 : (int)((nmodes + 31) / 32 * 32);
    L.block = dim3((unsigned)th);
    const long long gy = nslabs < 65535 ? nslabs : 65535;
    L.grid = dim3((unsigned)((nmodes + th - 1) / th), (unsigned)gy,
                  (unsigned)((nslabs + gy - 1) / gy));
    return L;
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_spec_smooth(const T *__restrict__ uin, T *__restrict__ uout, const T *__restrict__ f,
                  const T *__restrict__ mu_tab, Grid g, const __grid_constant__ SpecCoefs<T> c,
                  T omega, int slabs_per_prob, long long nslabs, int uin_zero) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long slab = slab_index();
    if (k >= g.nxyz || slab >= nslabs) return;
    const int nt = c.nt;
    const long long base = slab * nt * g.nxyz + k;
    const T mu = mu_tab[k];
    T u[NTMAX], r[NTMAX], v[NTMAX];
    T uprev = T(0);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        u[i] = (i < nt && !uin_zero) ? uin[base + (long long)i * g.nxyz] : T(0);
        r[i] = (i < nt) ? f[base + (long long)i * g.nxyz] : T(0);
    }
    if (!uin_zero && (slab % slabs_per_prob) != 0) uprev = uin[base - g.nxyz];
    spec_residual(c, mu, u, uprev, r);
    spec_block_solve(c, mu, r, v);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i)
        if (i < nt) uout[base + (long long)i * g.nxyz] = u[i] + omega * v[i];
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_spec_res_restrict(const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ fc,
                        const T *__restrict__ mu_tab, Grid g, const __grid_constant__ SpecCoefs<T> c,
                        const __grid_constant__ ProlongCoefs<T> pc, int slabs_per_prob,
                        long long ncoarse) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long m = slab_index();
    if (k >= g.nxyz || m >= ncoarse) return;
    const int nt = c.nt;
    const T mu = mu_tab[k];
    const long long a = 2 * m;  // first fine slab (same problem as a + 1)
    const long long ba = a * nt * g.nxyz + k, bb = ba + (long long)nt * g.nxyz;
    T ua[NTMAX], ub[NTMAX], ra[NTMAX], rb[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        const bool in = i < nt;
        ua[i] = in ? u[ba + (long long)i * g.nxyz] : T(0);
        ub[i] = in ? u[bb + (long long)i * g.nxyz] : T(0);
        ra[i] = in ? f[ba + (long long)i * g.nxyz] : T(0);
        rb[i] = in ? f[bb + (long long)i * g.nxyz] : T(0);
    }
    const T uprev = ((a % slabs_per_prob) != 0) ? u[ba - g.nxyz] : T(0);
    T ua_last = T(0);
    ua_last = last_of(ua, nt);
    spec_residual(c, mu, ua, uprev, ra);
    spec_residual(c, mu, ub, ua_last, rb);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        if (i >= nt) break;
        T s = T(0);
#pragma unroll
        for (int j = 0; j < NTMAX; ++j)
            if (j < nt) s += pc.P[j * NTMAX + i] * ra[j] + pc.P[(nt + j) * NTMAX + i] * rb[j];
        fc[(m * nt + i) * g.nxyz + k] = s;
    }
}

// Last pre-smoothing step fused with the residual and its restriction: one
// thread per (coarse slab m, mode k) takes the fine slabs a = 2m, b = 2m + 1.
// Jacobi: the smoothed slabs see their predecessors' OLD iterates; the
// residual of the smoothed iterate needs the NEW last entry of slab a - 1,
// which the thread recomputes (one more block solve instead of a pass over
// HBM).  ZERO: the incoming iterate is zero (uin not read), so the step is
// u = omega A^{-1} f.  Writes the smoothed slabs to uout and P_t^T r to fc.
template <typename T, bool ZERO>
__global__ void __launch_bounds__(256)
    k_spec_down(const T *__restrict__ uin, T *__restrict__ uout, const T *__restrict__ f,
                T *__restrict__ fc, const T *__restrict__ mu_tab, Grid g, const __grid_constant__ SpecCoefs<T> c,
                const __grid_constant__ ProlongCoefs<T> pc, T omega, int slabs_per_prob,
                long long ncoarse) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long m = slab_index(), S = g.nxyz;
    if (k >= S || m >= ncoarse) return;
    const int nt = c.nt;
    const T mu = mu_tab[k];
    const long long a = 2 * m;
    const bool first = (a % slabs_per_prob) == 0;
    const long long ba = a * nt * S + k, bb = ba + (long long)nt * S;
    T v[NTMAX];
    // new last entry of slab a - 1 (and its old one, seen by slab a's step)
    T new_prev = T(0), old_prev = T(0);
    if (!first) {
        const long long bp = ba - (long long)nt * S;
        T r[NTMAX], u[NTMAX];
#pragma unroll
        for (int i = 0; i < NTMAX; ++i) {
            r[i] = (i < nt) ? f[bp + (long long)i * S] : T(0);
            u[i] = (i < nt && !ZERO) ? uin[bp + (long long)i * S] : T(0);
        }
        if (!ZERO) {
            const T up2 = ((a - 1) % slabs_per_prob) != 0 ? uin[bp - S] : T(0);
            spec_residual(c, mu, u, up2, r);
        }
        spec_block_solve(c, mu, r, v);
        old_prev = last_of(u, nt);
        new_prev = old_prev + omega * last_of(v, nt);
    }
    // smoothed slabs a and b
    T ua[NTMAX], ub[NTMAX], r[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        ua[i] = (i < nt && !ZERO) ? uin[ba + (long long)i * S] : T(0);
        ub[i] = (i < nt && !ZERO) ? uin[bb + (long long)i * S] : T(0);
    }
    T old_a_last = T(0);
    old_a_last = last_of(ua, nt);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) r[i] = (i < nt) ? f[ba + (long long)i * S] : T(0);
    if (!ZERO) spec_residual(c, mu, ua, old_prev, r);
    spec_block_solve(c, mu, r, v);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) ua[i] += omega * v[i];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) r[i] = (i < nt) ? f[bb + (long long)i * S] : T(0);
    if (!ZERO) spec_residual(c, mu, ub, old_a_last, r);
    spec_block_solve(c, mu, r, v);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        ub[i] += omega * v[i];
        if (i < nt) {
            uout[ba + (long long)i * S] = ua[i];
            uout[bb + (long long)i * S] = ub[i];
        }
    }
    // residual of the new iterate on both slabs, restricted
    T ra[NTMAX], rb[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        ra[i] = (i < nt) ? f[ba + (long long)i * S] : T(0);
        rb[i] = (i < nt) ? f[bb + (long long)i * S] : T(0);
    }
    T new_a_last = T(0);
    new_a_last = last_of(ua, nt);
    spec_residual(c, mu, ua, new_prev, ra);
    spec_residual(c, mu, ub, new_a_last, rb);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        if (i >= nt) break;
        T sacc = T(0);
#pragma unroll
        for (int j = 0; j < NTMAX; ++j)
            if (j < nt) sacc += pc.P[j * NTMAX + i] * ra[j] + pc.P[(nt + j) * NTMAX + i] * rb[j];
        fc[(m * nt + i) * S + k] = sacc;
    }
}

// Prolongation of the coarse correction fused with the first post-smoothing
// step: one thread per (coarse slab m, mode k) forms the corrected iterate
// u + P_t e on the fine slabs a = 2m, b = 2m + 1 (and the corrected last entry
// of slab a - 1 from coarse slab m - 1) and smooths both slabs out of place.
template <typename T>
__global__ void __launch_bounds__(256)
    k_spec_up(const T *__restrict__ ec, const T *__restrict__ uin, T *__restrict__ uout,
              const T *__restrict__ f, const T *__restrict__ mu_tab, Grid g, const __grid_constant__ SpecCoefs<T> c,
              const __grid_constant__ ProlongCoefs<T> pc, T omega, int slabs_per_prob,
              long long ncoarse) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long m = slab_index(), S = g.nxyz;
    if (k >= S || m >= ncoarse) return;
    const int nt = c.nt;
    const T mu = mu_tab[k];
    const long long a = 2 * m;
    const long long ba = a * nt * S + k, bb = ba + (long long)nt * S;
    T e[NTMAX], ua[NTMAX], ub[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) e[i] = (i < nt) ? ec[(m * nt + i) * S + k] : T(0);
#pragma unroll
    for (int j = 0; j < NTMAX; ++j) {
        T pa = T(0), pb = T(0);
#pragma unroll
        for (int i = 0; i < NTMAX; ++i)
            if (i < nt && j < nt) {
                pa += pc.P[j * NTMAX + i] * e[i];
                pb += pc.P[(nt + j) * NTMAX + i] * e[i];
            }
        ua[j] = (j < nt) ? uin[ba + (long long)j * S] + pa : T(0);
        ub[j] = (j < nt) ? uin[bb + (long long)j * S] + pb : T(0);
    }
    T uprev = T(0);
    if ((a % slabs_per_prob) != 0) {  // corrected last entry of slab a - 1
        T pl = T(0);
#pragma unroll
        for (int i = 0; i < NTMAX; ++i)
            if (i < nt) pl += pc.P[(2 * nt - 1) * NTMAX + i] * ec[((m - 1) * nt + i) * S + k];
        uprev = uin[ba - S] + pl;
    }
    T a_last = T(0);
    a_last = last_of(ua, nt);
    T r[NTMAX], v[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) r[i] = (i < nt) ? f[ba + (long long)i * S] : T(0);
    spec_residual(c, mu, ua, uprev, r);
    spec_block_solve(c, mu, r, v);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i)
        if (i < nt) uout[ba + (long long)i * S] = ua[i] + omega * v[i];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) r[i] = (i < nt) ? f[bb + (long long)i * S] : T(0);
    spec_residual(c, mu, ub, a_last, r);
    spec_block_solve(c, mu, r, v);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i)
        if (i < nt) uout[bb + (long long)i * S] = ub[i] + omega * v[i];
}

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
template <typename T>
__global__ void __launch_bounds__(256)
    k_spec_op(const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ out,
              const T *__restrict__ mu_tab,
              Grid g, const __grid_constant__ SpecCoefs<T> c, int slabs_per_prob, long long nslabs,
              int res) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long slab = slab_index();
    if (k >= g.nxyz || slab >= nslabs) return;
    const int nt = c.nt;
    const long long base = slab * nt * g.nxyz + k;
    const T mu = mu_tab[k];
    T uu[NTMAX], r[NTMAX];
#pragma unroll
    for (int i = 0; i < NTMAX; ++i) {
        uu[i] = (i < nt) ? u[base + (long long)i * g.nxyz] : T(0);
        r[i] = (i < nt && res) ? f[base + (long long)i * g.nxyz] : T(0);
    }
    const T up = ((slab % slabs_per_prob) != 0) ? u[base - g.nxyz] : T(0);
    spec_residual(c, mu, uu, up, r);
#pragma unroll
    for (int i = 0; i < NTMAX; ++i)
        if (i < nt) out[base + (long long)i * g.nxyz] = res ? r[i] : -r[i];
}

template <typename T>
cudaError_t launch_spec_op(const T *u, const T *f, T *out, const T *mu, const Grid &g,
                           const SpecCoefs<T> &c, int slabs_per_prob, long long nslabs, int res,
                           cudaStream_t s) {
    if (nslabs <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, nslabs);
    k_spec_op<T><<<L.grid, L.block, 0, s>>>(u, f, out, mu,
                                                                g, c, slabs_per_prob, nslabs, res);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The whole eigenbasis V-cycle in shared memory.  CTA (problem r, mode block
// b) owns modes k0 .. k0 + MB - 1 of problem r on every slab of every level:
// per level l it keeps u_l and f_l as [nt][N_l][MB] (mode fastest, so a
// warp's 32 consecutive (slab, mode) items hit 32 consecutive words), plus
// one level-0 sized scratch array for the out-of-place Jacobi steps.  All
// levels' time coefficients arrive as one __grid_constant__ parameter block
// (constant-bank operands).  HBM is touched twice: f^ read once, u^ written
// once.  Same arithmetic as k_spec_smooth / k_spec_res_restrict /
// k_prolong_add / k_spec_coarse.
// ---------------------------------------------------------------------------
template <typename T>
struct FusedParams {
    static constexpr int LMAX = sizeof(T) == 4 ? 16 : 8;
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
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_spec_vcycle<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        attr = true;
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
template <typename T>
__global__ void __launch_bounds__(256)
    k_spec_coarse(T *__restrict__ u, const T *__restrict__ f, const T *__restrict__ mu_tab, Grid g,
                  const __grid_constant__ SpecCoefs<T> c, int slabs_per_prob, int nprob) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long prob = slab_index();
    if (k >= g.nxyz || prob >= nprob) return;
    const int nt = c.nt;
    const T mu = mu_tab[k];
    T prev = T(0);
    for (int n = 0; n < slabs_per_prob; ++n) {
        const long long base = ((prob * slabs_per_prob + n) * nt) * g.nxyz + k;
        T r[NTMAX], v[NTMAX];
#pragma unroll
        for (int i = 0; i < NTMAX; ++i) r[i] = (i < nt) ? f[base + (long long)i * g.nxyz] : T(0);
        r[0] += prev;
        spec_block_solve(c, mu, r, v);
#pragma unroll
        for (int i = 0; i < NTMAX; ++i)
            if (i < nt) u[base + (long long)i * g.nxyz] = v[i];
        prev = last_of(v, nt);
    }
}

template <typename T>
cudaError_t launch_spec_smooth(const T *uin, T *uout, const T *f, const T *mu,
                               const Grid &g, const SpecCoefs<T> &c, T omega, int slabs_per_prob,
                               long long nslabs, int uin_zero, cudaStream_t s) {
    if (nslabs <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, nslabs);
    k_spec_smooth<T><<<L.grid, L.block, 0, s>>>(
        uin, uout, f, mu, g, c, omega, slabs_per_prob, nslabs, uin_zero);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_res_restrict(const T *u, const T *f, T *fc, const T *mu,
                                     const Grid &g, const SpecCoefs<T> &c,
                                     const ProlongCoefs<T> &pc, int slabs_per_prob,
                                     long long ncoarse, cudaStream_t s) {
    if (ncoarse <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, ncoarse);
    k_spec_res_restrict<T><<<L.grid, L.block, 0, s>>>(
        u, f, fc, mu, g, c, pc, slabs_per_prob, ncoarse);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_down(const T *uin, T *uout, const T *f, T *fc, const T *mu,
                             const Grid &g, const SpecCoefs<T> &c, const ProlongCoefs<T> &pc,
                             T omega, int slabs_per_prob, long long ncoarse, cudaStream_t s) {
    if (ncoarse <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, ncoarse);
    if (uin)
        k_spec_down<T, false><<<L.grid, L.block, 0, s>>>(uin, uout, f, fc, mu, g, c,
                                                   pc, omega, slabs_per_prob, ncoarse);
    else
        k_spec_down<T, true><<<L.grid, L.block, 0, s>>>(uin, uout, f, fc, mu, g, c,
                                                  pc, omega, slabs_per_prob, ncoarse);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_up(const T *ec, const T *uin, T *uout, const T *f, const T *mu,
                           const Grid &g, const SpecCoefs<T> &c, const ProlongCoefs<T> &pc,
                           T omega, int slabs_per_prob, long long ncoarse, cudaStream_t s) {
    if (ncoarse <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, ncoarse);
    k_spec_up<T><<<L.grid, L.block, 0, s>>>(
        ec, uin, uout, f, mu, g, c, pc, omega, slabs_per_prob, ncoarse);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_coarse(T *u, const T *f, const T *mu, const Grid &g,
                               const SpecCoefs<T> &c, int slabs_per_prob, int nprob,
                               cudaStream_t s) {
    if (nprob <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, nprob);
    k_spec_coarse<T><<<L.grid, L.block, 0, s>>>(u, f, mu, g, c, slabs_per_prob, nprob);
    return cudaGetLastError();
}

#define ST_INST(T)                                                                             \
    template cudaError_t launch_spec_smooth<T>(const T *, T *, const T *, const T *,   \
                                               const Grid &, const SpecCoefs<T> &, T, int,     \
                                               long long, int, cudaStream_t);                  \
    template cudaError_t launch_spec_res_restrict<T>(const T *, const T *, T *,                \
                                                     const T *, const Grid &,          \
                                                     const SpecCoefs<T> &,                     \
                                                     const ProlongCoefs<T> &, int, long long,  \
                                                     cudaStream_t);                            \
    template cudaError_t launch_spec_down<T>(const T *, T *, const T *, T *, const T *, \
                                             const Grid &, const SpecCoefs<T> &,                 \
                                             const ProlongCoefs<T> &, T, int, long long,         \
                                             cudaStream_t);                                      \
    template cudaError_t launch_spec_up<T>(const T *, const T *, T *, const T *,                 \
                                           const T *, const Grid &,                     \
                                           const SpecCoefs<T> &, const ProlongCoefs<T> &, T,    \
                                           int, long long, cudaStream_t);                       \
    template cudaError_t launch_spec_coarse<T>(T *, const T *, const T *, const Grid &, \
                                               const SpecCoefs<T> &, int, int, cudaStream_t);     \
    template cudaError_t launch_mode_solve<T>(T *, const T *, const Grid &,             \
                                              const SpecCoefs<T> &, long long, cudaStream_t);     \
    template cudaError_t launch_spec_op<T>(const T *, const T *, T *, const T *,        \
                                           const Grid &, const SpecCoefs<T> &, int, long long,  \
                                           int, cudaStream_t);                                  \
    template cudaError_t launch_spec_vcycle<T>(const T *, T *, const SpecCoefs<T> *,            \
                                               const T *, const Grid &,                 \
                                               const ProlongCoefs<T> &, int, int, int, int, int, \
                                               T, int, int, cudaStream_t);
ST_INST(double)
ST_INST(float)
#undef ST_INST

}  // namespace st

// Level kernels of the eigenbasis time-multigrid V-cycle (arXiv:1802.09277,
// Sec. 3.1: damped block-Jacobi smoother, time coarsening by slab pairs, with
// the slab inverse of Eq. 3.1 applied per spatial mode).
//
// In the spatial eigenbasis the slab block of mode k is the N_t x N_t matrix
// A_k = K_t + mu_k M_t, with A_k^{-1} = X (Z + mu_k I)^{-1} Y (Eq. 3.1 for one
// mode).  k_mode_inverse forms these inverses once per level in FP64 with the
// Schur-form block solve and stores them in the V-cycle precision as
// inv[(i * N_t + j) * nxyz + k] (mode fastest: a warp reads 32 consecutive
// words per entry).  The level kernels apply them as dense N_t x N_t products
// and use A_k^{-1} A_k = I to drop the residual from the smoothing step:
//
//   u_new = u + w A^{-1} (f - A u + e_0 u_prev) = (1 - w) u + w A^{-1} (f + e_0 u_prev)
//
// and, from a zero iterate (u = u_prev = 0, so A u_new = w f), the residual of
// the smoothed iterate is r = f - A u_new + e_0 u_prev,new = (1 - w) f +
// e_0 u_prev,new.  (e_0 u_prev is the coupling -B^ u_{n-1} = N_t u_{n-1}:
// the last time dof of the previous slab enters the first equation.)
//
// One thread per spatial mode (x of a 2D grid) and slab or slab pair (y, z);
// every kernel is a template on N_t so that all loops have exact length.
//
//  k_lv_smooth        one damped block-Jacobi step, out of place
//  k_lv_down0         from a zero iterate: the smoothing step, the residual of
//                     the new iterate and its restriction P_t^T (two slab pairs
//                     per thread)
//  k_lv_down          the same from a given iterate (the last of nu1 > 1 steps)
//  k_lv_up            prolongation u + P_t e and the first post-smoothing step
//                     (two slab pairs per thread)
//  k_lv_coarse        exact solve of the coarsest level: forward substitution
//                     u_n = A^{-1} (f_n + e_0 u_{n-1, last}) over its slabs
//  k_lv_res_restrict  residual and restriction without smoothing (nu1 = 0)
//  k_lv_op            the eigenbasis operator L^ (or f - L^ u) pointwise
#include <type_traits>

#include "pdl.cuh"
#include "spec_common.cuh"

namespace st {

namespace {

template <typename T, int NT>
__device__ __forceinline__ void load_inv(const T *__restrict__ inv, long long S, int k,
                                         T (&m)[NT * NT]) {
#pragma unroll
    for (int e = 0; e < NT * NT; ++e) m[e] = inv[(long long)e * S + k];
}

template <typename T, int NT>
__device__ __forceinline__ void matvec(const T (&m)[NT * NT], const T (&r)[NT], T (&v)[NT]) {
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        T a = T(0);
#pragma unroll
        for (int j = 0; j < NT; ++j) a += m[i * NT + j] * r[j];
        v[i] = a;
    }
}

// last row of A^{-1} times r
template <typename T, int NT>
__device__ __forceinline__ T lastrow(const T (&m)[NT * NT], const T (&r)[NT]) {
    T a = T(0);
#pragma unroll
    for (int j = 0; j < NT; ++j) a += m[(NT - 1) * NT + j] * r[j];
    return a;
}

template <typename T, int NT>
__device__ __forceinline__ void load_col(const T *__restrict__ x, long long base, long long S,
                                         T (&v)[NT]) {
#pragma unroll
    for (int i = 0; i < NT; ++i) v[i] = x[base + (long long)i * S];
}

template <typename T, int NT>
__device__ __forceinline__ void store_col(T *__restrict__ x, long long base, long long S,
                                          const T (&v)[NT]) {
#pragma unroll
    for (int i = 0; i < NT; ++i) x[base + (long long)i * S] = v[i];
}

// r = f - (K_t + mu M_t) u + e_0 uprev
template <typename T, int NT>
__device__ __forceinline__ void op_residual(const SpecCoefs<T> &c, T mu, const T (&u)[NT],
                                            T uprev, T (&r)[NT]) {
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        T a = r[i];
#pragma unroll
        for (int j = 0; j < NT; ++j) a -= (c.Kt[i * NTMAX + j] + mu * c.Mt[i * NTMAX + j]) * u[j];
        if (i == 0) a += uprev;
        r[i] = a;
    }
}

// fc = P_t^T [ra; rb]
template <typename T, int NT>
__device__ __forceinline__ void restrict_pair(const ProlongCoefs<T> &pc, const T (&ra)[NT],
                                              const T (&rb)[NT], T (&fc)[NT]) {
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < NT; ++j)
            s += pc.P[j * NTMAX + i] * ra[j] + pc.P[(NT + j) * NTMAX + i] * rb[j];
        fc[i] = s;
    }
}

}  // namespace

// inv[(i nt + j) S + k] = (A_k^{-1})_{ij}: column j is the block solve of e_j
template <typename TO>
__global__ void __launch_bounds__(256)
    k_mode_inverse(TO *__restrict__ inv, const double *__restrict__ mu_tab, Grid g,
                   const __grid_constant__ SpecCoefs<double> c) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nxyz) return;
    const long long S = g.nxyz;
    const int nt = c.nt;
    const double mu = mu_tab[k];
    for (int j = 0; j < nt; ++j) {
        double r[NTMAX], v[NTMAX];
#pragma unroll
        for (int i = 0; i < NTMAX; ++i) r[i] = (i == j) ? 1.0 : 0.0;
        spec_block_solve(c, mu, r, v);
#pragma unroll
        for (int i = 0; i < NTMAX; ++i)
            if (i < nt) inv[((long long)i * nt + j) * S + k] = (TO)v[i];
    }
}

template <typename T, int NT>
__global__ void __launch_bounds__(256)
    k_lv_smooth(const T *__restrict__ uin, T *__restrict__ uout, const T *__restrict__ f,
                const T *__restrict__ inv, long long S, T omega, int spp, long long nslabs,
                int zero) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = slab_index();
    if (k >= S || n >= nslabs) return;
    const long long base = n * NT * S + k;
    T m[NT * NT], r[NT], v[NT];
    load_inv<T, NT>(inv, S, k, m);
    load_col<T, NT>(f, base, S, r);
    if (zero) {
        matvec<T, NT>(m, r, v);
#pragma unroll
        for (int i = 0; i < NT; ++i) v[i] *= omega;
    } else {
        T u[NT];
        load_col<T, NT>(uin, base, S, u);
        if (((int)n % spp) != 0) r[0] += uin[base - S];
        matvec<T, NT>(m, r, v);
#pragma unroll
        for (int i = 0; i < NT; ++i) v[i] = (T(1) - omega) * u[i] + omega * v[i];
    }
    store_col<T, NT>(uout, base, S, v);
}

// The last of nu1 > 1 pre-smoothing steps (from a given iterate), the
// residual of the new iterate and its restriction, one slab pair per thread.
// Jacobi: the smoothed slabs see their predecessors' OLD iterates; the
// residual needs the NEW last entry of slab a - 1, which the thread
// recomputes (one more block product instead of a pass over HBM).
template <typename T, int NT>
__global__ void __launch_bounds__(256)
    k_lv_down(const T *__restrict__ uin, T *__restrict__ uout, const T *__restrict__ f,
              T *__restrict__ fc, const T *__restrict__ inv, const T *__restrict__ mu_tab,
              long long S, const __grid_constant__ SpecCoefs<T> c,
              const __grid_constant__ ProlongCoefs<T> pc, T omega, int spp, long long ncoarse) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long mc = slab_index();
    if (k >= S || mc >= ncoarse) return;
    const long long a = 2 * mc;
    const bool first = ((int)a % spp) == 0;
    const long long ba = a * NT * S + k, bb = ba + (long long)NT * S;
    T m[NT * NT];
    load_inv<T, NT>(inv, S, k, m);
    T new_prev = T(0), old_prev = T(0);
    if (!first) {
        const long long bp = ba - (long long)NT * S;
        T rp[NT];
        load_col<T, NT>(f, bp, S, rp);
        old_prev = uin[bp + (long long)(NT - 1) * S];
        if (((int)a - 1) % spp != 0) rp[0] += uin[bp - S];
        new_prev = (T(1) - omega) * old_prev + omega * lastrow<T, NT>(m, rp);
    }
    T fa[NT], fb[NT], ua[NT], ub[NT], oa[NT], ob[NT], r[NT];
    load_col<T, NT>(f, ba, S, fa);
    load_col<T, NT>(f, bb, S, fb);
    load_col<T, NT>(uin, ba, S, oa);
    load_col<T, NT>(uin, bb, S, ob);
#pragma unroll
    for (int i = 0; i < NT; ++i) r[i] = fa[i];
    r[0] += old_prev;
    matvec<T, NT>(m, r, ua);
#pragma unroll
    for (int i = 0; i < NT; ++i) ua[i] = (T(1) - omega) * oa[i] + omega * ua[i];
#pragma unroll
    for (int i = 0; i < NT; ++i) r[i] = fb[i];
    r[0] += oa[NT - 1];
    matvec<T, NT>(m, r, ub);
#pragma unroll
    for (int i = 0; i < NT; ++i) ub[i] = (T(1) - omega) * ob[i] + omega * ub[i];
    store_col<T, NT>(uout, ba, S, ua);
    store_col<T, NT>(uout, bb, S, ub);
    // residual of the smoothed iterate, formed directly
    const T mu = mu_tab[k];
    T out[NT];
    op_residual<T, NT>(c, mu, ua, new_prev, fa);
    op_residual<T, NT>(c, mu, ub, ua[NT - 1], fb);
    restrict_pair<T, NT>(pc, fa, fb, out);
    store_col<T, NT>(fc, mc * NT * S + k, S, out);
}

// Pre-smoothing from zero + residual + restriction for PP consecutive slab
// pairs of one mode per thread: the mode's inverse is loaded once for all of
// them, and the new last entry of the slab before pair q > 0 is the previous
// pair's (from zero, so A u_new = w f and the residual is (1 - w) f + e_0 u_prev,new).
template <typename T, int NT, int PP>
__global__ void __launch_bounds__(256)
    k_lv_down0(T *__restrict__ uout, const T *__restrict__ f, T *__restrict__ fc,
               const T *__restrict__ inv, long long S, const __grid_constant__ ProlongCoefs<T> pc,
               T omega, int spp, long long ncoarse) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long mc0 = slab_index() * PP;
    if (k >= S || mc0 >= ncoarse) return;
    T m[NT * NT];
    load_inv<T, NT>(inv, S, k, m);
    T carried = T(0);
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        const long long mc = mc0 + q;
        if (mc >= ncoarse) break;
        const long long a = 2 * mc;
        const long long ba = a * NT * S + k, bb = ba + (long long)NT * S;
        T new_prev = T(0);
        if (((int)a % spp) != 0) {
            if (q > 0) {
                new_prev = carried;
            } else {
                T rp[NT];
                load_col<T, NT>(f, ba - (long long)NT * S, S, rp);
                new_prev = omega * lastrow<T, NT>(m, rp);
            }
        }
        T fa[NT], fb[NT], ua[NT], ub[NT];
        load_col<T, NT>(f, ba, S, fa);
        load_col<T, NT>(f, bb, S, fb);
        matvec<T, NT>(m, fa, ua);
        matvec<T, NT>(m, fb, ub);
        T ra[NT], rb[NT], out[NT];
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            ua[i] *= omega;
            ub[i] *= omega;
            ra[i] = (T(1) - omega) * fa[i];
            rb[i] = (T(1) - omega) * fb[i];
        }
        store_col<T, NT>(uout, ba, S, ua);
        store_col<T, NT>(uout, bb, S, ub);
        ra[0] += new_prev;
        rb[0] += ua[NT - 1];
        carried = ub[NT - 1];
        restrict_pair<T, NT>(pc, ra, rb, out);
        store_col<T, NT>(fc, mc * NT * S + k, S, out);
    }
}

// Prolongation + first post-smoothing step for PP consecutive slab pairs of
// one mode per thread (Jacobi: each slab sees its predecessor corrected but
// not yet smoothed): the corrected last
// entry of the slab before pair q > 0 is the previous pair's.
template <typename T, int NT, int PP>
__global__ void __launch_bounds__(256)
    k_lv_up(const T *__restrict__ ec, const T *__restrict__ uin, T *__restrict__ uout,
             const T *__restrict__ f, const T *__restrict__ inv, long long S,
             const __grid_constant__ ProlongCoefs<T> pc, T omega, int spp, long long ncoarse) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long mc0 = slab_index() * PP;
    if (k >= S || mc0 >= ncoarse) return;
    T m[NT * NT];
    load_inv<T, NT>(inv, S, k, m);
    T carried = T(0);
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        const long long mc = mc0 + q;
        if (mc >= ncoarse) break;
        const long long a = 2 * mc;
        const long long ba = a * NT * S + k, bb = ba + (long long)NT * S;
        T e[NT], ua[NT], ub[NT], fa[NT], fb[NT];
        load_col<T, NT>(ec, mc * NT * S + k, S, e);
        load_col<T, NT>(uin, ba, S, ua);
        load_col<T, NT>(uin, bb, S, ub);
        load_col<T, NT>(f, ba, S, fa);
        load_col<T, NT>(f, bb, S, fb);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            T pa = T(0), pb = T(0);
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                pa += pc.P[j * NTMAX + i] * e[i];
                pb += pc.P[(NT + j) * NTMAX + i] * e[i];
            }
            ua[j] += pa;
            ub[j] += pb;
        }
        T uprev = T(0);
        if (((int)a % spp) != 0) {
            if (q > 0) {
                uprev = carried;
            } else {
                T ep[NT];
                load_col<T, NT>(ec, (mc - 1) * NT * S + k, S, ep);
                T pl = T(0);
#pragma unroll
                for (int i = 0; i < NT; ++i) pl += pc.P[(2 * NT - 1) * NTMAX + i] * ep[i];
                uprev = uin[ba - S] + pl;
            }
        }
        carried = ub[NT - 1];
        T v[NT];
        fa[0] += uprev;
        matvec<T, NT>(m, fa, v);
#pragma unroll
        for (int i = 0; i < NT; ++i) v[i] = (T(1) - omega) * ua[i] + omega * v[i];
        store_col<T, NT>(uout, ba, S, v);
        fb[0] += ua[NT - 1];
        matvec<T, NT>(m, fb, v);
#pragma unroll
        for (int i = 0; i < NT; ++i) v[i] = (T(1) - omega) * ub[i] + omega * v[i];
        store_col<T, NT>(uout, bb, S, v);
    }
}

template <typename T, int NT>
__global__ void __launch_bounds__(256)
    k_lv_coarse(T *__restrict__ u, const T *__restrict__ f, const T *__restrict__ inv, long long S,
                int spp, long long nprob) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long q = slab_index();
    if (k >= S || q >= nprob) return;
    T m[NT * NT];
    load_inv<T, NT>(inv, S, k, m);
    T prev = T(0);
    for (int n = 0; n < spp; ++n) {
        const long long base = ((q * spp + n) * NT) * S + k;
        T r[NT], v[NT];
        load_col<T, NT>(f, base, S, r);
        r[0] += prev;
        matvec<T, NT>(m, r, v);
        store_col<T, NT>(u, base, S, v);
        prev = v[NT - 1];
    }
}

template <typename T, int NT>
__global__ void __launch_bounds__(256)
    k_lv_res_restrict(const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ fc,
                      const T *__restrict__ mu_tab, long long S,
                      const __grid_constant__ SpecCoefs<T> c,
                      const __grid_constant__ ProlongCoefs<T> pc, int spp, long long ncoarse) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long mc = slab_index();
    if (k >= S || mc >= ncoarse) return;
    const long long a = 2 * mc;
    const long long ba = a * NT * S + k, bb = ba + (long long)NT * S;
    const T mu = mu_tab[k];
    T ua[NT], ub[NT], ra[NT], rb[NT], out[NT];
    load_col<T, NT>(u, ba, S, ua);
    load_col<T, NT>(u, bb, S, ub);
    load_col<T, NT>(f, ba, S, ra);
    load_col<T, NT>(f, bb, S, rb);
    const T uprev = (((int)a % spp) != 0) ? u[ba - S] : T(0);
    op_residual<T, NT>(c, mu, ua, uprev, ra);
    op_residual<T, NT>(c, mu, ub, ua[NT - 1], rb);
    restrict_pair<T, NT>(pc, ra, rb, out);
    store_col<T, NT>(fc, mc * NT * S + k, S, out);
}

// res = 1: out = f - L^ u, else out = L^ u
template <typename T, int NT>
__global__ void __launch_bounds__(256)
    k_lv_op(const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ out,
            const T *__restrict__ mu_tab, long long S, const __grid_constant__ SpecCoefs<T> c,
            int spp, long long nslabs, int res) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = slab_index();
    if (k >= S || n >= nslabs) return;
    const long long base = n * NT * S + k;
    const T mu = mu_tab[k];
    T uu[NT], r[NT];
    load_col<T, NT>(u, base, S, uu);
    if (res) {
        load_col<T, NT>(f, base, S, r);
    } else {
#pragma unroll
        for (int i = 0; i < NT; ++i) r[i] = T(0);
    }
    const T up = (((int)n % spp) != 0) ? u[base - S] : T(0);
    op_residual<T, NT>(c, mu, uu, up, r);
    if (!res) {
#pragma unroll
        for (int i = 0; i < NT; ++i) r[i] = -r[i];
    }
    store_col<T, NT>(out, base, S, r);
}

// Sweeping level kernels for nu >= 2 smoothing steps: one thread per
// spatial mode and chunk of C consecutive slabs of one right-hand side walks
// its slabs in time order.  A Jacobi step of slab n needs only the previous
// slab's last entry from the step before, so all NU steps of a slab run in
// registers as the sweep passes it (the previous slab's last entry after
// each step is kept): every level is read and written once whatever NU.  A
// chunk first recomputes the NU slabs before it (halo; their results are not
// stored), after which its own slabs are exact.
//
// k_lv_sweep_down: from u = 0, NU steps, the residual of the result and its
// restriction.  In residual form a step is u' = u + w A^-1 r and the residual
// moves to r' = (1 - w) r + e_0 (p' - p), p / p' the previous slab's last
// entry before / after the step, so only A^-1 is needed; r starts at f.
// CTAs per SM the down sweep is compiled for: five (48 registers) where its
// prefetching loop fits them without spilling (FP32, N_t <= 3, or N_t = 4
// with up to four steps); there the prefetch at 61 registers lost a CTA per
// SM and more time than it saved
template <typename T, int NT, int NU>
constexpr int sweep_down_min_blocks() {
    return (sizeof(T) == 4 && (NT <= 3 || (NT == 4 && NU <= 4))) ? 5 : 1;
}

template <typename T, int NT, int NU>
__global__ void __launch_bounds__(256, sweep_down_min_blocks<T, NT, NU>())
    k_lv_sweep_down(const T *__restrict__ f, T *__restrict__ u, T *__restrict__ fc,
                    const T *__restrict__ inv, long long S, const __grid_constant__ ProlongCoefs<T> pc,
                    T omega, int N, int C, int nchunk, long long nwork) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long w = slab_index();
    if (k >= S || w >= nwork) return;
    const long long q = w / nchunk;
    const int n0 = (int)(w % nchunk) * C;
    const int n1 = (n0 + C < N) ? n0 + C : N;
    const int h = (n0 - NU > 0) ? n0 - NU : 0;
    const long long slab = (long long)NT * S;
    const long long fb = q * N * slab + k, cb = q * (N / 2) * slab + k;
    T m[NT * NT];
    load_inv<T, NT>(inv, S, k, m);
    T last[NU + 1];  // previous slab's last entry after step s (s = 0: the zero start)
#pragma unroll
    for (int st = 0; st <= NU; ++st) last[st] = T(0);
    T reven[NT];
    // the next slab's column is loaded while this one is computed: two
    // slabs' loads in flight per thread (one alone left the kernel
    // latency-bound at about 5 TB/s)
    T rn[NT];
    if (h < n1) load_col<T, NT>(f, fb + h * slab, S, rn);
    for (int n = h; n < n1; ++n) {
        T r[NT], x[NT];
#pragma unroll
        for (int i = 0; i < NT; ++i) r[i] = rn[i];
        if (n + 1 < n1) load_col<T, NT>(f, fb + (n + 1) * slab, S, rn);
#pragma unroll
        for (int i = 0; i < NT; ++i) x[i] = T(0);
        T nl[NU + 1];
        nl[0] = T(0);
#pragma unroll
        for (int st = 1; st <= NU; ++st) {
            T d[NT];
            matvec<T, NT>(m, r, d);
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                x[i] += omega * d[i];
                r[i] = (T(1) - omega) * r[i];
            }
            r[0] += last[st] - last[st - 1];
            nl[st] = x[NT - 1];
        }
#pragma unroll
        for (int st = 0; st <= NU; ++st) last[st] = nl[st];
        if (n < n0) continue;
        store_col<T, NT>(u, fb + n * slab, S, x);
        if (((n - n0) & 1) == 0) {
#pragma unroll
            for (int i = 0; i < NT; ++i) reven[i] = r[i];
        } else {
            T out[NT];
            restrict_pair<T, NT>(pc, reven, r, out);
            store_col<T, NT>(fc, cb + (long long)(n / 2) * slab, S, out);
        }
    }
}

// k_lv_sweep_up: the prolongation u + P_t e and NU Jacobi steps
// u' = (1 - w) u + w A^-1 (f + e_0 p), p the previous slab's last entry
// before the step, out of place (uin -> uout: the next chunk's halo reads uin).
template <typename T, int NT, int NU>
__global__ void __launch_bounds__(256)
    k_lv_sweep_up(const T *__restrict__ ec, const T *__restrict__ uin, T *__restrict__ uout,
                  const T *__restrict__ f, const T *__restrict__ inv, long long S,
                  const __grid_constant__ ProlongCoefs<T> pc, T omega, int N, int C, int nchunk,
                  long long nwork) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long w = slab_index();
    if (k >= S || w >= nwork) return;
    const long long q = w / nchunk;
    const int n0 = (int)(w % nchunk) * C;
    const int n1 = (n0 + C < N) ? n0 + C : N;
    const int h = (n0 - NU > 0) ? n0 - NU : 0;
    const long long slab = (long long)NT * S;
    const long long fb = q * N * slab + k, cb = q * (N / 2) * slab + k;
    T m[NT * NT];
    load_inv<T, NT>(inv, S, k, m);
    T last[NU];  // previous slab's last entry before step s + 1
#pragma unroll
    for (int st = 0; st < NU; ++st) last[st] = T(0);
    // the next slab's columns are loaded while this one is computed (the
    // coarse column once per slab pair)
    T xn[NT], en[NT], fn[NT];
    if (h < n1) {
        load_col<T, NT>(uin, fb + h * slab, S, xn);
        load_col<T, NT>(ec, cb + (long long)(h / 2) * slab, S, en);
        load_col<T, NT>(f, fb + h * slab, S, fn);
    }
    for (int n = h; n < n1; ++n) {
        T x[NT], e[NT], fr[NT];
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            x[i] = xn[i];
            e[i] = en[i];
            fr[i] = fn[i];
        }
        if (n + 1 < n1) {
            load_col<T, NT>(uin, fb + (n + 1) * slab, S, xn);
            if (((n + 1) & 1) == 0) load_col<T, NT>(ec, cb + (long long)((n + 1) / 2) * slab, S, en);
            load_col<T, NT>(f, fb + (n + 1) * slab, S, fn);
        }
        const int half = (n & 1) ? NT : 0;  // row block of P_t for this slab of the pair
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            T pj = T(0);
#pragma unroll
            for (int i = 0; i < NT; ++i) pj += pc.P[(half + j) * NTMAX + i] * e[i];
            x[j] += pj;
        }
        T nl[NU];
#pragma unroll
        for (int st = 0; st < NU; ++st) {
            T rr[NT], v[NT];
#pragma unroll
            for (int i = 0; i < NT; ++i) rr[i] = fr[i];
            rr[0] += last[st];
            nl[st] = x[NT - 1];
            matvec<T, NT>(m, rr, v);
#pragma unroll
            for (int i = 0; i < NT; ++i) x[i] = (T(1) - omega) * x[i] + omega * v[i];
        }
#pragma unroll
        for (int st = 0; st < NU; ++st) last[st] = nl[st];
        if (n >= n0) store_col<T, NT>(uout, fb + n * slab, S, x);
    }
}

// The coarse end of the V-cycle, levels l0 .. L (N_{l0} <= TAIL_SLABS slabs
// per problem, nu1, nu2 <= 8 smoothing steps, zero initial iterate on every
// level), in one launch: one thread per (spatial mode, rhs) runs the
// sub-cycle sequentially over its slabs, the same steps as k_lv_down0 /
// k_lv_coarse / k_lv_up: the Jacobi steps see the previous slab's iterate
// from before the step, which the sequential sweep keeps in a register.  The
// level vectors are thread-local arrays: in local memory for a run-time slab
// count (L1-resident only while few threads run), in registers for the small
// tails whose slab and level counts are compile-time constants.
constexpr int TAIL_SLABS = 16;
template <typename T>
struct TailArgs {
    const T *inv[16];  // per-mode inverses of levels l0 .. L
    int nlev;          // L - l0 + 1
    int nu1, nu2;      // smoothing steps before / after the coarse correction
};

// N0C > 0: the top level's slab count N0C and the level count NLC fixed at
// compile time, so that every loop unrolls and the level vectors live in
// registers (a few slabs); N0C = 0: both at run time, the vectors in local
// memory (up to TAIL_SLABS slabs).
template <typename T, int NT, int N0C = 0, int NLC = 0>
__global__ void __launch_bounds__(128)
    k_lv_tail(const T *__restrict__ fin, T *__restrict__ uout, const __grid_constant__ TailArgs<T> ta,
              const __grid_constant__ ProlongCoefs<T> pc, long long S, int n0_arg, T omega) {
    griddep_wait();
    griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const long long q = slab_index();  // right-hand side
    if (k >= S) return;
    constexpr int NMAX = N0C > 0 ? N0C : TAIL_SLABS;
    constexpr int CAP = 2 * NMAX * NT;  // slabs of all tail levels, per vector
    const int n0 = N0C > 0 ? N0C : n0_arg;
    const int nlev = NLC > 0 ? NLC : ta.nlev;
    T f[CAP], u[CAP];
    int off[16];
    {
        int o = 0;
#pragma unroll
        for (int l = 0; l < (NLC > 0 ? NLC : 16); ++l) {
            if (l >= nlev) break;
            off[l] = o;
            o += (n0 >> l) * NT;
        }
    }
    const long long gbase = q * n0 * NT * S + k;
#pragma unroll
    for (int e = 0; e < NMAX * NT; ++e)
        if (e < n0 * NT) f[e] = fin[gbase + (long long)e * S];
    // down: nu1 smoothing steps from zero, the residual, restriction.  The
    // first step from zero is u = w A^-1 f with residual (1 - w) f + e_0 p'
    // (p' the new last entry of the slab before); each further Jacobi step
    // u' = u + w A^-1 r carries the residual forward without A:
    // r' = (1 - w) r + e_0 (p' - p), p / p' that entry before / after the step.
#pragma unroll
    for (int l = 0; l + 1 < (NLC > 0 ? NLC : 16); ++l) {
        if (l + 1 >= nlev) break;
        const int N = n0 >> l;
        T m[NT * NT];
        load_inv<T, NT>(ta.inv[l], S, k, m);
        T *fl = f + off[l], *ul = u + off[l], *fc = f + off[l + 1];
        T r[NMAX * NT];
        if (ta.nu1 == 0) {
            #pragma unroll
            for (int e = 0; e < (N0C > 0 ? NMAX * NT : N * NT); ++e) {
                if (e >= N * NT) break;
                ul[e] = T(0);
                r[e] = fl[e];
            }
        } else {
            T prev = T(0);  // new last entry of the slab before
            #pragma unroll
            for (int n = 0; n < (N0C > 0 ? NMAX : N); ++n) {
                if (n >= N) break;
                T fa[NT], ua[NT];
#pragma unroll
                for (int i = 0; i < NT; ++i) fa[i] = fl[n * NT + i];
                matvec<T, NT>(m, fa, ua);
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    ua[i] *= omega;
                    ul[n * NT + i] = ua[i];
                    r[n * NT + i] = (T(1) - omega) * fa[i];
                }
                r[n * NT] += prev;
                prev = ua[NT - 1];
            }
        }
        for (int st = 1; st < ta.nu1; ++st) {
            T old_prev = T(0), new_prev = T(0);
            #pragma unroll
            for (int n = 0; n < (N0C > 0 ? NMAX : N); ++n) {
                if (n >= N) break;
                T ra[NT], d[NT];
#pragma unroll
                for (int i = 0; i < NT; ++i) ra[i] = r[n * NT + i];
                matvec<T, NT>(m, ra, d);
                const T old_last = ul[n * NT + NT - 1];
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    ul[n * NT + i] += omega * d[i];
                    r[n * NT + i] = (T(1) - omega) * ra[i];
                }
                r[n * NT] += new_prev - old_prev;
                old_prev = old_last;
                new_prev = ul[n * NT + NT - 1];
            }
        }
        #pragma unroll
        for (int mc = 0; mc < (N0C > 0 ? NMAX / 2 : N / 2); ++mc) {
            if (mc >= N / 2) break;
            T ra[NT], rb[NT], out[NT];
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                ra[i] = r[(2 * mc) * NT + i];
                rb[i] = r[(2 * mc + 1) * NT + i];
            }
            restrict_pair<T, NT>(pc, ra, rb, out);
#pragma unroll
            for (int i = 0; i < NT; ++i) fc[mc * NT + i] = out[i];
        }
    }
    {  // coarsest level: forward substitution
        const int l = nlev - 1, N = n0 >> l;
        T m[NT * NT];
        load_inv<T, NT>(ta.inv[l], S, k, m);
        T prev = T(0);
        #pragma unroll
            for (int n = 0; n < (N0C > 0 ? NMAX : N); ++n) {
                if (n >= N) break;
            T r[NT], v[NT];
#pragma unroll
            for (int i = 0; i < NT; ++i) r[i] = f[off[l] + n * NT + i];
            r[0] += prev;
            matvec<T, NT>(m, r, v);
#pragma unroll
            for (int i = 0; i < NT; ++i) u[off[l] + n * NT + i] = v[i];
            prev = v[NT - 1];
        }
    }
    // up: prolongation of the coarse correction, then nu2 Jacobi steps
    // u' = (1 - w) u + w A^-1 (f + e_0 p), p the previous slab's last entry
    // before the step (the first step fused with the prolongation)
    #pragma unroll
    for (int l = (NLC > 0 ? NLC : 16) - 2; l >= 0; --l) {
        if (l > nlev - 2) continue;
        const int N = n0 >> l;
        T m[NT * NT];
        load_inv<T, NT>(ta.inv[l], S, k, m);
        const T *fl = f + off[l], *uc = u + off[l + 1];
        T *ul = u + off[l];
        T prev = T(0);  // corrected (not yet smoothed) last entry of the slab before
        #pragma unroll
        for (int mc = 0; mc < (N0C > 0 ? NMAX / 2 : N / 2); ++mc) {
            if (mc >= N / 2) break;
            T e[NT], ua[NT], ub[NT], r[NT], v[NT];
#pragma unroll
            for (int i = 0; i < NT; ++i) e[i] = uc[mc * NT + i];
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                T pa = T(0), pb = T(0);
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    pa += pc.P[j * NTMAX + i] * e[i];
                    pb += pc.P[(NT + j) * NTMAX + i] * e[i];
                }
                ua[j] = ul[(2 * mc) * NT + j] + pa;
                ub[j] = ul[(2 * mc + 1) * NT + j] + pb;
            }
            if (ta.nu2 == 0) {
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    ul[(2 * mc) * NT + i] = ua[i];
                    ul[(2 * mc + 1) * NT + i] = ub[i];
                }
                continue;
            }
#pragma unroll
            for (int i = 0; i < NT; ++i) r[i] = fl[(2 * mc) * NT + i];
            r[0] += prev;
            matvec<T, NT>(m, r, v);
            const T a_last = ua[NT - 1];
            prev = ub[NT - 1];
#pragma unroll
            for (int i = 0; i < NT; ++i) ul[(2 * mc) * NT + i] = (T(1) - omega) * ua[i] + omega * v[i];
#pragma unroll
            for (int i = 0; i < NT; ++i) r[i] = fl[(2 * mc + 1) * NT + i];
            r[0] += a_last;
            matvec<T, NT>(m, r, v);
#pragma unroll
            for (int i = 0; i < NT; ++i)
                ul[(2 * mc + 1) * NT + i] = (T(1) - omega) * ub[i] + omega * v[i];
        }
        for (int st = 1; st < ta.nu2; ++st) {
            T old_prev = T(0);
            #pragma unroll
            for (int n = 0; n < (N0C > 0 ? NMAX : N); ++n) {
                if (n >= N) break;
                T r[NT], v[NT];
#pragma unroll
                for (int i = 0; i < NT; ++i) r[i] = fl[n * NT + i];
                r[0] += old_prev;
                matvec<T, NT>(m, r, v);
                old_prev = ul[n * NT + NT - 1];
#pragma unroll
                for (int i = 0; i < NT; ++i)
                    ul[n * NT + i] = (T(1) - omega) * ul[n * NT + i] + omega * v[i];
            }
        }
    }
#pragma unroll
    for (int e = 0; e < NMAX * NT; ++e)
        if (e < n0 * NT) uout[gbase + (long long)e * S] = u[e];
}

// ---- launchers: dispatch on N_t ----
#define ST_NT_DISPATCH(nt, CALL)          \
    switch (nt) {                         \
        case 2: { constexpr int NT = 2; CALL; break; } \
        case 3: { constexpr int NT = 3; CALL; break; } \
        case 4: { constexpr int NT = 4; CALL; break; } \
        case 5: { constexpr int NT = 5; CALL; break; } \
        case 6: { constexpr int NT = 6; CALL; break; } \
        case 7: { constexpr int NT = 7; CALL; break; } \
        case 8: { constexpr int NT = 8; CALL; break; } \
        default: return cudaErrorNotSupported;         \
    }

template <typename TO>
cudaError_t launch_mode_inverse(TO *inv, const double *mu64, const Grid &g,
                                const SpecCoefs<double> &c, cudaStream_t s) {
    if (g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, 1);
    k_mode_inverse<TO><<<L.grid, L.block, 0, s>>>(inv, mu64, g, c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_smooth(const T *uin, T *uout, const T *f, const T *inv, const Grid &g,
                               int nt, T omega, int spp, long long nslabs, int uin_zero,
                               cudaStream_t s) {
    if (nslabs <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, nslabs);
    cudaError_t e = cudaSuccess;
    ST_NT_DISPATCH(nt, (e = launch_pdl(k_lv_smooth<T, NT>, L.grid, L.block, 0, s, uin, uout, f,
                                       inv, g.nxyz, omega, spp, nslabs, uin_zero)));
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_down(const T *uin, T *uout, const T *f, T *fc, const T *inv,
                             const T *mu, const Grid &g, const SpecCoefs<T> &c,
                             const ProlongCoefs<T> &pc, T omega, int spp, long long ncoarse,
                             cudaStream_t s) {
    if (ncoarse <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, ncoarse);
    cudaError_t e = cudaSuccess;
    if (uin) {
        ST_NT_DISPATCH(c.nt, (e = launch_pdl(k_lv_down<T, NT>, L.grid, L.block, 0, s, uin, uout,
                                             f, fc, inv, mu, g.nxyz, c, pc, omega, spp,
                                             ncoarse)));
    } else {  // from zero: two slab pairs per thread
        const ModeLaunch L2 = mode_launch(g.nxyz, (ncoarse + 1) / 2);
        ST_NT_DISPATCH(c.nt, (e = launch_pdl(k_lv_down0<T, NT, 2>, L2.grid, L2.block, 0, s, uout,
                                             f, fc, inv, g.nxyz, pc, omega, spp, ncoarse)));
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_up(const T *ec, const T *uin, T *uout, const T *f, const T *inv,
                           const Grid &g, const ProlongCoefs<T> &pc, T omega, int spp,
                           long long ncoarse, cudaStream_t s) {
    if (ncoarse <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, (ncoarse + 1) / 2);  // two slab pairs per thread
    cudaError_t e = cudaSuccess;
    ST_NT_DISPATCH(pc.nt, (e = launch_pdl(k_lv_up<T, NT, 2>, L.grid, L.block, 0, s, ec, uin, uout,
                                          f, inv, g.nxyz, pc, omega, spp, ncoarse)));
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_coarse(T *u, const T *f, const T *inv, const Grid &g, int nt, int spp,
                               int nprob, cudaStream_t s) {
    if (nprob <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, nprob);
    cudaError_t e = cudaSuccess;
    ST_NT_DISPATCH(nt, (e = launch_pdl(k_lv_coarse<T, NT>, L.grid, L.block, 0, s, u, f, inv,
                                       g.nxyz, spp, (long long)nprob)));
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_res_restrict(const T *u, const T *f, T *fc, const T *mu, const Grid &g,
                                     const SpecCoefs<T> &c, const ProlongCoefs<T> &pc, int spp,
                                     long long ncoarse, cudaStream_t s) {
    if (ncoarse <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, ncoarse);
    cudaError_t e = cudaSuccess;
    ST_NT_DISPATCH(c.nt, (e = launch_pdl(k_lv_res_restrict<T, NT>, L.grid, L.block, 0, s, u, f,
                                         fc, mu, g.nxyz, c, pc, spp, ncoarse)));
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_op(const T *u, const T *f, T *out, const T *mu, const Grid &g,
                           const SpecCoefs<T> &c, int spp, long long nslabs, int res,
                           cudaStream_t s) {
    if (nslabs <= 0 || g.nxyz <= 0) return cudaSuccess;
    const ModeLaunch L = mode_launch(g.nxyz, nslabs);
    cudaError_t e = cudaSuccess;
    ST_NT_DISPATCH(c.nt, (e = launch_pdl(k_lv_op<T, NT>, L.grid, L.block, 0, s, u, f, out, mu,
                                         g.nxyz, c, spp, nslabs, res)));
    return e != cudaSuccess ? e : cudaGetLastError();
}
// the sub-cycle of levels l0 .. L in one launch; cudaErrorNotSupported when
// n0 > TAIL_SLABS or more than 16 levels
template <typename T>
cudaError_t launch_spec_tail(const T *fin, T *uout, const T *const *inv, int nlev,
                             const Grid &g, const ProlongCoefs<T> &pc, T omega, int n0, int nrhs,
                             int nu1, int nu2, cudaStream_t s) {
    if (n0 > TAIL_SLABS || nlev > 16 || nlev < 1 || (n0 >> (nlev - 1)) < 1) return cudaErrorNotSupported;
    if (nu1 < 0 || nu2 < 0 || nu1 > 8 || nu2 > 8) return cudaErrorNotSupported;
    if (g.nxyz <= 0 || nrhs <= 0) return cudaSuccess;
    TailArgs<T> ta;
    for (int l = 0; l < nlev; ++l) ta.inv[l] = inv[l];
    ta.nlev = nlev;
    ta.nu1 = nu1;
    ta.nu2 = nu2;
    ModeLaunch L = mode_launch(g.nxyz, nrhs);
    if (L.block.x > 128) {  // smaller CTAs: more SMs share the few modes
        L.block.x = 128;
        L.grid.x = (unsigned)((g.nxyz + 127) / 128);
    }
    cudaError_t e = cudaSuccess;
    // the complete power-of-two tails of at most 4 slabs in registers (FP32)
    if (std::is_same<T, float>::value && n0 == 4 && nlev == 3) {
        ST_NT_DISPATCH(pc.nt, (e = launch_pdl(k_lv_tail<T, NT, 4, 3>, L.grid, L.block, 0, s, fin,
                                              uout, ta, pc, g.nxyz, n0, omega)));
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    if (std::is_same<T, float>::value && n0 == 2 && nlev == 2) {
        ST_NT_DISPATCH(pc.nt, (e = launch_pdl(k_lv_tail<T, NT, 2, 2>, L.grid, L.block, 0, s, fin,
                                              uout, ta, pc, g.nxyz, n0, omega)));
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    ST_NT_DISPATCH(pc.nt, (e = launch_pdl(k_lv_tail<T, NT>, L.grid, L.block, 0, s, fin, uout, ta,
                                          pc, g.nxyz, n0, omega)));
    return e != cudaSuccess ? e : cudaGetLastError();
}
// Chunk length of the sweeping kernels: enough (mode, chunk) threads to fill
// the GPU, chunks even and at least 4 NU slabs long (halo overhead <= 1/4).
static void sweep_chunks(long long S, int R, int N, int nu, int *C, int *nchunk) {
    const long long want = 152LL * 2048;
    long long nc = (want + S * R - 1) / (S * R);
    const long long cmax = N / (4 * nu) > 1 ? N / (4 * nu) : 1;
    if (nc > cmax) nc = cmax;
    if (nc < 1) nc = 1;
    int c = (int)((N + nc - 1) / nc);
    c = (c + 1) & ~1;
    *C = c;
    *nchunk = (N + c - 1) / c;
}

template <typename T>
cudaError_t launch_spec_sweep_down(const T *f, T *u, T *fc, const T *inv, const Grid &g,
                                   const ProlongCoefs<T> &pc, T omega, int N, int nrhs, int nu,
                                   cudaStream_t s) {
    if (nu < 2 || nu > 6 || N % 2 != 0) return cudaErrorNotSupported;
    if (g.nxyz <= 0 || nrhs <= 0) return cudaSuccess;
    int C = 0, nch = 0;
    sweep_chunks(g.nxyz, nrhs, N, nu, &C, &nch);
    const long long nwork = (long long)nrhs * nch;
    const ModeLaunch L = mode_launch(g.nxyz, nwork);
    cudaError_t e = cudaSuccess;
#define ST_SWEEP_D(NU)                                                                          \
    if (nu == NU)                                                                               \
        ST_NT_DISPATCH(pc.nt, (e = launch_pdl(k_lv_sweep_down<T, NT, NU>, L.grid, L.block, 0, s, \
                                              f, u, fc, inv, g.nxyz, pc, omega, N, C, nch,       \
                                              nwork)));
    ST_SWEEP_D(2) ST_SWEEP_D(3) ST_SWEEP_D(4) ST_SWEEP_D(5) ST_SWEEP_D(6)
#undef ST_SWEEP_D
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_sweep_up(const T *ec, const T *uin, T *uout, const T *f, const T *inv,
                                 const Grid &g, const ProlongCoefs<T> &pc, T omega, int N,
                                 int nrhs, int nu, cudaStream_t s) {
    if (nu < 2 || nu > 6 || N % 2 != 0) return cudaErrorNotSupported;
    if (g.nxyz <= 0 || nrhs <= 0) return cudaSuccess;
    int C = 0, nch = 0;
    sweep_chunks(g.nxyz, nrhs, N, nu, &C, &nch);
    const long long nwork = (long long)nrhs * nch;
    const ModeLaunch L = mode_launch(g.nxyz, nwork);
    cudaError_t e = cudaSuccess;
#define ST_SWEEP_U(NU)                                                                          \
    if (nu == NU)                                                                               \
        ST_NT_DISPATCH(pc.nt, (e = launch_pdl(k_lv_sweep_up<T, NT, NU>, L.grid, L.block, 0, s,   \
                                              ec, uin, uout, f, inv, g.nxyz, pc, omega, N, C,    \
                                              nch, nwork)));
    ST_SWEEP_U(2) ST_SWEEP_U(3) ST_SWEEP_U(4) ST_SWEEP_U(5) ST_SWEEP_U(6)
#undef ST_SWEEP_U
    return e != cudaSuccess ? e : cudaGetLastError();
}
#undef ST_NT_DISPATCH

template cudaError_t launch_mode_inverse<double>(double *, const double *, const Grid &,
                                                 const SpecCoefs<double> &, cudaStream_t);
template cudaError_t launch_mode_inverse<float>(float *, const double *, const Grid &,
                                                const SpecCoefs<double> &, cudaStream_t);
#define ST_INST(T)                                                                              \
    template cudaError_t launch_spec_sweep_down<T>(const T *, T *, T *, const T *, const Grid &, \
                                                   const ProlongCoefs<T> &, T, int, int, int,    \
                                                   cudaStream_t);                                \
    template cudaError_t launch_spec_sweep_up<T>(const T *, const T *, T *, const T *,          \
                                                 const T *, const Grid &, const ProlongCoefs<T> &, \
                                                 T, int, int, int, cudaStream_t);                \
    template cudaError_t launch_spec_tail<T>(const T *, T *, const T *const *, int, const Grid &, \
                                             const ProlongCoefs<T> &, T, int, int, int, int,     \
                                             cudaStream_t);                                      \
    template cudaError_t launch_spec_smooth<T>(const T *, T *, const T *, const T *,            \
                                               const Grid &, int, T, int, long long, int,       \
                                               cudaStream_t);                                   \
    template cudaError_t launch_spec_down<T>(const T *, T *, const T *, T *, const T *,         \
                                             const T *, const Grid &, const SpecCoefs<T> &,     \
                                             const ProlongCoefs<T> &, T, int, long long,        \
                                             cudaStream_t);                                     \
    template cudaError_t launch_spec_up<T>(const T *, const T *, T *, const T *, const T *,     \
                                           const Grid &, const ProlongCoefs<T> &, T, int,       \
                                           long long, cudaStream_t);                            \
    template cudaError_t launch_spec_coarse<T>(T *, const T *, const T *, const Grid &, int,    \
                                               int, int, cudaStream_t);                         \
    template cudaError_t launch_spec_res_restrict<T>(const T *, const T *, T *, const T *,      \
                                                     const Grid &, const SpecCoefs<T> &,        \
                                                     const ProlongCoefs<T> &, int, long long,   \
                                                     cudaStream_t);                             \
    template cudaError_t launch_spec_op<T>(const T *, const T *, T *, const T *, const Grid &,  \
                                           const SpecCoefs<T> &, int, long long, int,           \
                                           cudaStream_t);
ST_INST(double)
ST_INST(float)
#undef ST_INST

}  // namespace st

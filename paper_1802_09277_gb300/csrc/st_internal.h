// Internal declarations shared by the CUDA translation units (not part of
// the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "dfloat.h"
#include "st_iga.h"

#include <atomic>
#include <cstdint>

struct st_handle_s;

namespace st {

// Raise a kernel's dynamic shared-memory limit to `bytes` once per device
// (the attribute belongs to the function on the current device; bit d of
// `done` records device d), safe to call from several threads.
inline cudaError_t smem_attr_once(const void *func, int bytes,
                                  std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Allocate the outer iteration's Krylov space now (st_solve would do it on
// first use); used by the server to account a setup's memory up front.
int prepare_solve(st_handle_s *h);
// st_setup with the handle's device memory taken from a stream-ordered pool
// on `stream` (released by st_destroy with cudaFreeAsync on the handle's
// stream at that time); used by the serving loop.
int setup_pooled(st_handle_s **out, int geometry, int degree, const int *spans, int slabs,
                 const st_options *opt, cudaStream_t stream, cudaMemPool_t pool);

constexpr int NTMAX = 8;  // max time dofs per slab (ne + p)
constexpr int PMAX = 3;   // max B-spline degree
constexpr int MAXV = 32;  // max vectors in one multi-vector kernel call

// Spatial grid: interior dofs per axis (unused axes 1), dimension, degree.
struct Grid {
    int nx, ny, nz;
    int dim;
    int p;
    long long nxyz;
};

// Stencil output modes of the residual kernel
enum StencilMode { MODE_RES = 0, MODE_APPLY = 1, MODE_MASS = 2 };

// Per-launch time coefficients, row-major with row stride NTMAX, converted on
// the host to the kernel's scalar type.
template <typename T>
struct TimeCoefs {
    T CK[NTMAX * NTMAX];  // multiplies M_x u_j (K_t; M_t in MODE_MASS)
    T CM[NTMAX * NTMAX];  // multiplies K_x u_j (M_t; 0 in MODE_MASS)
    T Y[NTMAX * NTMAX];   // fused forward time transform (used if fuse_y)
    int nt;
    int fuse_y;
    int mode;
    // slab partition: the last time plane of the slab before the first slab
    // of every problem ([problem][nxyz], data type of u), which then couples
    // like an interior slab; nullptr: the first slab has no predecessor
    const void *halo;
};

// Quasi-triangular Schur factor for the shift solve, plus X for the update
template <typename T>
struct SchurCoefs {
    T Z[NTMAX * NTMAX];
    T X[NTMAX * NTMAX];
    int blk[NTMAX];  // blk[i] = 1: row i is the second row of a 2x2 block
    int nt;
};

// Time factors of one level for the per-mode block solve
// (K_t + mu M_t)^{-1} = X (Z + mu I)^{-1} Y.  variant 0: real Schur (Z quasi
// triangular, X, Y real); variant 1: diagonalisation (complex eigenvalues
// lre + i lim, X = Xr + i Xi, Y = Y + i Yi).
template <typename T>
struct SpecCoefs {
    T Kt[NTMAX * NTMAX];
    T Mt[NTMAX * NTMAX];
    T Y[NTMAX * NTMAX];
    T Z[NTMAX * NTMAX];
    T X[NTMAX * NTMAX];
    T Yi[NTMAX * NTMAX];
    T Xi[NTMAX * NTMAX];
    T Zi[NTMAX * NTMAX];  // complex Schur variant: imaginary part of Z
    T lre[NTMAX];
    T lim[NTMAX];
    int blk[NTMAX];
    int nt;
    int variant;
};

template <typename T>
struct ProlongCoefs {
    T P[2 * NTMAX * NTMAX];  // (2nt x nt) row-major
    int nt;
};

// Banded 1D matrices on the device: band[a][i][o+p] = Mat_a[i][i+o].
template <typename T>
struct Bands {
    const T *M[3];
    const T *K[3];
};

// ---- launchers (kernels_stencil.cu) ----
// T: data type in HBM; C: arithmetic (T itself, or dfloat on FP64 data).
// sch: slabs per CTA of the double-float kernel (0: chosen from the grid
// size; 1, 2, 4 or 8); one slab per CTA otherwise
template <typename T, typename C = T>
cudaError_t launch_stencil(const T *u, const T *f, T *out, const Bands<T> &bands, const Grid &g,
                           const TimeCoefs<C> &tc, int slabs_per_prob, int slab0, int nslabs,
                           cudaStream_t s, int sch = 0);

// ---- launchers (kernels_transform.cu) ----
// C[b][m][n] = sum_k A(b,m,k) B(b,k,n) with arbitrary strides
template <typename T>
cudaError_t launch_gemm_strided(int batch, int M, int N, int K, const T *A, long long sAb,
                                long long sAm, long long sAk, const T *B, long long sBb,
                                long long sBk, long long sBn, T *C, long long sCb, long long sCm,
                                long long sCn, cudaStream_t s);

template <typename T>
cudaError_t launch_shift_solve(T *w, const T *lam0, const T *lam1, const T *lam2, const Grid &g,
                               const SchurCoefs<T> &sc, long long nslabs, cudaStream_t s);

template <typename T>
cudaError_t launch_update(T *u, const T *z, const SchurCoefs<T> &sc, T omega, const Grid &g,
                          long long nslabs, int overwrite, cudaStream_t s);

template <typename T>
cudaError_t launch_restrict(const T *rf, T *fc, const ProlongCoefs<T> &pc, const Grid &g,
                            long long ncoarse, cudaStream_t s);

template <typename T>
cudaError_t launch_prolong_add(const T *ec, T *uf, const ProlongCoefs<T> &pc, const Grid &g,
                               long long ncoarse, cudaStream_t s);
// y += x
template <typename T>
cudaError_t launch_add(T *y, const T *x, long long n, cudaStream_t s);

// ---- tensor-core transforms (kernels_tc.cu) ----
// kind: 2 = TF32, 1 = BF16, 3 = split TF32 (hi*hi + hi*lo + lo*hi, FP32
// accuracy); mode 0: contracted axis contiguous, 1: strided by
// `inner`.  wt = W^T row-major (n_out x n_in).  cudaErrorNotSupported when the
// shape is not covered.
cudaError_t launch_tc_axis(int kind, int mode, const float *in, float *out, const float *wt,
                           int n_in, int n_out, long long ncols, long long inner, int *err,
                           int nsm, cudaStream_t s, int ctas_per_sm = 0,
                           unsigned long long wait_ns = 1000000000ull);

// ---- eigenbasis V-cycle kernels (kernels_spectral.cu) ----
// ---- eigenbasis level kernels (kernels_modes.cu) ----
// inv: per-mode slab inverses of one level, inv[(i nt + j) nxyz + k]
// = ((K_t + mu_k M_t)^{-1})_{ij}; built by launch_mode_inverse from the FP64
// factors.  spp: slabs per problem on the level (slab pairs never straddle).
template <typename TO>
cudaError_t launch_mode_inverse(TO *inv, const double *mu64, const Grid &g,
                                const SpecCoefs<double> &c, cudaStream_t s);
// the V-cycle's coarse levels l0 .. l0 + nlev - 1 (n0 slabs per problem on
// level l0, nu1 / nu2 smoothing steps, zero start) in one launch: fin = f on
// level l0, uout = u on level l0; inv[i] = the per-mode inverses of level
// l0 + i.  cudaErrorNotSupported when n0 > 16, nlev > 16 or nu > 8
template <typename T>
cudaError_t launch_spec_tail(const T *fin, T *uout, const T *const *inv, int nlev,
                             const Grid &g, const ProlongCoefs<T> &pc, T omega, int n0, int nrhs,
                             int nu1, int nu2, cudaStream_t s);
// nu = 2..6 smoothing steps of a level in one pass (one thread per mode and
// chunk of slabs, see kernels_modes.cu): down = from u = 0, nu steps, the
// residual and its restriction into fc; up = prolongation of the coarse
// correction ec and nu steps, uin -> uout (out of place).  N = slabs per
// problem (even).  cudaErrorNotSupported outside nu = 2..6.
template <typename T>
cudaError_t launch_spec_sweep_down(const T *f, T *u, T *fc, const T *inv, const Grid &g,
                                   const ProlongCoefs<T> &pc, T omega, int N, int nrhs, int nu,
                                   cudaStream_t s);
template <typename T>
cudaError_t launch_spec_sweep_up(const T *ec, const T *uin, T *uout, const T *f, const T *inv,
                                 const Grid &g, const ProlongCoefs<T> &pc, T omega, int N,
                                 int nrhs, int nu, cudaStream_t s);
// uout = (1 - omega) uin + omega A^{-1} (f + e_0 uin_prev) (uin_zero: uin = 0)
template <typename T>
cudaError_t launch_spec_smooth(const T *uin, T *uout, const T *f, const T *inv, const Grid &g,
                               int nt, T omega, int spp, long long nslabs, int uin_zero,
                               cudaStream_t s);
// last pre-smoothing step + residual + restriction (uin == nullptr: zero
// incoming iterate); writes the smoothed slabs to uout and P_t^T r to fc
template <typename T>
cudaError_t launch_spec_down(const T *uin, T *uout, const T *f, T *fc, const T *inv,
                             const T *mu, const Grid &g, const SpecCoefs<T> &c,
                             const ProlongCoefs<T> &pc, T omega, int spp, long long ncoarse,
                             cudaStream_t s);
// uout = smooth(uin + P e) on the fine slabs of ncoarse coarse slabs
template <typename T>
cudaError_t launch_spec_up(const T *ec, const T *uin, T *uout, const T *f, const T *inv,
                           const Grid &g, const ProlongCoefs<T> &pc, T omega, int spp,
                           long long ncoarse, cudaStream_t s);
// exact solve of the coarsest level (forward substitution over its slabs)
template <typename T>
cudaError_t launch_spec_coarse(T *u, const T *f, const T *inv, const Grid &g, int nt, int spp,
                               int nprob, cudaStream_t s);
// residual of slab pairs restricted onto the coarse slabs (no smoothing)
template <typename T>
cudaError_t launch_spec_res_restrict(const T *u, const T *f, T *fc, const T *mu, const Grid &g,
                                     const SpecCoefs<T> &c, const ProlongCoefs<T> &pc, int spp,
                                     long long ncoarse, cudaStream_t s);
// res = 1: out = f - L^ u, else out = L^ u
template <typename T>
cudaError_t launch_spec_op(const T *u, const T *f, T *out, const T *mu, const Grid &g,
                           const SpecCoefs<T> &c, int spp, long long nslabs, int res,
                           cudaStream_t s);
// the whole eigenbasis V-cycle in shared memory (one launch); lvc_host: HOST
// array of the nlev levels' coefficients (passed as a kernel parameter
// block); cudaErrorNotSupported if one mode's levels do not fit in max_smem
// bytes or there are too many levels
template <typename T>
cudaError_t launch_spec_vcycle(const T *fin, T *uout, const SpecCoefs<T> *lvc_host,
                               const T *mu, const Grid &g, const ProlongCoefs<T> &pc,
                               int nlev, int N, int nrhs, int nu1, int nu2, T omega, int max_smem,
                               int nsm, cudaStream_t s);

// in place per (slab, mode): w <- (K_t + mu_k M_t)^{-1} w
template <typename T>
cudaError_t launch_mode_solve(T *w, const T *mu, const Grid &g, const SpecCoefs<T> &c,
                              long long nslabs, cudaStream_t s);

// ---- vector kernels (kernels_vector.cu) ----
template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin *x, Tout *y, long long n, cudaStream_t s);
// y = float(x) * float(scale[r]) over rhs r of len values each (one FP32 rounding
// of the conversion, one of the product)
cudaError_t launch_convert_scale(const double *x, float *y, const double *scale, int nrhs,
                                 long long len, cudaStream_t s);

// Krylov vector kernels over a group of members (handles) whose vectors hold
// different numbers of right-hand sides of different lengths.  A launch
// covers the systems s < nsys; system s is right-hand side sr[s] of member
// sm[s] (len[k] values at offset sr[s] * len[k] of member k's vectors).
// Vector v of member k is xs[v * nmem + k]; a target of member k is t[k].
// A single handle is the group of one member with systems r = 0 .. R-1, so
// every system gets the same arithmetic whatever else is in its launch.
constexpr int GH = 16;        // members of one group launch
constexpr int NSYS_MAX = 32;  // systems of one group launch
struct GLaunch {
    int nmem = 0, nsys = 0, nblk = 0;  // nblk: partial sums per system and dot
    long long len[GH] = {};
    int R[GH] = {};                    // right-hand sides of member k
    double *part[GH] = {};             // member k's partial sums: rows x R[k] x nblk
    int sm[NSYS_MAX] = {}, sr[NSYS_MAX] = {};
    int snv[NSYS_MAX] = {};            // launch_gaxpy: vectors system s uses (<= nv)
};

// out[v * nsys + s] = dot of vector v with target w over system s (FP64 sums)
template <typename T>
cudaError_t launch_gdot(const GLaunch &g, int nv, const T *const *xs, const T *const *w,
                        double *out, cudaStream_t s);
// out[v * nsys + s] = dot of vector v with itself over system s (FP64 sums)
template <typename T>
cudaError_t launch_gnorm2(const GLaunch &g, int nv, const T *const *xs, double *out,
                          cudaStream_t s);
// out[(v * 2 + t) * nsys + s] = dot of vector v with target t (t1, t2) over system s
template <typename T>
cudaError_t launch_ggram2(const GLaunch &g, int nv, const T *const *xs, const T *const *t1,
                          const T *const *t2, double *out, cudaStream_t s);
// y_s = post_s (y_s + sum_{v < snv[s]} coef[v * nsys + s] x_v)  (post NULL = 1;
// y_zero: y_s is taken as zero and not read)
template <typename T>
cudaError_t launch_gaxpy(const GLaunch &g, int nv, const T *const *xs, const double *coef,
                         T *const *y, const double *post, cudaStream_t s, bool y_zero = false);
// y1 <- post1 (y1 + sum_v c1 x_v);  y2 <- post2 (y2 + c21 y1_old + sum_v c2 x_v)
// (coefficients [v * nsys + s], scalars [s]); write1[s] = 0 leaves system
// s's y1 untouched
template <typename T>
cudaError_t launch_gaxpy2(const GLaunch &g, int nv, const T *const *xs, const double *c1,
                          const double *c2, const double *c21, const double *post1,
                          const double *post2, T *const *y1, T *const *y2, const int *write1,
                          cudaStream_t s);

// f = sum_k gt_k (x) gz_k (x) gy_k (x) gx_k, g packed per k as
// [nslab_t | nx | ny | nz] doubles
cudaError_t launch_separable_sum(double *f, const double *g, int K, long long nslab_t, int nx,
                                 int ny, int nz, cudaStream_t s);

// y (FP64) += a_r * x (FP32) per rhs r (store: y = 0 + a_r * x, y not read)
cudaError_t launch_axpy_f32_f64(const float *x, double *y, const double *a, int nrhs,
                                long long len, cudaStream_t s, bool store = false);

// y = a_r * x (per rhs), y may alias x
cudaError_t launch_scale(const double *x, double *y, const double *a, int nrhs, long long len,
                         cudaStream_t s);

template <typename T>
cudaError_t launch_zero(T *x, long long n, cudaStream_t s);

// ---- preconditioned MinRes on spatial block systems (kernels_minres.cu) ----
// Per-system scalars of the iteration (one thread per system updates them).
struct MrState {
    double beta1;           // ||r_0||_{P^{-1}}
    double eta;             // signed ||r_k||_{P^{-1}} of the QR recurrence
    double bk;              // beta_k of the Lanczos process
    double c1, s1, c2, s2;  // rotations k-1 and k-2
    double cd, cdel, ceps, cx;  // this step: 1/rho, delta, eps, c * eta_{k-1}
    double invb;            // 1 / beta_{k+1} (0 once the system stopped)
    double relres;          // ||r_k||_{P^{-1}} / ||r_0||_{P^{-1}}
    int active;             // still iterating
    int upd;                // this step updates the iterate
    int iters;              // steps taken
    int pad;
};
constexpr int MR_MAX_CHUNKS = 32;
// CTAs per system of the dot kernel for a system of len elements
int mr_dot_chunks(long long len);
template <typename T>
cudaError_t launch_seg_dot(const T *a, const T *b, double *part, long long len, int nsys,
                           cudaStream_t s);
cudaError_t launch_mr_init(const double *partB, int chunks, MrState *st, int nsys, cudaStream_t s);
template <typename T>
cudaError_t launch_mr_init_vec(T *q, T *p, const T *z, T *qp, T *d1, T *d2, T *x,
                               const MrState *st, long long len, int nsys, cudaStream_t s);
template <typename T>
cudaError_t launch_mr_lanczos(T *t, const T *q, const T *qp, const double *partA, int chunks,
                              const MrState *st, long long len, int nsys, cudaStream_t s);
// rotation of every system (state st_in -> st_out) fused with its direction,
// iterate and normalisation update
template <typename T>
cudaError_t launch_mr_step(T *p, const T *z, T *t, const T *d1, T *d2, T *x, const double *partA,
                           const double *partB, int chunks, const MrState *st_in, MrState *st_out,
                           double tol, long long len, int nsys, cudaStream_t s);
// w[sys][comp][k] /= pw_comp (mu_k + shift)  (pw (K_x + shift M_x) inverted in the eigenbasis)
template <typename T>
cudaError_t launch_fd_scale(T *w, const T *mu, double shift, double pw0, double pw1, int c,
                            long long m, int nsys, cudaStream_t s);
// compact batch <-> slab vectors (nt planes per slab): component 0 at row0 of
// src0 / dst0, component 1 (c = 2) at row1 of src1 / dst1, scaled / signed
template <typename T>
cudaError_t launch_mr_gather(const T *src0, int row0, const T *src1, int row1, T *dst, int c,
                             int nt, long long m, double sc0, double sc1, int nsys, cudaStream_t s);
template <typename T>
cudaError_t launch_mr_scatter(const T *src, T *dst0, int row0, T *dst1, int row1, int c, int nt,
                              long long m, double sg0, double sg1, int nsys, cudaStream_t s);
cudaError_t launch_mr_count(const MrState *st, int nsys, int *count, cudaStream_t s);

}  // namespace st

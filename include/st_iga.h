/*
 * st_iga.h -- C ABI of the GB300 space-time multigrid library (libst_iga.so).
 *
 * The library solves the linear system L_h u = f of the space-time
 * discontinuous-Galerkin isogeometric (SUPG, "time-upwind") discretisation of
 * the heat equation  d_t u - Laplace u = f  on (0,1)^d x (0,T), u = 0 on the
 * spatial boundary, u(0) = 0 (Hofer, Langer, Neumueller, arXiv:1802.09277,
 * Eq. 1.1 and Sec. 2.2-2.3).  L_h is block lower bidiagonal over N time slabs
 * (Eq. 2.4): diagonal blocks A_n = K_t (x) M_x + M_t (x) K_x (Eq. 2.5, time
 * matrices Eq. 2.6) and sub-diagonal blocks -B_n = -N_t (x) M_x.
 *
 * The solver is the time-parallel multigrid of Sec. 3.1: damped block-Jacobi
 * smoothing u <- u + omega D^{-1} (f - L_h u), D = blockdiag(A_n), where each
 * A_n^{-1} is applied through the factorisation of Eq. 3.1,
 *   A^{-1} = (X (x) I) (Z (x) M_x + I (x) K_x)^{-1} (Y (x) I),  Y = (M_t X)^{-1},
 * with (X, Z) the real Schur factors of M_t^{-1} K_t (Sec. 3.5, Eq. 3.5), and
 * the spatial problems K_x + z M_x solved exactly by fast diagonalisation in
 * the generalized eigenbasis of the 1D matrices (K1 U = M1 U Lambda,
 * U^T M1 U = I).  Time coarsening merges slab pairs.  The V-cycle
 * preconditions an FP64 FGMRES (or is iterated directly).
 *
 * Conventions for every entry point:
 *  - Vectors are FP64 DEVICE pointers, owned by the caller, never freed or
 *    retained by the library, laid out as v[rhs][slab][t][z][y][x] (x fastest;
 *    unused axes have extent 1).  Length = st_sizes().n_dofs.
 *  - All device work is enqueued on the handle's CUDA stream (st_setup /
 *    st_set_stream).  Calls returning results to the host (st_solve's info,
 *    st_last_error) synchronise that stream; the others do not.
 *  - Every function returns ST_OK (0) or a negative ST_ERR_* code; the
 *    message of the last failure on the calling thread is st_last_error().
 *    No C++ exception crosses this interface.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef ST_IGA_H
#define ST_IGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ST_OK                   0
#define ST_ERR_INVALID_ARG     -1  /* bad pointer, size, option or geometry      */
#define ST_ERR_OOM             -2  /* device allocation failed                   */
#define ST_ERR_NOT_POSITIVE    -3  /* Re lambda(K_t, M_t) <= 0 (Sec. 3.2 remark: use smaller theta) */
#define ST_ERR_ILL_CONDITIONED -4  /* a time or space factorisation failed its residual check */
#define ST_ERR_NO_CONVERGENCE  -5  /* iteration cap reached above the tolerance  */
#define ST_ERR_TIMEOUT         -6  /* a bounded device wait ran out              */
#define ST_ERR_CUDA            -7  /* a CUDA runtime call failed                 */
#define ST_ERR_OVER_BUDGET     -8  /* request exceeds the HBM budget             */
#define ST_ERR_UNSUPPORTED     -9  /* valid but not built (e.g. degree > 3)      */
#define ST_ERR_COMM           -12  /* a communication callback of a partitioned handle failed */

/* geometry: the spatial domain (0,1)^d */
#define ST_INTERVAL 1
#define ST_SQUARE   2
#define ST_CUBE     3

/* factorisation of M_t^{-1} K_t used for the slab solves (Eq. 3.1) */
#define ST_RSCHUR 0  /* real Schur form, 2x2 blocks for complex pairs (Sec. 3.5)   */
#define ST_EIG    1  /* diagonalisation with complex eigenvalues (Sec. 3.3); setup
                        fails with ST_ERR_ILL_CONDITIONED if cond(X) > 1e8        */
#define ST_CSCHUR 2  /* complex Schur form, triangular solve with complex shifts
                        (Sec. 3.4, Algorithm 1)                                   */

/* precision of the multigrid preconditioner (the outer iteration is FP64) */
#define ST_FP64        0  /* everything FP64                                  */
#define ST_MIXED_FP32  1  /* V-cycle in FP32 (CUDA cores), FP64 outer          */
#define ST_MIXED_TF32  2  /* V-cycle FP32, spatial transforms on TF32 tensor cores */
#define ST_MIXED_BF16  3  /* V-cycle FP32, spatial transforms on BF16 tensor cores */

/* basis of the V-cycle (both give the same iterates up to rounding) */
#define ST_BASIS_NODAL    0 /* B-spline basis: every smoothing step computes the
                               residual with the banded 1D matrices and applies
                               A_n^{-1} by time transform, spatial transforms,
                               shift solve, inverse transforms (Sec. 3.1, Eq. 3.1) */
#define ST_BASIS_SPECTRAL 1 /* spatial eigenbasis: the spatial transforms are
                               applied once on entry and once on exit of the
                               V-cycle; they commute with the time-only
                               coarsening and the block-Jacobi smoother, and in
                               between every operator is pointwise in the mode */

/* spatial solves K_x + z M_x inside each slab inverse of the B-spline-basis
 * V-cycle (option spatial_solver) */
#define ST_SPATIAL_FD     0 /* exact: fast diagonalisation in the generalized
                               eigenbasis of the 1D matrices (default)       */
#define ST_SPATIAL_MINRES 1 /* inexact (Sec. 3.3-3.5, Theorems 3.2/3.3).
                               ST_RSCHUR: the real Schur form's 2x2 blocks
                               are standardised to [[alpha, beta1], [beta2,
                               alpha]]; Algorithm 1 runs over its diagonal
                               blocks from the last to the first, every 2x2
                               block's spatial system solved by MinRes
                               preconditioned by Theorem 3.3's block-diagonal
                               P (P^{-1} by fast diagonalisation) to
                               minres_tol, every 1x1 block (SPD, its own
                               preconditioner) by one application of P^{-1}.
                               ST_EIG / ST_CSCHUR: complex time transforms
                               (real and imaginary parts as separate
                               vectors), Algorithm 1 over the rows of the
                               diagonal / upper triangular T, every complex
                               shift alpha + i beta by MinRes in Theorem 3.2's
                               form (twice the work of ST_RSCHUR: a conjugate
                               pair is two complex solves).  Needs
                               ST_BASIS_NODAL; the V-cycle is then inexact,
                               so pair it with ST_OUTER_FGMRES (flexible)   */

/* outer iteration */
#define ST_OUTER_FGMRES 0 /* FGMRES(restart), right-preconditioned by one V-cycle */
#define ST_OUTER_MG     1 /* multigrid iteration u <- u + V(f - L u)             */
#define ST_OUTER_IR     2 /* mixed modes: iterative refinement, FP64 residual and
                             update around FGMRES on FP32 vectors (FP32 operator,
                             FP32 V-cycle) solved to inner_tol; FP64 handles
                             fall back to ST_OUTER_FGMRES                       */

typedef struct st_handle_s *st_handle;

typedef struct {
    double T;             /* final time (default 1)                              */
    double theta;         /* SUPG parameter theta_n, all slabs (default 1)       */
    double omega;         /* block-Jacobi damping (default 0.5, Sec. 3.1)        */
    int ne_per_slab;      /* time elements per slab (default 2)                  */
    int nu1, nu2;         /* pre/post smoothing steps (default 1, 1)             */
    int precision;        /* ST_FP64 / ST_MIXED_*                                */
    int outer;            /* ST_OUTER_FGMRES / ST_OUTER_MG                       */
    int gmres_restart;    /* FGMRES restart length (default 20)                  */
    int max_it;           /* outer iteration cap (default 200)                   */
    int nrhs;             /* independent right-hand sides solved together (1)    */
    size_t hbm_budget;    /* bytes the handle may allocate; 0 = unlimited        */
    int basis;            /* ST_BASIS_NODAL (default) / ST_BASIS_SPECTRAL         */
    double inner_tol;     /* ST_OUTER_IR: inner relative tolerance (default 1e-4) */
    int use_graphs;       /* 1 (default): replay each preconditioner application
                             inside st_solve as a captured CUDA graph            */
    int variant;          /* ST_RSCHUR (default) / ST_EIG                          */
    int autotune;         /* 1 (default): the first st_solve times the candidate
                             kernels of each spatial transform and keeps the
                             fastest (see st_autotune)                          */
    int fused_vcycle;     /* 0 (default): ST_BASIS_SPECTRAL runs the V-cycle
                             level by level (one launch per step); 1: the whole
                             V-cycle in one shared-memory kernel per block of
                             spatial modes when a mode's levels fit            */
    int spatial_solver;   /* ST_SPATIAL_FD (default) / ST_SPATIAL_MINRES         */
    double minres_tol;    /* ST_SPATIAL_MINRES: reduction of ||r||_{P^{-1}} per
                             block solve (default 1e-4, the inner tolerance of
                             the paper's multigrid runs, Sec. 4.4)            */
    int minres_maxit;     /* ST_SPATIAL_MINRES: MinRes steps per block solve;
                             0 (default) = the count after which the MinRes
                             bound for cond(P^{-1} A) <= sqrt 2 guarantees
                             minres_tol, 2 ceil(ln(tol/2) / ln(3 - 2 sqrt 2))
                             (12 for 1e-4).  Systems that converge earlier
                             stop updating; the steps always run, so the
                             smoother replays as one CUDA graph             */
    double space_ratio;   /* 0 (default): coarsen in time only (slab pairs).
                             > 0 (ST_BASIS_NODAL): before merging slabs, halve
                             every axis' spans while the level's
                             tau / h_x^2 (slab length over the square of the
                             largest element) exceeds space_ratio and the
                             spans stay even and >= 4 (Sec. 3.1's multigrid
                             coarsens in space and time; the rule is ours):
                             space levels keep the slabs, prolongation
                             P = I (x) P_z (x) P_y (x) P_x by B-spline knot
                             insertion, restriction P^T, coarse operators
                             rediscretised on the coarse grid (= Galerkin,
                             the spaces are nested)                          */
} st_options;

typedef struct {
    int iterations;       /* Krylov / multigrid iterations (V-cycles) taken      */
    int refinements;      /* ST_OUTER_IR: FP64 refinement steps (else 0)          */
    int status;           /* ST_OK or ST_ERR_NO_CONVERGENCE                      */
    double rel_residual;  /* max over rhs of ||f - L u||_2 / ||f||_2 (FP64)       */
    double seconds;       /* wall time of the solve, host clock                 */
    int host_syncs;       /* host synchronisations to read reductions back      */
    int vector_launches;  /* Krylov vector-kernel launches (dots, updates); for
                             st_solve_group both count the whole group's calls */
} st_solve_info;

/* Fill *opt with the defaults listed above. */
void st_options_default(st_options *opt);

/* Build a handle: B-spline bases (Sec. 2.1), the 1D matrices M1, K1 (after
 * Eq. 2.5) and per multigrid level K_t, M_t (Eq. 2.6, theta*h frozen at the
 * finest value on coarse levels), the real Schur factors of M_t^{-1} K_t with
 * Y = (M_t X)^{-1} (Sec. 3.2, 3.5), the generalized eigenpairs of (K1, M1),
 * and the time prolongation of two slabs onto one (Sec. 3.1); uploads them and
 * allocates all device work buffers.
 *   geometry : ST_INTERVAL / ST_SQUARE / ST_CUBE (d = 1, 2, 3)
 *   degree   : B-spline degree p in space and time, 1..3
 *   spans    : d knot-span counts (x, y, z), each >= 2; n = spans + p - 2
 *              interior dofs per axis (Dirichlet ends removed)
 *   slabs    : number N of time slabs, >= 1
 *   opt      : options (NULL = defaults)
 *   stream   : cudaStream_t to enqueue on (NULL = legacy default stream)
 * Errors: INVALID_ARG, UNSUPPORTED, NOT_POSITIVE (Re lambda <= 0 on some
 * level), ILL_CONDITIONED, OVER_BUDGET, OOM, CUDA.  *out is NULL on error. */
int st_setup(st_handle *out, int geometry, int degree, const int *spans,
             int slabs, const st_options *opt, void *stream);

/* Same as st_setup but builds only the host-side FP64 factors (no CUDA call,
 * no device memory): st_sizes, st_time_factors, st_space_factors and
 * st_time_prolongation work on such a handle, every entry point that touches
 * device vectors returns ST_ERR_INVALID_ARG.  Usable on a machine without a
 * GPU. */
int st_setup_host(st_handle *out, int geometry, int degree, const int *spans,
                  int slabs, const st_options *opt);

/* Release every device and host resource of the handle (NULL is a no-op). */
void st_destroy(st_handle h);

/* Change the stream later calls enqueue on. */
int st_set_stream(st_handle h, void *stream);

/* Sizes: total dofs (all rhs), time dofs per slab N_t = ne + p, interior
 * dofs per axis (3 entries, unused axes 1), number of multigrid levels and
 * device bytes held by the handle.  Any output pointer may be NULL. */
int st_sizes(st_handle h, int64_t *n_dofs, int *n_t, int *n_x_per_axis,
             int *n_levels, size_t *device_bytes);

/* y = L_h x (Eq. 2.4), matrix-free through the Kronecker factors of
 * Eq. 2.5 (FP64).  x, y: device, n_dofs each, must not alias. */
int st_apply(st_handle h, const double *x, double *y);

/* r = f - L_h u (FP64).  u, f, r: device, n_dofs each; r must not alias u. */
int st_residual(st_handle h, const double *u, const double *f, double *r);

/* r = f - L_h u (Eq. 2.4, through the Kronecker factors of Eq. 2.5) on FP64
 * data in double-float arithmetic: every value a pair of FP32 numbers
 * hi + lo (about 48 significant bits), products summed by compensated Dot2
 * sums.  This is the residual the ST_OUTER_IR refinement takes at every step
 * of a mixed-precision handle, here on any handle; it agrees with
 * st_residual to about 1e-14 relative.  u, f, r: device, n_dofs each; r must
 * not alias u.  slabs_per_cta: 0 lets the library choose how many
 * consecutive slabs one CTA of the tiled kernel handles (several on large
 * grids: the coupling plane B_n u_{n-1} of a CTA's later slabs is then taken
 * from the slab before instead of recomputed); 1, 2, 4 or 8 sets it.  The
 * result has the same bits for every value.  The 3D p = 3 residual marches
 * in z, one slab per CTA, and ignores it.  Errors: ST_ERR_INVALID_ARG for a
 * null or host-only handle, a null pointer, aliasing or another
 * slabs_per_cta; ST_ERR_CUDA if a launch fails. */
int st_residual_df(st_handle h, const double *u, const double *f, double *r, int slabs_per_cta);

/* Load vector of a source given by its B-spline coefficients in the trial
 * basis of every slab: f = (M_t (x) M_x) c, which is l_h(phi_i) of Sec. 2.3
 * exactly (u0 = 0).  c, f: device, n_dofs each, must not alias. */
int st_load_coeffs(st_handle h, const double *c, double *f);

/* Load vector of a source made of space-time Gaussian bumps,
 *   f(x, t) = sum_k amps[k] exp(-|(x, t) - c_k|^2 / (2 widths[k]^2)),
 * l_h(phi_i) of Sec. 2.3 by Gauss-Legendre quadrature with 2p + 4 points per
 * element (every bump is a product of 1D functions).  centers: HOST,
 * nbumps x (d + 1) in (x, y, z, t) order; widths, amps: HOST, nbumps each;
 * f: DEVICE, n_dofs (every rhs gets the same source).  Synchronises. */
int st_load_gaussians(st_handle h, int nbumps, const double *centers, const double *widths,
                      const double *amps, double *f);

/* nsteps damped block-Jacobi steps on the finest level (Sec. 3.1):
 * u <- u + omega D^{-1}(f - L_h u), A_n^{-1} applied through Eq. 3.1.
 * Runs in the handle's precision (FP32 inside for the mixed modes, u and f
 * stay FP64 at the interface).  u: in/out, f: in, device, n_dofs each. */
int st_smooth(st_handle h, double *u, const double *f, int nsteps);

/* Bound on each device-side wait of the tensor-core transforms (the wait for
 * an MMA group's completion signal), in seconds: 0 <= seconds <= 60, default
 * 1.  When a wait runs out, the kernel records it, waits (bounded) for its
 * MMAs in flight, frees its tensor memory and returns, and the next
 * st_solve / st_vcycle returns ST_ERR_TIMEOUT; the handle stays usable.
 * 0 makes every such wait a single test of the signal (for fault-handling
 * tests).  Errors: INVALID_ARG (null handle, out of range). */
int st_set_wait_limit(st_handle h, double seconds);

/* Allocation-free smoothing steps.  The paper has no counterpart: this is a
 * deployment variant of st_smooth for callers that cannot allocate device
 * memory -- for example a host application whose memory pool already owns
 * the GPU's memory, or code that runs where a cudaMalloc would stall or is
 * forbidden, such as a real-time control loop.  Such a caller builds the
 * factors with st_setup_host (no device memory), allocates u and f itself,
 * and calls this function; it performs nsteps FP64 damped block-Jacobi
 * steps exactly like st_smooth on an FP64 handle.  Its two work vectors and
 * the uploaded 1D factors live in one file-scope static device array of
 * ST_STATIC_SCRATCH_BYTES (about 9.7 MB) that every GPU which loads the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *   h      : a handle from st_setup or st_setup_host with variant ST_RSCHUR
 *            and spatial_solver ST_SPATIAL_FD (any other variant or spatial
 *            solver: ST_ERR_UNSUPPORTED before any copy or launch); only its
 *            host factors are read, its precision option is ignored (the
 *            steps run in FP64)
 *   u, f   : device, n_dofs doubles each (u in/out), must not alias
 *   stream : cudaStream_t for all work of this call (NULL = default stream)
 * Limits: n_dofs <= ST_STATIC_MAX_DOFS and at most ST_STATIC_MAX_N interior
 * dofs per axis, else ST_ERR_INVALID_ARG.  The first call on a device looks
 * up the static array's device address with that device current; make that
 * first call before any stream capture.  Every call uploads the handle's 1D
 * factors (at most about 1.3 MB) into the array and reuses the same work space,
 * which keeps the last call's contents: calls that overlap on the GPU (other
 * streams or threads) race with each other. */
#define ST_STATIC_MAX_DOFS 524288
#define ST_STATIC_MAX_N    160
#define ST_STATIC_SCRATCH_BYTES (8 * (2 * ST_STATIC_MAX_DOFS + 3 * (2 * ST_STATIC_MAX_N * 7 + 2 * ST_STATIC_MAX_N * ST_STATIC_MAX_N + ST_STATIC_MAX_N)))
int st_smooth_static(st_handle h, double *u, const double *f, int nsteps, void *stream);

/* Inexact spatial block solve of Sec. 3.5 (Theorem 3.3) on the handle's
 * spatial grid, in FP64 whatever the handle's precision: for nsys
 * independent right-hand sides
 *   [[K_x + alpha M_x, beta1 M_x], [beta2 M_x, K_x + alpha M_x]] [x; y] = [f; g]
 * is rescaled to the symmetric indefinite matrix
 *   Abar = [[|beta2| Kc, -beta1 |beta2| M_x], [|beta1| beta2 M_x, -|beta1| Kc]],
 *   Kc = K_x + alpha M_x, acting on [x; -y] with right-hand side
 *   [|beta2| f; |beta1| g], and solved by MinRes preconditioned by
 *   P = diag(|beta2| (K_x + s M_x), |beta1| (K_x + s M_x)),
 *   s = alpha + sqrt|beta1 beta2| (cond(P^{-1} Abar) <= sqrt 2), with P^{-1}
 * applied by fast diagonalisation.  A complex shift alpha + i beta
 * (Theorem 3.2, Sec. 3.3/3.4) is the case beta1 = -beta, beta2 = beta:
 * (K_x + (alpha + i beta) M_x)(x + i y) = f + i g.
 *   alpha > 0, beta1 * beta2 < 0 (a complex pair), else ST_ERR_INVALID_ARG
 *   f      : device, nsys x 2 x n_x doubles ([sys][f then g][x fastest],
 *            n_x = spatial dofs), not modified
 *   u      : device, same layout: x then y of every system (output; must not
 *            alias f)
 *   tol    : stop a system once ||r_k||_{P^{-1}} <= tol ||r_0||_{P^{-1}}
 *            (zero initial guess)
 *   maxit  : step cap per system (0 = the bound's count for tol, as minres_tol)
 *   iters, relres : host arrays of nsys (may be NULL): steps taken and the
 *            final ||r_k||_{P^{-1}} / ||r_0||_{P^{-1}} of each system
 * 1 <= nsys <= 32767.  Allocates and frees its own work space (9 vectors of
 * the batch), synchronises the handle's stream, and returns
 * ST_ERR_NO_CONVERGENCE (u holds the last iterates) when a system stopped at
 * maxit above tol. */
int st_block_minres(st_handle h, double alpha, double beta1, double beta2, const double *f,
                    double *u, int nsys, double tol, int maxit, int *iters, double *relres);

/* One V-cycle on L_h u = f starting from u (in/out), precision as above. */
int st_vcycle(st_handle h, double *u, const double *f);

/* Solve L_h u = rhs to ||rhs - L_h u||_2 <= tol ||rhs||_2 per right-hand
 * side with the outer iteration of opt.outer, zero initial guess when
 * use_guess == 0 (else u holds the guess).  rhs, u: device, n_dofs.
 * info may be NULL.  Returns ST_ERR_NO_CONVERGENCE (u holds the last
 * iterate) when max_it is reached. */
int st_solve(st_handle h, const double *rhs, double tol, double *u,
             int use_guess, st_solve_info *info);

/* Solve the problems of n handles together (batching of uneven requests):
 * the handles may differ in geometry, degree, spans, slabs and nrhs; each
 * must be a mixed-precision handle with ST_OUTER_IR (the refinement of
 * Sec. 3.1's outer solve around FP32 FGMRES, as st_solve runs it), not
 * slab-partitioned, and all must share gmres_restart.  The members'
 * refinement and Krylov iterations advance in lockstep: every Krylov vector
 * operation of the members still iterating (Gram products and their
 * reduction, the basis updates, the solution update) is ONE launch over all
 * their right-hand sides, read back with one host synchronisation for the
 * whole group, while each member's operator, V-cycle, transforms and FP64
 * residual run on a stream of their own so that they overlap on the device.
 * Every loop bound is kept per member and every decision per right-hand
 * side, so each right-hand side gets exactly the result st_solve gives it on
 * its own handle.
 *   hs        : n distinct handles, 1 <= n <= 16, at most 32 right-hand sides
 *               in all (the sum of their nrhs)
 *   rhs, u    : n device pointers each, member k's n_dofs doubles (u: the
 *               solution; the initial guess when use_guess != 0)
 *   info      : n entries (may be NULL): member k's iterations, refinements,
 *               residual and status; seconds = the group's wall time
 * Work is queued on member 0's stream (and on internal streams ordered after
 * it and after each member's own stream); the call returns with every
 * member's work complete and its stream unchanged.  Errors: INVALID_ARG,
 * UNSUPPORTED (a member of another kind), those of st_solve;
 * NO_CONVERGENCE if any member stopped at max_it (its info says which; the
 * others hold their solutions). */
int st_solve_group(int n, const st_handle *hs, const double *const *rhs, double tol,
                   double *const *u, int use_guess, st_solve_info *info);

/* st_solve on HOST buffers for a stream of nbatch batches of the handle's
 * systems (each batch: nrhs right-hand sides, st_solve's layout; batch k at
 * offset k x n_dofs doubles).  Batch k solves on the handle's stream while
 * batch k+1's right-hand sides are copied to the device and batch k-1's
 * solutions back to the host, each on a stream of its own, so the transfers
 * hide behind the solves but for the first copy in and the last copy out.
 * The copies back are issued in 256 MB chunks at the solve's host
 * synchronisation points, one chunk in flight at a time: a bulk
 * device-to-host transfer would hold up the solve's own small reads of its
 * dot products (with use_guess the copy of a slot is issued in full before
 * its guess is copied in).
 *   rhs  : host, nbatch x n_dofs doubles, not modified
 *   u    : host, nbatch x n_dofs doubles: the solutions (output); the initial
 *          guesses when use_guess != 0 (else zero guesses)
 *   info : may be NULL; iterations, refinements and rel_residual are the
 *          maxima over the batches, seconds the wall time of the whole call
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister) lets the copies
 * overlap the solves; pageable memory works, each copy then blocks the host.
 * On first use allocates two device staging slots per vector (4 x n_dofs
 * doubles, counted against hbm_budget, kept until st_destroy) and two copy
 * streams.  Returns after every copy has completed.  Errors: those of
 * st_solve; INVALID_ARG (nbatch < 1, null, aliased or device pointers);
 * OVER_BUDGET / OOM for the staging slots.  A batch that fails (e.g.
 * ST_ERR_NO_CONVERGENCE) ends the call: the solutions of the batches before
 * it are in u, its own and the later ones are not written.  st_solve_history
 * then describes the last batch solved. */
int st_solve_host(st_handle h, int nbatch, const double *rhs, double tol, double *u,
                  int use_guess, st_solve_info *info);

/* Residual history of the last st_solve on the handle: the FP64 relative
 * residual ||f - L u||_2 / ||f||_2 (max over the right-hand sides) as the
 * solver recomputes it -- at the start of every FGMRES cycle, every
 * multigrid iteration, every refinement step of ST_OUTER_IR -- with the
 * (inner) iteration count at which it was taken; the last entry is the
 * final residual.  Copies up to cap entries into its / res (either may be
 * NULL) and stores the number of entries in *n.  Host only, no device work.
 * Errors: INVALID_ARG (null handle, cap < 0). */
int st_solve_history(st_handle h, int cap, int *its, double *res, int *n);

/* Per-kernel-class device timing for measurement.  While enabled, every
 * kernel launch of the handle is bracketed by CUDA events on the handle's
 * stream and its algorithmic bytes and flops (counted from the launch sizes:
 * each input and output vector once, the arithmetic of the method, no halo
 * or tile overhead) are accumulated per class.  st_profile(h, 1) resets and
 * starts, st_profile(h, 0) stops; both synchronise the stream.
 * st_profile_read returns launches, summed device milliseconds, bytes and
 * flops of one class; it synchronises the stream. */
#define ST_PROF_STENCIL64 0  /* residual / operator / load vector, FP64      */
#define ST_PROF_STENCIL32 1  /* residual (+ fused forward time transform), FP32 */
#define ST_PROF_GEMM64    2  /* spatial transform (one axis), FP64, CUDA cores */
#define ST_PROF_GEMM32    3  /* spatial transform (one axis), FP32, CUDA cores */
#define ST_PROF_SHIFT     4  /* quasi-triangular shift solve per mode        */
#define ST_PROF_UPDATE    5  /* backward time transform + damped update      */
#define ST_PROF_TRANSFER  6  /* time restriction / prolongation             */
#define ST_PROF_VECTOR    7  /* Krylov updates, scaling, precision conversion */
#define ST_PROF_DOT       8  /* Krylov dot products (deterministic reduction) */
#define ST_PROF_TC        9  /* spatial transform (one axis), tensor cores    */
#define ST_PROF_SPEC     10  /* eigenbasis smoothing step / coarse solve      */
#define ST_PROF_STENCILDF 11 /* refinement residual, double-float on FP64 data */
#define ST_PROF_MINRES   12  /* MinRes block solves: dots, Lanczos and update
                                vectors, rotations, preconditioner scaling,
                                gathers / scatters (its operator applications
                                and transforms count in their own classes)  */
#define ST_PROF_NCLASS   13
int st_profile(st_handle h, int enable);
int st_profile_read(st_handle h, int cls, int64_t *launches, double *ms,
                    double *bytes, double *flops);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of many solves (no counterpart in the paper,
 * which solves one problem at a time).  A server owns W worker threads, each
 * with its own CUDA stream, so solves of different requests overlap on the
 * GPU.  A free worker takes the oldest pending request together with up to
 * max_batch - 1 further pending requests of the same configuration
 * (geometry, degree, spans, slabs, tolerance) and solves them as one
 * multi-right-hand-side problem (opt.nrhs = the batch size rounded up to a
 * power of two, the unused right-hand sides zero; every right-hand side is
 * refined independently, so its result does not depend on the batch).
 * Setups (factors + work space, st_setup) are cached per configuration and
 * batch-size class and evicted least-recently-used; their device memory
 * comes from a stream-ordered memory pool of the server, so building or
 * releasing one never synchronises the device, and no lock is held while a
 * setup is built or released.  A batch is admitted only when its setup and
 * vectors fit the HBM budget; otherwise it waits for running solves to
 * release memory (or fails with ST_ERR_OVER_BUDGET if it cannot fit even on
 * an idle server).  st_serve_opts_default turns opt.autotune off (tuning
 * would time kernels for every new configuration on the serving path).
 * ------------------------------------------------------------------------ */
typedef struct st_server_s *st_server;

typedef struct {
    size_t hbm_budget;    /* device bytes the server may hold; 0 = 90% of the free memory */
    int workers;          /* concurrent solves (default 4)                          */
    int max_batch;        /* right-hand sides per batched solve, 1..32 (default 8)  */
    st_options opt;       /* solver options for every request (nrhs is set per batch) */
    int start_paused;     /* 1: workers take no request until st_serve_resume, so a
                             whole mix can be queued before batches are formed
                             (deterministic batching); default 0                */
    long long batch_dofs; /* a batch grows only while its total dofs stay within
                             this (the oldest request always runs): large solves
                             already saturate the GPU and only wait longer in a
                             batch; 0 = no limit; default 8388608.  A group's
                             total dofs stay within it too                      */
    int group_members;    /* up to this many configurations (each with its batch,
                             oldest first, none with more dofs per request than
                             the oldest request's, so a group never delays it)
                             are solved together by one st_solve_group call:
                             one launch per Krylov vector operation and one host
                             synchronisation per reduction for all of them, the
                             members' V-cycles overlapping (at most 32 right-hand
                             sides in all); 1 = every batch alone; default 8;
                             used when opt is mixed precision with ST_OUTER_IR */
} st_server_opts;

typedef struct {
    int geometry, degree; /* as st_setup                                          */
    int spans[3];         /* first `geometry` entries used                        */
    int slabs;
    const double *rhs;    /* HOST pointer, n_dofs doubles; copied by st_serve_submit */
    int rhs_is_coeffs;    /* 1: rhs holds B-spline coefficients c and the load
                             vector (M_t (x) M_x) c is formed on the device      */
    double tol;           /* relative residual tolerance                          */
} st_request;

#define ST_ERR_NOT_READY -10  /* st_serve_poll: the request is still pending */
#define ST_ERR_CANCELLED -11  /* st_serve_cancel removed the request before it ran */

typedef struct {
    int status;           /* ST_OK or the solve's error code                      */
    int iterations, refinements;
    double rel_residual;
    double queue_seconds; /* submit -> admitted                                   */
    double solve_seconds; /* admitted -> solution on the host                     */
    double latency_seconds; /* submit -> solution on the host                     */
    int batch_size;       /* requests of this configuration solved with it (incl. itself) */
    int64_t n_dofs;
    char error[128];      /* message of a failure ("" on success)              */
    int group_requests;   /* requests in the same solve call (all configurations) */
    int host_syncs;       /* of that call (st_solve_info.host_syncs)             */
    int vector_launches;  /* of that call (st_solve_info.vector_launches)        */
} st_result;

void st_serve_opts_default(st_server_opts *o);
/* Start the worker threads.  Errors: INVALID_ARG, CUDA. */
int st_serve_start(st_server *out, const st_server_opts *o);
/* Queue a request (its rhs is copied before returning); *ticket identifies it.
 * Errors: INVALID_ARG (bad sizes), UNSUPPORTED. */
int st_serve_submit(st_server s, const st_request *req, uint64_t *ticket);
/* Let the workers take requests again after start_paused = 1 or
 * st_serve_pause (no effect otherwise).  Errors: INVALID_ARG (null server). */
int st_serve_resume(st_server s);
/* Stop the workers from taking further requests until st_serve_resume:
 * submitted requests queue (so batches of equal configurations can form
 * from the whole queue); batches already taken run to the end.
 * Errors: INVALID_ARG (null server). */
int st_serve_pause(st_server s);
/* Withdraw a request that no worker has taken yet: its result becomes ready
 * with status ST_ERR_CANCELLED and no solution.  Returns ST_OK when it was
 * withdrawn, ST_ERR_NOT_READY when a worker is already solving it (it then
 * completes normally), ST_ERR_INVALID_ARG for an unknown or finished ticket. */
int st_serve_cancel(st_server s, uint64_t ticket);
/* Non-blocking: ST_ERR_NOT_READY while pending; otherwise fills *res, copies
 * the solution (n_dofs doubles) into u_host if it is not NULL, releases the
 * request and returns ST_OK (the request's own status is res->status). */
int st_serve_poll(st_server s, uint64_t ticket, st_result *res, double *u_host);
/* As st_serve_poll but blocks up to timeout_s seconds (< 0: no limit). */
int st_serve_wait(st_server s, uint64_t ticket, double timeout_s, st_result *res, double *u_host);
/* Finish queued work, stop the workers, free every device and host resource. */
int st_serve_stop(st_server s);

/* ------------------------------------------------------------------------
 * Slab partition over several processes (one GPU each).  The smoother of
 * Sec. 3.1 is block Jacobi over the time slabs, so every slab is smoothed on
 * its own; the only coupling of the operator is B_n u_{n-1} = (N_t (x) M_x)
 * u_{n-1} of Eq. 2.4, which reads the last time plane of the previous slab.
 * A partitioned handle holds a contiguous range of slabs of every
 * right-hand side: before each residual or smoothing step on a partitioned
 * level it receives that one plane (N_x values per right-hand side) from the
 * previous rank and sends its own last plane to the next.  The time
 * coarsening merges slab pairs on each rank until a rank holds one slab; that
 * level is gathered on every rank and the rest of the V-cycle runs there
 * redundantly (the coarse levels are small), so a V-cycle gives the same bits
 * as on one process.  The Krylov dot products are summed over the ranks.
 * All entry points on a partitioned handle are collective: every rank calls
 * them in the same order with its own slabs of u, f (layout as st_setup,
 * n_dofs = the local slabs).
 * ------------------------------------------------------------------------ */
typedef struct {
    int rank, size;      /* this process and the number of processes         */
    int host_buffers;    /* 1: the callbacks below take HOST buffers (the
                            library stages device data through pinned host
                            memory and synchronises its stream first); 0:
                            DEVICE buffers, stream-ordered on `stream`      */
    void *ctx;           /* passed to every callback                          */
    /* send `bytes` bytes of `send` to rank dst and receive `bytes` bytes from
     * rank src into `recv` (dst / src = -1: no send / receive); must not
     * deadlock when every rank sends to rank + 1 and receives from rank - 1 */
    int (*sendrecv)(void *ctx, const void *send, int dst, void *recv, int src, size_t bytes,
                    void *stream);
    /* recv (size * bytes bytes) = every rank's `send` block, in rank order   */
    int (*allgather)(void *ctx, const void *send, void *recv, size_t bytes, void *stream);
    /* in-place sum over the ranks of `count` HOST doubles (blocking); every
     * rank must receive the same bits                                        */
    int (*allreduce_sum)(void *ctx, double *vals, size_t count);
} st_comm;
/* Every callback returns 0 on success; anything else makes the calling entry
 * point fail with ST_ERR_COMM. */

/* Partitioned setup: rank r of `comm->size` holds slabs
 * [r * slabs_global / size, (r + 1) * slabs_global / size) of every
 * right-hand side.  slabs_global / size must be a power of two >= 2 (the
 * local time coarsening ends at one slab per rank); opt as st_setup with
 * basis ST_BASIS_NODAL, spatial_solver ST_SPATIAL_FD, space_ratio 0 and
 * fused_vcycle 0 (else ST_ERR_UNSUPPORTED); CUDA graphs are not used (the
 * exchanges run on the host).  The comm struct is copied; its ctx must stay
 * valid until st_destroy.  Errors: as st_setup, INVALID_ARG for a bad comm
 * or slab count. */
int st_setup_partitioned(st_handle *out, int geometry, int degree, const int *spans,
                         int slabs_global, const st_options *opt, const st_comm *comm,
                         void *stream);
/* The partition of slabs_global slabs over `size` ranks, as
 * st_setup_partitioned makes it (host only): rank's first slab, its slab
 * count and the first level that is gathered on every rank.  INVALID_ARG if
 * it cannot be partitioned. */
int st_partition_plan(int slabs_global, int size, int rank, int *slab_begin, int *slabs_local,
                      int *gathered_level);
/* NCCL communication for st_setup_partitioned: device buffers, stream-ordered
 * NCCL send/receive, all-gather and all-reduce on `stream`.  libnccl.so.2 is
 * loaded at run time (ST_ERR_UNSUPPORTED if it cannot be).  unique_id: 128
 * bytes from st_comm_nccl_unique_id on one rank, given to every rank.
 * st_comm_nccl_destroy releases the communicator. */
int st_comm_nccl_unique_id(void *unique_id);
int st_comm_nccl_create(st_comm *out, int size, int rank, const void *unique_id);
void st_comm_nccl_destroy(st_comm *c);

/* Host copies of the FP64 setup factors, for inspection and tests.
 * Time factors of level lvl (0 = finest), each nt x nt row-major, nt <= 8:
 * K_t, M_t, X (= Q, orthogonal), Z (quasi upper triangular Schur form; with
 * ST_SPATIAL_MINRES its 2x2 blocks are standardised to [[a, b1], [b2, a]]),
 * Y = (M_t X)^{-1}; any output may be NULL. */
int st_time_factors(st_handle h, int lvl, int *nt, double *Kt, double *Mt,
                    double *X, double *Z, double *Y);

/* Host copies of the 1D space factors of axis a (0 = x): dense n x n M1, K1,
 * the generalized eigenvectors U (columns, U^T M1 U = I) and eigenvalues. */
int st_space_factors(st_handle h, int axis, int *n, double *M1, double *K1,
                     double *U, double *lam);

/* Autotune the FP32 spatial transforms (mixed modes): for every axis, time
 * the tensor-core kernel at 1..4 CTAs per SM (TF32 / BF16 modes; the
 * candidates give identical results, so tuning never changes the numbers)
 * with CUDA events on the handle's stream and keep the fastest.
 * choice[a]: 0 = CUDA cores (ST_MIXED_FP32), k > 0 = tensor cores with k
 * CTAs per SM (-1 for unused axes); ms[a]: its time per pass.  Either may
 * be NULL.  Synchronises; FP64 handles return immediately. */
int st_autotune(st_handle h, int *choice, double *ms);

/* Generalized eigenvalues lambda = lam_re + i lam_im of K_t z = lambda M_t z
 * on level lvl (Sec. 3.2; their real parts must be positive) and the 2-norm
 * condition number of the eigenvector matrix X with unit columns (Table 1 of
 * Sec. 4.1 reports it).  nt entries each; any output may be NULL. */
int st_time_spectrum(st_handle h, int lvl, double *lam_re, double *lam_im, double *cond_x);

/* The time prolongation P_t (2 nt x nt, row-major) that expresses one coarse
 * slab in the bases of the two fine slabs it merges (Sec. 3.1). */
int st_time_prolongation(st_handle h, int *nt, double *Pt);

/* Shape of multigrid level lvl (0 = finest) of the space-time hierarchy
 * (Sec. 3.1 coarsens in time and, with opt.space_ratio, in space): slabs
 * per right-hand side, knot spans per axis (spans[3], unused axes 1) and
 * whether the level was obtained from the previous one by halving the spans
 * (*space_step = 1) or by merging slab pairs (0; level 0: 0).  Any output
 * may be NULL; ST_ERR_INVALID_ARG for a level out of range. */
int st_level_shape(st_handle h, int lvl, int *slabs, int *spans, int *space_step);

/* The 1D space prolongation of axis a used between level lvl and level
 * lvl + 1 when the latter was obtained by halving the spans: P (n_f x n_c,
 * row-major) expresses the interior B-splines of the coarse grid in those of
 * level lvl's grid (knot insertion).  *nf, *nc receive the sizes; P may be
 * NULL to query them.  ST_ERR_INVALID_ARG when level lvl + 1 is not a space
 * step or a is not an axis of the domain. */
int st_space_prolongation(st_handle h, int lvl, int axis, int *nf, int *nc, double *P);

/* Message of the last failure on the calling thread ("" if none). */
const char *st_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ST_IGA_H */

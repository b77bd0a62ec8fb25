// C ABI of the space-time multigrid library (see include/st_iga.h).
//
// Host orchestration: setup of the FP64 factors, device buffers, the damped
// block-Jacobi smoothing step (Sec. 3.1 with A_n^{-1} through Eq. 3.1), the
// time-coarsening V-cycle and the FP64 outer iteration (FGMRES or plain
// multigrid iteration).  All arithmetic on vectors runs in the kernels of
// kernels_*.cu on the handle's stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/st_iga.h"
#include "host_setup.h"
#include "st_internal.h"

using namespace st;
using host::Mat;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(...)                                                                          \
    do {                                                                                 \
        cudaError_t e_ = (__VA_ARGS__);                                                  \
        if (e_ != cudaSuccess)                                                           \
            return fail(ST_ERR_CUDA, "%s failed: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)

#define CKS(...)                       \
    do {                               \
        int s_ = (__VA_ARGS__);        \
        if (s_ != ST_OK) return s_;    \
    } while (0)

struct LevelHost {
    int nslab;  // slabs per problem
    int sp = 0;          // index of the level's spatial grid (st_handle_s::ls)
    bool xstep = false;  // obtained from the previous level by halving the spans
    double tau;
    Mat Kt, Mt, X, Z, Y;  // real Schur factors (Sec. 3.5)
    std::vector<int> blk;
    // diagonalisation (Sec. 3.3): eigenvalues, unit-column eigenvectors, Y = (M_t X)^{-1}
    std::vector<double> lre, lim;
    Mat Xre, Xim, Yre, Yim;
    double condX = 0.0;
    bool eig_ok = false;
    // complex Schur form (Sec. 3.4): K_t Q_c = M_t Q_c T_c, T_c upper
    // triangular, Q_c unitary; Y_c = (M_t Q_c)^{-1}
    Mat Qcre, Qcim, Tcre, Tcim, Ycre, Ycim;
};

template <typename T>
struct DevSpace {  // device copies of the 1D factors in one precision
    Bands<T> bands{};
    const T *U[3] = {nullptr, nullptr, nullptr};   // W = U  (forward, U^T applied)
    const T *Ut[3] = {nullptr, nullptr, nullptr};  // W = U^T (inverse, U applied)
    const T *lam[3] = {nullptr, nullptr, nullptr};
    const T *mu = nullptr;  // per spatial mode k: the shift sum over axes of lambda_axis
};

template <typename T>
struct Work {  // multigrid vectors in the V-cycle precision
    std::vector<T *> u, f;  // per level (level 0 entries only used in mixed mode)
    T *w0 = nullptr, *w1 = nullptr;
};

// Work space of the MinRes block solves (ST_SPATIAL_MINRES): compact batches
// [sys][comp][n_x] of up to `cap` systems with two components, the slab
// solution of Algorithm 1 (nt planes per slab), chunk partials and states.
template <typename T>
struct MrWork {
    T *q = nullptr, *qp = nullptr, *t = nullptr, *p = nullptr;  // Lanczos vectors
    T *d1 = nullptr, *d2 = nullptr, *x = nullptr;                // directions, iterate
    T *z0 = nullptr, *z1 = nullptr;                              // preconditioner ping-pong
    T *zs = nullptr;                                             // slab-layout solution
    // complex time factors: imaginary part of the solution, of w, and the
    // real / imaginary right-hand sides of Algorithm 1
    T *zi = nullptr, *wi = nullptr, *g0 = nullptr, *g1 = nullptr;
    double *partA = nullptr, *partB = nullptr;
    MrState *st = nullptr, *st2 = nullptr;  // current state, the next step's
    int *count = nullptr;
    long long cap = 0;  // systems
};

// One spatial grid of the multigrid hierarchy: 1D factors per axis (K1 U =
// M1 U Lambda, U^T M1 U = I), their bands, and -- when a coarser grid follows
// -- the 1D prolongations Pc[a] (this grid's n x the coarser grid's n) that
// express the coarser B-splines in this grid's (knot insertion).
struct LevelSpace {
    int spans[3] = {1, 1, 1}, n[3] = {1, 1, 1};
    Grid g{};
    Mat M1[3], K1[3], U[3], Pc[3];
    std::vector<double> lam[3], bandM[3], bandK[3];
    DevSpace<double> s64;
    DevSpace<float> s32;
    const double *P64[3] = {nullptr, nullptr, nullptr};
    const float *P32[3] = {nullptr, nullptr, nullptr};
};

}  // namespace

struct st_handle_s {
    int dim = 1, p = 1, N = 1, nt = 2, nrhs = 1, nlev = 1;
    int spans[3] = {1, 1, 1};
    int n[3] = {1, 1, 1};
    st_options opt{};
    cudaStream_t stream = nullptr;
    Grid g{};
    long long len = 0;  // dofs per rhs on level 0
    bool host_only = false;
    bool mixed = false;
    int nsm = 152;
    int max_smem = 48 * 1024;  // opt-in shared memory per block
    std::vector<SpecCoefs<float>> lvc32;   // per-level coefficients for the fused V-cycle
    std::vector<SpecCoefs<double>> lvc64;
    // per level: the per-mode slab inverses of the eigenbasis V-cycle
    std::vector<float *> inv32;
    std::vector<double *> inv64;
    // autotuned transform per axis: -1 = not tuned (heuristic), 0 = CUDA
    // cores, k > 0 = tensor cores with at most k CTAs per SM
    int tune[3] = {-1, -1, -1};
    // the same for the split-TF32 (FP32-accurate) transforms of the refinement
    int tune3[3] = {-1, -1, -1};
    double tune_ms[3] = {0, 0, 0};
    bool tuned = false;
    int *tc_err = nullptr;  // device flag: a tensor-core kernel's bounded wait ran out
    unsigned long long wait_ns = 1000000000ull;  // bound of each such wait (st_set_wait_limit)
    // host factors
    Mat M1[3], K1[3], U[3], Pt;
    std::vector<double> lam[3];
    std::vector<LevelHost> lv;
    // device
    std::vector<void *> allocs;
    size_t bytes = 0;
    // device memory from this stream-ordered pool instead of cudaMalloc (the
    // serving loop: releasing a setup then needs no device-wide synchronisation)
    cudaMemPool_t pool = nullptr;
    // slab partition (st_setup_partitioned): levels < gathered are split over
    // the ranks (this rank: lv[l].nslab slabs starting at global slab
    // slab_begin >> l), levels >= gathered hold every rank's slabs
    bool part = false;
    st_comm comm{};
    int slab_begin = 0, N_global = 0, gathered = 0;
    long long work_len = 0;              // largest level's dofs per rhs (work vectors)
    void *send_plane = nullptr, *halo = nullptr;  // [rhs][nxyz], FP64-sized
    void *agg_send = nullptr, *agg_recv = nullptr;  // gathered-level transfers
    void *stage = nullptr;               // pinned host staging for host-buffer comms
    size_t stage_bytes = 0;
    DevSpace<double> s64;
    DevSpace<float> s32;
    Work<double> w64;
    Work<float> w32;
    MrWork<double> mr64;
    MrWork<float> mr32;
    std::vector<LevelSpace> ls;   // spatial grids, finest first
    void *xtmp = nullptr;         // scratch of level-0 size for space transfers
    // per-kernel-class profiling (CUDA events around each launch)
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
        double bytes, flops;
    };
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    std::vector<ProfRec> recs;
    long long prof_n[ST_PROF_NCLASS] = {0};
    double prof_ms[ST_PROF_NCLASS] = {0}, prof_bytes[ST_PROF_NCLASS] = {0},
           prof_flops[ST_PROF_NCLASS] = {0};
    // outer iteration
    std::vector<double *> V, Zk;
    std::vector<float *> V32, Z32;  // FP32 Krylov space of the refinement's inner solver
    // CUDA graphs of the preconditioner, keyed by its (input, output) buffers
    struct GraphRec {
        const void *in;
        void *out;
        int uses;
        cudaGraphExec_t exec;
    };
    std::vector<GraphRec> graphs;
    cudaStream_t cap_stream = nullptr;
    double *r64 = nullptr;
    float *rhs32 = nullptr, *e32 = nullptr;
    int krylov32_m = 0;
    double *partial = nullptr, *dots = nullptr;
    // page-locked host block the reduced dot products are copied into (one
    // DMA, no staging through pageable memory)
    double *dots_host = nullptr;
    size_t dots_host_cap = 0;
    int nblk_dot = 0;
    int krylov_m = 0;
    // residual history of the last st_solve: (iterations so far, max over
    // the rhs of the FP64 relative residual) at every restart, multigrid
    // iteration or refinement step (st_solve_history)
    std::vector<std::pair<int, double>> hist;
    bool record_hist = false;  // set while the outer iteration runs
    // host synchronisations for reductions and Krylov vector-kernel launches
    // of the current solve (a group's operations count on its first member)
    long long n_sync = 0, n_vl = 0;
    // st_solve_host: two device staging slots per vector (allocated on first
    // use), the copy-in and copy-out streams, and per slot the events "copied
    // in", "solved" and "copied out"
    double *hs_f[2] = {nullptr, nullptr}, *hs_u[2] = {nullptr, nullptr};
    cudaStream_t cp_in = nullptr, cp_out = nullptr;
    cudaEvent_t hs_in[2] = {}, hs_solved[2] = {}, hs_out[2] = {};
    // solutions still to be copied back to the host: issued in chunks at the
    // solve's host synchronisation points, one chunk in flight at a time (a
    // device-to-host transfer delays the solve's own small reads behind it)
    struct BgCopy {
        double *dst;
        const double *src;
        size_t n, done;
        int slot;
    };
    std::deque<BgCopy> bg;
    cudaEvent_t bg_ev = nullptr;  // the last chunk issued
    cudaError_t bg_err = cudaSuccess;
};

namespace {

int dalloc(st_handle h, size_t bytes, void **out) {
    if (h->opt.hbm_budget && h->bytes + bytes > h->opt.hbm_budget)
        return fail(ST_ERR_OVER_BUDGET, "allocation of %zu bytes exceeds the HBM budget (%zu of %zu used)",
                    bytes, h->bytes, h->opt.hbm_budget);
    void *p = nullptr;
    cudaError_t e;
    if (h->pool) {
        // complete before any other stream (or a synchronous copy) uses it
        e = cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, h->pool, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    } else {
        e = cudaMalloc(&p, bytes ? bytes : 16);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ST_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    h->allocs.push_back(p);
    h->bytes += bytes;
    *out = p;
    return ST_OK;
}

// ---- profiling --------------------------------------------------------------
cudaEvent_t next_event(st_handle h) {
    if (h->ev_next == h->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_next++];
}

// Fold completed records into the per-class totals.  Only called when the
// handle's stream is idle (after a synchronisation).
void prof_fold(st_handle h) {
    for (const auto &r : h->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        h->prof_n[r.cls] += 1;
        h->prof_ms[r.cls] += ms;
        h->prof_bytes[r.cls] += r.bytes;
        h->prof_flops[r.cls] += r.flops;
    }
    h->recs.clear();
    h->ev_next = 0;
}

// A named host range for timeline profilers (NVTX): one per API call,
// refinement step, Krylov cycle, preconditioner application and V-cycle
// level.  A replayed CUDA graph shows as its preconditioner range (the level
// ranges appear where the cycle is launched directly).  Without an attached
// tool a range costs two calls through no-op function pointers.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
const char *level_range_name(int l) {
    static const char *const names[] = {
        "V-cycle level 0",  "V-cycle level 1",  "V-cycle level 2",  "V-cycle level 3",
        "V-cycle level 4",  "V-cycle level 5",  "V-cycle level 6",  "V-cycle level 7",
        "V-cycle level 8",  "V-cycle level 9",  "V-cycle level 10", "V-cycle level 11",
        "V-cycle level 12", "V-cycle level 13", "V-cycle level 14", "V-cycle level >= 15"};
    return names[l < 0 ? 0 : (l > 15 ? 15 : l)];
}

// Records [start, stop) events around one launch when profiling is on.
struct KScope {
    st_handle h;
    int cls;
    double bytes, flops;
    cudaEvent_t a = nullptr;
    KScope(st_handle h_, int c, double by, double fl) : h(h_), cls(c), bytes(by), flops(fl) {
        if (h->prof_on && (a = next_event(h))) cudaEventRecord(a, h->stream);
    }
    // nothing was launched in the scope: record nothing
    void cancel() { a = nullptr; }
    ~KScope() {
        if (!a) return;
        cudaEvent_t b = next_event(h);
        if (!b) return;
        cudaEventRecord(b, h->stream);
        h->recs.push_back({cls, a, b, bytes, flops});
    }
};

template <typename T>
constexpr int cls_of(int c64, int c32) { return sizeof(T) == 8 ? c64 : c32; }

template <typename T>
int upload(st_handle h, const std::vector<double> &src, const T **out) {
    std::vector<T> tmp(src.begin(), src.end());
    void *p;
    CKS(dalloc(h, tmp.size() * sizeof(T), &p));
    CK(cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    *out = static_cast<const T *>(p);
    return ST_OK;
}

template <typename T>
int upload_space(st_handle h, DevSpace<T> &ds, const LevelSpace &S) {
    for (int a = 0; a < h->dim; ++a) {
        const int n = S.n[a];
        CKS(upload<T>(h, S.bandM[a], &ds.bands.M[a]));
        CKS(upload<T>(h, S.bandK[a], &ds.bands.K[a]));
        CKS(upload<T>(h, S.U[a], &ds.U[a]));
        Mat Ut(n * n);
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) Ut[k * n + i] = S.U[a][i * n + k];
        CKS(upload<T>(h, Ut, &ds.Ut[a]));
        CKS(upload<T>(h, S.lam[a], &ds.lam[a]));
    }
    for (int a = h->dim; a < 3; ++a) {
        ds.bands.M[a] = ds.bands.K[a] = nullptr;
        ds.U[a] = ds.Ut[a] = ds.lam[a] = nullptr;
    }
    // mu_k = lambda_x[kx] + lambda_y[ky] + lambda_z[kz], k = (kz * ny + ky) * nx + kx
    std::vector<double> mu((size_t)S.n[0] * S.n[1] * S.n[2]);
    for (int kz = 0; kz < S.n[2]; ++kz)
        for (int ky = 0; ky < S.n[1]; ++ky)
            for (int kx = 0; kx < S.n[0]; ++kx) {
                double m = S.lam[0][kx];
                if (h->dim >= 2) m += S.lam[1][ky];
                if (h->dim >= 3) m += S.lam[2][kz];
                mu[((size_t)kz * S.n[1] + ky) * S.n[0] + kx] = m;
            }
    CKS(upload<T>(h, mu, &ds.mu));
    return ST_OK;
}

// Spatial factors of the grid with the given spans: M1, K1, the generalized
// eigenpairs (checked), the bands of M1 and K1.
int build_space(st_handle h, const int spans[3], LevelSpace &S) {
    const int degree = h->p;
    const int W = 2 * degree + 1;
    for (int a = 0; a < 3; ++a) {
        S.spans[a] = (a < h->dim) ? spans[a] : 1;
        S.n[a] = (a < h->dim) ? spans[a] + degree - 2 : 1;
    }
    S.g.nx = S.n[0];
    S.g.ny = S.n[1];
    S.g.nz = S.n[2];
    S.g.dim = h->dim;
    S.g.p = degree;
    S.g.nxyz = (long long)S.n[0] * S.n[1] * S.n[2];
    for (int a = 0; a < h->dim; ++a) {
        const int n = S.n[a];
        host::space_matrices(S.spans[a], degree, S.M1[a], S.K1[a]);
        std::string err;
        if (!host::sym_gen_eig(n, S.K1[a], S.M1[a], S.U[a], S.lam[a], err))
            return fail(ST_ERR_ILL_CONDITIONED, "space eigenproblem axis %d: %s", a, err.c_str());
        // checks: K1 U = M1 U Lambda, U^T M1 U = I
        Mat MU = host::matmul(n, S.M1[a], S.U[a]);
        Mat KU = host::matmul(n, S.K1[a], S.U[a]);
        double r1 = 0, r2 = 0;
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) {
                r1 = std::max(r1, std::fabs(KU[i * n + k] - MU[i * n + k] * S.lam[a][k]));
                double sum = 0;
                for (int j = 0; j < n; ++j) sum += S.U[a][j * n + i] * MU[j * n + k];
                r2 = std::max(r2, std::fabs(sum - (i == k ? 1.0 : 0.0)));
            }
        if (r1 > 1e-9 * S.lam[a][n - 1] || r2 > 1e-9)
            return fail(ST_ERR_ILL_CONDITIONED, "space eigen residuals %.2e %.2e", r1, r2);
        S.bandM[a].assign((size_t)n * W, 0.0);
        S.bandK[a].assign((size_t)n * W, 0.0);
        for (int i = 0; i < n; ++i)
            for (int oo = -degree; oo <= degree; ++oo) {
                const int j = i + oo;
                if (j < 0 || j >= n) continue;
                S.bandM[a][(size_t)i * W + oo + degree] = S.M1[a][i * n + j];
                S.bandK[a][(size_t)i * W + oo + degree] = S.K1[a][i * n + j];
            }
    }
    return ST_OK;
}

template <typename T>
int alloc_work(st_handle h, Work<T> &w, bool level0) {
    const size_t e0 = (size_t)std::max(h->len, h->work_len) * h->nrhs;
    void *p;
    CKS(dalloc(h, e0 * sizeof(T), &p));
    w.w0 = (T *)p;
    CKS(dalloc(h, e0 * sizeof(T), &p));
    w.w1 = (T *)p;
    w.u.assign(h->nlev, nullptr);
    w.f.assign(h->nlev, nullptr);
    for (int l = level0 ? 0 : 1; l < h->nlev; ++l) {
        const size_t e = (size_t)h->lv[l].nslab * h->nt * h->ls[h->lv[l].sp].g.nxyz * h->nrhs;
        CKS(dalloc(h, e * sizeof(T), &p));
        w.u[l] = (T *)p;
        CKS(dalloc(h, e * sizeof(T), &p));
        w.f[l] = (T *)p;
    }
    return ST_OK;
}

// ---- coefficient packing ----------------------------------------------------
template <typename T>
TimeCoefs<T> pack_time(st_handle h, int l, int mode, bool fuse_y) {
    TimeCoefs<T> tc;
    std::memset(&tc, 0, sizeof tc);
    const int nt = h->nt;
    const LevelHost &L = h->lv[l];
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nt; ++j) {
            if (mode == MODE_MASS) {
                tc.CK[i * NTMAX + j] = (T)L.Mt[i * nt + j];
                tc.CM[i * NTMAX + j] = T(0);
            } else {
                tc.CK[i * NTMAX + j] = (T)L.Kt[i * nt + j];
                tc.CM[i * NTMAX + j] = (T)L.Mt[i * nt + j];
            }
            tc.Y[i * NTMAX + j] = (T)L.Y[i * nt + j];
        }
    tc.nt = nt;
    tc.fuse_y = fuse_y ? 1 : 0;
    tc.mode = mode;
    return tc;
}

template <typename T>
SchurCoefs<T> pack_schur(st_handle h, int l) {
    SchurCoefs<T> sc;
    std::memset(&sc, 0, sizeof sc);
    const int nt = h->nt;
    const LevelHost &L = h->lv[l];
    for (int i = 0; i < nt; ++i) {
        for (int j = 0; j < nt; ++j) {
            sc.Z[i * NTMAX + j] = (T)L.Z[i * nt + j];
            sc.X[i * NTMAX + j] = (T)L.X[i * nt + j];
        }
        sc.blk[i] = L.blk[i];
    }
    sc.nt = nt;
    return sc;
}

template <typename T>
ProlongCoefs<T> pack_prolong(st_handle h) {
    ProlongCoefs<T> pc;
    std::memset(&pc, 0, sizeof pc);
    const int nt = h->nt;
    for (int r = 0; r < 2 * nt; ++r)
        for (int c = 0; c < nt; ++c) pc.P[r * NTMAX + c] = (T)h->Pt[r * nt + c];
    pc.nt = nt;
    return pc;
}

template <typename T>
SpecCoefs<T> pack_spec(st_handle h, int l) {
    SpecCoefs<T> c;
    std::memset(&c, 0, sizeof c);
    const int nt = h->nt;
    const LevelHost &L = h->lv[l];
    for (int i = 0; i < nt; ++i) {
        for (int j = 0; j < nt; ++j) {
            c.Kt[i * NTMAX + j] = (T)L.Kt[i * nt + j];
            c.Mt[i * NTMAX + j] = (T)L.Mt[i * nt + j];
            c.Y[i * NTMAX + j] = (T)L.Y[i * nt + j];
            c.Z[i * NTMAX + j] = (T)L.Z[i * nt + j];
            c.X[i * NTMAX + j] = (T)L.X[i * nt + j];
        }
        c.blk[i] = L.blk[i];
    }
    c.nt = nt;
    c.variant = h->opt.variant;
    if (h->opt.variant == ST_CSCHUR) {
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < nt; ++j) {
                c.X[i * NTMAX + j] = (T)L.Qcre[i * nt + j];
                c.Xi[i * NTMAX + j] = (T)L.Qcim[i * nt + j];
                c.Y[i * NTMAX + j] = (T)L.Ycre[i * nt + j];
                c.Yi[i * NTMAX + j] = (T)L.Ycim[i * nt + j];
                c.Z[i * NTMAX + j] = (T)L.Tcre[i * nt + j];
                c.Zi[i * NTMAX + j] = (T)L.Tcim[i * nt + j];
            }
    }
    if (h->opt.variant == ST_EIG) {
        for (int i = 0; i < nt; ++i) {
            for (int j = 0; j < nt; ++j) {
                c.X[i * NTMAX + j] = (T)L.Xre[i * nt + j];
                c.Xi[i * NTMAX + j] = (T)L.Xim[i * nt + j];
                c.Y[i * NTMAX + j] = (T)L.Yre[i * nt + j];
                c.Yi[i * NTMAX + j] = (T)L.Yim[i * nt + j];
            }
            c.lre[i] = (T)L.lre[i];
            c.lim[i] = (T)L.lim[i];
        }
    }
    return c;
}

template <typename T>
DevSpace<T> &space(st_handle h);
template <>
DevSpace<double> &space<double>(st_handle h) { return h->s64; }
template <>
DevSpace<float> &space<float>(st_handle h) { return h->s32; }
template <typename T>
Work<T> &work(st_handle h);
template <>
Work<double> &work<double>(st_handle h) { return h->w64; }
template <>
Work<float> &work<float>(st_handle h) { return h->w32; }

// ---- slab partition: communication ----------------------------------------
// Each call runs the comm callback (staging through pinned host memory for
// host-buffer comms) and turns a failure into ST_ERR_COMM.
int comm_sendrecv(st_handle h, const void *send, int dst, void *recv, int src, size_t bytes) {
    const st_comm &c = h->comm;
    if (!c.host_buffers) {
        if (c.sendrecv(c.ctx, send, dst, recv, src, bytes, h->stream) != 0)
            return fail(ST_ERR_COMM, "sendrecv callback failed");
        return ST_OK;
    }
    char *hs = static_cast<char *>(h->stage), *hr = hs + bytes;
    if (dst >= 0) CK(cudaMemcpyAsync(hs, send, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (c.sendrecv(c.ctx, hs, dst, hr, src, bytes, h->stream) != 0)
        return fail(ST_ERR_COMM, "sendrecv callback failed");
    if (src >= 0) {
        CK(cudaMemcpyAsync(recv, hr, bytes, cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));  // the staging buffer is reused
    }
    return ST_OK;
}

int comm_allgather(st_handle h, const void *send, void *recv, size_t bytes) {
    const st_comm &c = h->comm;
    if (!c.host_buffers) {
        if (c.allgather(c.ctx, send, recv, bytes, h->stream) != 0)
            return fail(ST_ERR_COMM, "allgather callback failed");
        return ST_OK;
    }
    char *hs = static_cast<char *>(h->stage), *hr = hs + bytes;
    CK(cudaMemcpyAsync(hs, send, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (c.allgather(c.ctx, hs, hr, bytes, h->stream) != 0)
        return fail(ST_ERR_COMM, "allgather callback failed");
    CK(cudaMemcpyAsync(recv, hr, bytes * c.size, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ST_OK;
}

int comm_allreduce(st_handle h, std::vector<double> &v) {
    if (v.empty()) return ST_OK;
    if (h->comm.allreduce_sum(h->comm.ctx, v.data(), v.size()) != 0)
        return fail(ST_ERR_COMM, "allreduce callback failed");
    return ST_OK;
}

// The coupling plane of a partitioned level: send the last time plane of this
// rank's last slab (every rhs) to the next rank, receive the previous rank's
// into the halo buffer; returns the halo pointer for the stencil (nullptr on
// rank 0, whose first slab has no predecessor).
template <typename T>
int exchange_halo(st_handle h, int l, const T *u, const void **halo) {
    *halo = nullptr;
    if (!h->part || l >= h->gathered) return ST_OK;
    const long long nxyz = h->g.nxyz, slab = (long long)h->nt * nxyz;
    const int Nl = h->lv[l].nslab, R = h->nrhs, rank = h->comm.rank, size = h->comm.size;
    T *sp = static_cast<T *>(h->send_plane), *hp = static_cast<T *>(h->halo);
    if (rank + 1 < size)
        CK(cudaMemcpy2DAsync(sp, nxyz * sizeof(T), u + (Nl - 1) * slab + (h->nt - 1) * nxyz,
                             Nl * slab * sizeof(T), nxyz * sizeof(T), R, cudaMemcpyDeviceToDevice,
                             h->stream));
    CKS(comm_sendrecv(h, sp, rank + 1 < size ? rank + 1 : -1, hp, rank > 0 ? rank - 1 : -1,
                      (size_t)R * nxyz * sizeof(T)));
    if (rank > 0) *halo = hp;
    return ST_OK;
}

// ---- operator pieces --------------------------------------------------------
template <typename T>
int stencil(st_handle h, int l, const T *u, const T *f, T *out, int mode, bool fuse_y, int slab0,
            int nslabs) {
    const TimeCoefs<T> tc = pack_time<T>(h, l, mode, fuse_y);
    // algorithmic traffic: u and out once (+ f for the residual, + the
    // coupling plane), flops of the sum-factorised applies on every plane
    const double E = (double)nslabs * h->nt * h->g.nxyz;
    const double planes_pt = (double)nslabs * (h->nt + (mode == MODE_MASS ? 0 : 1)) * h->g.nxyz;
    const int W = 2 * h->p + 1;
    const double fsp = 4.0 * W + (h->dim >= 2 ? 6.0 * W : 0) + (h->dim >= 3 ? 6.0 * W : 0);
    const double bytes = sizeof(T) * (2.0 * E + (mode == MODE_RES ? E : 0.0) +
                                      (mode == MODE_MASS ? 0.0 : (double)nslabs * h->g.nxyz));
    const double flops = planes_pt * fsp + E * 4.0 * h->nt + (fuse_y ? E * 2.0 * h->nt : 0.0);
    TimeCoefs<T> tcl = tc;
    if (mode != MODE_MASS) CKS(exchange_halo<T>(h, l, u, &tcl.halo));
    KScope ks(h, cls_of<T>(ST_PROF_STENCIL64, ST_PROF_STENCIL32), bytes, flops);
    CK(launch_stencil<T>(u, f, out, space<T>(h).bands, h->g, tcl, h->lv[l].nslab, slab0, nslabs,
                         h->stream));
    return ST_OK;
}

// out[..k..] = sum_i W[i][k] in[..i..] along every active axis (forward: W = U,
// i.e. U^T applied; inverse: W = U^T).  Ping-pongs in -> t0 -> t1 -> t0;
// *res is the buffer holding the result.  FP32 transforms run on the tensor
// cores in the TF32 / BF16 modes (CUDA cores for shapes the kernel does not
// cover), everything else on CUDA cores.
template <typename T>
int axis_pass(st_handle h, int axis, const T *in, T *out, bool forward, long long planes,
              bool full32 = false) {
    DevSpace<T> &ds = space<T>(h);
    const long long nx = h->g.nx, ny = h->g.ny, nz = h->g.nz;
    const long long n = (axis == 0) ? nx : (axis == 1) ? ny : nz;
    const double E = (double)planes * h->g.nxyz;
    const T *W = forward ? ds.U[axis] : ds.Ut[axis];
    const long long inner = (axis == 0) ? 1 : (axis == 1) ? nx : nx * ny;
    const long long outer = (long long)(E / (double)(n * inner) + 0.5);
    const int prec = h->opt.precision;
    if (sizeof(T) == 4 && (prec == ST_MIXED_TF32 || prec == ST_MIXED_BF16) && h->tune[axis] != 0) {
        const float *Wt = (const float *)(forward ? ds.Ut[axis] : ds.U[axis]);
        // full32: split TF32 on the tensor cores, as accurate as FP32
        const int kind = full32 ? 3 : (prec == ST_MIXED_TF32) ? 2 : 1;
        const long long ncols = (axis == 0) ? outer : outer * inner;
        KScope ks(h, ST_PROF_TC, sizeof(T) * (2.0 * E + n * n), 2.0 * E * n);
        const cudaError_t e = launch_tc_axis(kind, axis == 0 ? 0 : 1, (const float *)in,
                                             (float *)out, Wt, (int)n, (int)n, ncols, inner,
                                             h->tc_err, h->nsm, h->stream,
                                             full32 ? (h->tune3[axis] > 0 ? h->tune3[axis] : 0)
                                                    : (h->tune[axis] > 0 ? h->tune[axis] : 0),
                                             h->wait_ns);
        if (e == cudaSuccess) return ST_OK;
        if (e != cudaErrorNotSupported) CK(e);
        cudaGetLastError();
        ks.cancel();
    }
    KScope ks(h, cls_of<T>(ST_PROF_GEMM64, ST_PROF_GEMM32), sizeof(T) * (2.0 * E + n * n),
              2.0 * E * n);
    if (axis == 0) {
        CK(launch_gemm_strided<T>(1, (int)outer, (int)nx, (int)nx, in, 0, nx, 1, W, 0, nx, 1, out,
                                  0, nx, 1, h->stream));
    } else {
        CK(launch_gemm_strided<T>((int)outer, (int)n, (int)inner, (int)n, W, 0, 1, n, in,
                                  n * inner, inner, 1, out, n * inner, inner, 1, h->stream));
    }
    return ST_OK;
}

template <typename T>
int spatial(st_handle h, const T *in, T *t0, T *t1, bool forward, long long planes, T **res,
            bool full32 = false) {
    CKS(axis_pass<T>(h, 0, in, t0, forward, planes, full32));
    *res = t0;
    if (h->dim < 2) return ST_OK;
    CKS(axis_pass<T>(h, 1, t0, t1, forward, planes, full32));
    *res = t1;
    if (h->dim < 3) return ST_OK;
    CKS(axis_pass<T>(h, 2, t1, t0, forward, planes, full32));
    *res = t0;
    return ST_OK;
}

// Autotuner: time every candidate for each axis pass of the FP32 transform on
// the level-0 buffers (CUDA-event medians of 3 runs) and keep the fastest.
int autotune(st_handle h) {
    if (!h->mixed) {
        h->tuned = true;
        return ST_OK;
    }
    const bool tc_ok = h->opt.precision == ST_MIXED_TF32 || h->opt.precision == ST_MIXED_BF16;
    const long long planes = (long long)h->N * h->nrhs * h->nt;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const bool prof = h->prof_on;
    h->prof_on = false;
    for (int ax = 0; ax < h->dim; ++ax) {
        double best = 1e30;
        int best_c = 0;
        // only candidates that give identical numbers (the CTA count of the
        // tensor-core kernel); CUDA cores vs tensor cores is set by the mode
        for (int c = tc_ok ? 1 : 0; c <= (tc_ok ? 4 : 0); ++c) {
            h->tune[ax] = c;
            float t[3];
            for (int rep = 0; rep < 4; ++rep) {
                CK(cudaEventRecord(e0, h->stream));
                CKS(axis_pass<float>(h, ax, h->w32.w0, h->w32.w1, true, planes));
                CK(cudaEventRecord(e1, h->stream));
                CK(cudaEventSynchronize(e1));
                if (rep > 0) CK(cudaEventElapsedTime(&t[rep - 1], e0, e1));
            }
            std::sort(t, t + 3);
            if (t[1] < best) {
                best = t[1];
                best_c = c;
            }
        }
        h->tune[ax] = best_c;
        h->tune_ms[ax] = best;
        if (!tc_ok) continue;
        // the split-TF32 kind: CTAs per SM (its contraction is then staged in
        // K chunks small enough for that many CTAs; same numbers either way)
        double best3 = 1e30;
        int best3_c = 1;
        for (int c = 1; c <= 4; ++c) {
            h->tune3[ax] = c;
            float t[3];
            for (int rep = 0; rep < 4; ++rep) {
                CK(cudaEventRecord(e0, h->stream));
                CKS(axis_pass<float>(h, ax, h->w32.w0, h->w32.w1, true, planes, true));
                CK(cudaEventRecord(e1, h->stream));
                CK(cudaEventSynchronize(e1));
                if (rep > 0) CK(cudaEventElapsedTime(&t[rep - 1], e0, e1));
            }
            std::sort(t, t + 3);
            if (t[1] < best3) {
                best3 = t[1];
                best3_c = c;
            }
        }
        h->tune3[ax] = best3_c;
    }
    h->prof_on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tuned = true;
    return ST_OK;
}

// ---- inexact spatial solves (ST_SPATIAL_MINRES, Sec. 3.5) ---------------------
template <typename T>
MrWork<T> &mrwork(st_handle h);
template <>
MrWork<double> &mrwork<double>(st_handle h) { return h->mr64; }
template <>
MrWork<float> &mrwork<float>(st_handle h) { return h->mr32; }

// Steps after which the MinRes bound 2 q^floor(k/2), q = (sqrt2 - 1)/(sqrt2 + 1),
// for a spectrum of P^{-1} A inside [-1, -1/sqrt2] u [1/sqrt2, 1]
// (Theorems 3.2/3.3) falls to tol.
int minres_bound_steps(double tol) {
    const double q = 3.0 - 2.0 * std::sqrt(2.0);
    return 2 * (int)std::ceil(std::log(tol / 2.0) / std::log(q));
}

// Nine batch vectors of cap systems with two components, the slab-layout
// solution, partials and states, by `alloc` (the handle's budgeted
// allocator, or plain device memory for a one-off solve).
template <typename T, typename Alloc>
int alloc_mr(st_handle h, MrWork<T> &w, long long cap, bool with_slabs, Alloc alloc) {
    const size_t e = (size_t)cap * 2 * h->g.nxyz;
    void *p;
    T **vecs[9] = {&w.q, &w.qp, &w.t, &w.p, &w.d1, &w.d2, &w.x, &w.z0, &w.z1};
    for (T **v : vecs) {
        CKS(alloc(e * sizeof(T), &p));
        *v = (T *)p;
    }
    if (with_slabs) {
        T **slabv[5] = {&w.zs, &w.zi, &w.wi, &w.g0, &w.g1};
        const int nslabv = h->opt.variant == ST_RSCHUR ? 1 : 5;
        for (int k = 0; k < nslabv; ++k) {
            CKS(alloc((size_t)cap * h->nt * h->g.nxyz * sizeof(T), &p));
            *slabv[k] = (T *)p;
        }
    }
    CKS(alloc(sizeof(double) * cap * MR_MAX_CHUNKS, &p));
    w.partA = (double *)p;
    CKS(alloc(sizeof(double) * cap * MR_MAX_CHUNKS, &p));
    w.partB = (double *)p;
    CKS(alloc(sizeof(MrState) * cap, &p));
    w.st = (MrState *)p;
    CKS(alloc(sizeof(MrState) * cap, &p));
    w.st2 = (MrState *)p;
    CKS(alloc(sizeof(int), &p));
    w.count = (int *)p;
    w.cap = cap;
    return ST_OK;
}

// z = P^{-1} in for nsys systems of c components, P = diag(pw_c (K_x + shift M_x)):
// forward spatial transforms, the eigenbasis scaling, inverse transforms
// (FP32-accurate transforms in the mixed modes, so that P^{-1} stays
// symmetric to working precision).  *res is the buffer holding z (z0 or z1).
template <typename T>
int precond_fd(st_handle h, const T *in, T *z0, T *z1, T **res, int nsys, int c, double shift,
               double pw0, double pw1) {
    const long long planes = (long long)nsys * c;
    T *fw = nullptr;
    CKS(spatial<T>(h, in, z0, z1, true, planes, &fw, true));
    {
        const double E = (double)planes * h->g.nxyz;
        KScope ks(h, ST_PROF_MINRES, sizeof(T) * (2.0 * E + h->g.nxyz), 2.0 * E);
        CK(launch_fd_scale<T>(fw, space<T>(h).mu, shift, pw0, pw1, c, h->g.nxyz, nsys, h->stream));
    }
    T *other = (fw == z0) ? z1 : z0;
    CKS(spatial<T>(h, fw, other, fw, false, planes, res, true));
    return ST_OK;
}

// Algorithmic bytes and flops of one sum-factorised operator application on
// `planes` spatial planes without coupling plane (ntp planes per system).
inline void op_counts(st_handle h, double planes, int ntp, int tsize, double *bytes,
                      double *flops) {
    const int W = 2 * h->p + 1;
    const double fsp = 4.0 * W + (h->dim >= 2 ? 6.0 * W : 0) + (h->dim >= 3 ? 6.0 * W : 0);
    const double E = planes * h->g.nxyz;
    *bytes = tsize * 2.0 * E;
    *flops = E * fsp + E * 4.0 * ntp;
}

struct BlockCoef {
    double alpha, beta1, beta2;  // the standardised block [[alpha, beta1], [beta2, alpha]]
};

// Preconditioned MinRes (Theorem 3.3) on nsys systems whose scaled
// right-hand sides [|beta2| f; |beta1| g] are in w.q (zero initial guess);
// the iterate [x; -y] is in w.x on return.  `steps` MinRes steps run, a
// system that has converged stops updating; early: after every step read
// the number of running systems and stop when none is left (never during a
// stream capture).
template <typename T>
int block_minres(st_handle h, MrWork<T> &w, const BlockCoef &bc, int nsys, double tol, int steps,
                 bool early) {
    const long long m = h->g.nxyz, len = 2 * m;
    const int chunks = mr_dot_chunks(len);
    const double a1 = std::fabs(bc.beta2), a2 = std::fabs(bc.beta1);
    const double shift = bc.alpha + std::sqrt(a1 * a2);
    const cudaStream_t s = h->stream;
    const double E = (double)nsys * len;
    // Abar as a two-plane operator: y_i = sum_j CK[i][j] M_x u_j + CM[i][j] K_x u_j
    TimeCoefs<T> tc;
    std::memset(&tc, 0, sizeof tc);
    tc.CK[0] = (T)(a1 * bc.alpha);
    tc.CK[1] = (T)(-bc.beta1 * a1);
    tc.CK[NTMAX] = (T)(a2 * bc.beta2);
    tc.CK[NTMAX + 1] = (T)(-a2 * bc.alpha);
    tc.CM[0] = (T)a1;
    tc.CM[NTMAX + 1] = (T)(-a2);
    tc.nt = 2;
    tc.fuse_y = 0;
    tc.mode = MODE_APPLY;
    double ob, of;
    op_counts(h, 2.0 * nsys, 2, sizeof(T), &ob, &of);
    T *z = nullptr;
    CKS(precond_fd<T>(h, w.q, w.z0, w.z1, &z, nsys, 2, shift, a1, a2));
    {
        KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * E, 2.0 * E);
        CK(launch_seg_dot<T>(w.q, z, w.partB, len, nsys, s));
    }
    {
        KScope ks(h, ST_PROF_MINRES, 8.0 * chunks * nsys, 0.0);
        CK(launch_mr_init(w.partB, chunks, w.st, nsys, s));
    }
    {
        KScope ks(h, ST_PROF_MINRES, sizeof(T) * 8.0 * E, 2.0 * E);
        CK(launch_mr_init_vec<T>(w.q, w.p, z, w.qp, w.d1, w.d2, w.x, w.st, len, nsys, s));
    }
    T *q = w.q, *qp = w.qp, *t = w.t, *d1 = w.d1, *d2 = w.d2;
    for (int k = 0; k < steps; ++k) {
        {
            KScope ks(h, cls_of<T>(ST_PROF_STENCIL64, ST_PROF_STENCIL32), ob, of);
            CK(launch_stencil<T>(w.p, nullptr, t, space<T>(h).bands, h->g, tc, 1, 0, nsys, s));
        }
        {
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * E, 2.0 * E);
            CK(launch_seg_dot<T>(w.p, t, w.partA, len, nsys, s));
        }
        {
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 4.0 * E, 4.0 * E);
            CK(launch_mr_lanczos<T>(t, q, qp, w.partA, chunks, w.st, len, nsys, s));
        }
        CKS(precond_fd<T>(h, t, w.z0, w.z1, &z, nsys, 2, shift, a1, a2));
        {
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * E, 2.0 * E);
            CK(launch_seg_dot<T>(t, z, w.partB, len, nsys, s));
        }
        {
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 10.0 * E, 8.0 * E);
            CK(launch_mr_step<T>(w.p, z, t, d1, d2, w.x, w.partA, w.partB, chunks, w.st, w.st2,
                                 tol, len, nsys, s));
            std::swap(w.st, w.st2);
        }
        // the new direction is in d2; q_{k+1} is in t
        std::swap(d1, d2);
        T *free_q = qp;
        qp = q;
        q = t;
        t = free_q;
        if (early) {
            int left = 0;
            CK(launch_mr_count(w.st, nsys, w.count, s));
            CK(cudaMemcpyAsync(&left, w.count, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (left == 0) break;
        }
    }
    return ST_OK;
}

// The MinRes smoothing step with complex time factors (ST_EIG, Sec. 3.3;
// ST_CSCHUR, Sec. 3.4): w = (Y (x) I)(f - L u) in real and imaginary parts
// (two residual passes, Re Y and Im Y fused); Algorithm 1 over the rows of
// the upper triangular T from the last to the first,
//   g_i = w_i - sum_{j>i} T_ij M_x z_j   (four real operator passes when row i
//   of T has entries right of the diagonal; none for the diagonalisation),
// each complex shift lambda_i = alpha + i beta solved by MinRes in Theorem
// 3.2's form (beta1 = -beta, beta2 = beta, iterate [x; -y] for z_i = x + i y),
// a real one by one application of (K_x + lambda_i M_x)^{-1} to both parts;
// u <- (overwrite ? 0 : u) + omega Re((X (x) I) z) = ... + omega ((Re X) z_re - (Im X) z_im).
template <typename T>
int smooth_range_minres_cplx(st_handle h, int l, T *u, const T *f, T omega, int s0, int ns,
                             int overwrite) {
    Work<T> &w = work<T>(h);
    MrWork<T> &mw = mrwork<T>(h);
    const int nt = h->nt;
    const long long m = h->g.nxyz, sl = (long long)nt * m;
    const LevelHost &L = h->lv[l];
    const bool eig = h->opt.variant == ST_EIG;
    const Mat &Yr = eig ? L.Yre : L.Ycre, &Yi = eig ? L.Yim : L.Ycim;
    const Mat &Xr = eig ? L.Xre : L.Qcre, &Xi = eig ? L.Xim : L.Qcim;
    Mat Tr((size_t)nt * nt, 0.0), Ti((size_t)nt * nt, 0.0);
    if (eig) {
        for (int i = 0; i < nt; ++i) {
            Tr[i * nt + i] = L.lre[i];
            Ti[i * nt + i] = L.lim[i];
        }
    } else {
        Tr = L.Tcre;
        Ti = L.Tcim;
    }
    const cudaStream_t s = h->stream;
    const double tol = h->opt.minres_tol;
    const int steps = h->opt.minres_maxit > 0 ? h->opt.minres_maxit : minres_bound_steps(tol);
    const DevSpace<T> &ds = space<T>(h);
    double ob, of;
    op_counts(h, (double)ns * nt, nt, sizeof(T), &ob, &of);
    {
        TimeCoefs<T> tc = pack_time<T>(h, l, MODE_RES, true);
        for (int part = 0; part < 2; ++part) {
            const Mat &Yp = part ? Yi : Yr;
            for (int i = 0; i < nt; ++i)
                for (int j = 0; j < nt; ++j) tc.Y[i * NTMAX + j] = (T)Yp[i * nt + j];
            KScope ks(h, cls_of<T>(ST_PROF_STENCIL64, ST_PROF_STENCIL32), ob * 1.5, of);
            CK(launch_stencil<T>(u, f, part ? mw.wi : w.w0, ds.bands, h->g, tc, L.nslab, s0, ns,
                                 s));
        }
    }
    T *Wr = w.w0 + s0 * sl, *Wi = mw.wi + s0 * sl, *Gt = w.w1 + s0 * sl;
    T *Zr = mw.zs, *Zi = mw.zi, *Gr = mw.g0, *Gi = mw.g1;
    {
        KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * ns * sl, 0.0);
        CK(launch_zero<T>(Zr, ns * sl, s));
        CK(launch_zero<T>(Zi, ns * sl, s));
    }
    // out = fin - sign * C_{i, j>i} M_x zin on row i (other rows: fin)
    auto pass = [&](int i, const T *zin, const T *fin, T *out, const Mat &C, double sign) -> int {
        TimeCoefs<T> t2;
        std::memset(&t2, 0, sizeof t2);
        for (int j = i + 1; j < nt; ++j) t2.CK[i * NTMAX + j] = (T)(sign * C[i * nt + j]);
        t2.nt = nt;
        t2.fuse_y = 0;
        t2.mode = MODE_RES;
        KScope ks(h, cls_of<T>(ST_PROF_STENCIL64, ST_PROF_STENCIL32), ob * 1.5, of);
        CK(launch_stencil<T>(zin, fin, out, ds.bands, h->g, t2, 1, 0, ns, s));
        return ST_OK;
    };
    const double Eb = (double)ns * 2 * m;
    for (int i = nt - 1; i >= 0; --i) {
        const T *sr = Wr, *si = Wi;
        bool upper = false;
        for (int j = i + 1; j < nt; ++j)
            if (Tr[i * nt + j] != 0.0 || Ti[i * nt + j] != 0.0) upper = true;
        if (upper) {
            CKS(pass(i, Zr, Wr, Gt, Tr, 1.0));   // w_re - Re T M z_re
            CKS(pass(i, Zi, Gt, Gr, Ti, -1.0));  //      + Im T M z_im
            CKS(pass(i, Zi, Wi, Gt, Tr, 1.0));   // w_im - Re T M z_im
            CKS(pass(i, Zr, Gt, Gi, Ti, 1.0));   //      - Im T M z_re
            sr = Gr;
            si = Gi;
        }
        const double al = Tr[i * nt + i], be = Ti[i * nt + i];
        if (be != 0.0) {
            const BlockCoef bc{al, -be, be};
            {
                KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
                CK(launch_mr_gather<T>(sr, i, si, i, mw.q, 2, nt, m, std::fabs(be), std::fabs(be),
                                       ns, s));
            }
            CKS(block_minres<T>(h, mw, bc, ns, tol, steps, false));
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
            CK(launch_mr_scatter<T>(mw.x, Zr, i, Zi, i, 2, nt, m, 1.0, -1.0, ns, s));
        } else {
            {
                KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
                CK(launch_mr_gather<T>(sr, i, si, i, mw.q, 2, nt, m, 1.0, 1.0, ns, s));
            }
            T *z = nullptr;
            CKS(precond_fd<T>(h, mw.q, mw.z0, mw.z1, &z, ns, 2, al, 1.0, 1.0));
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
            CK(launch_mr_scatter<T>(z, Zr, i, Zi, i, 2, nt, m, 1.0, 1.0, ns, s));
        }
    }
    SchurCoefs<T> sc;
    std::memset(&sc, 0, sizeof sc);
    sc.nt = nt;
    const double E = (double)ns * sl;
    for (int part = 0; part < 2; ++part) {
        const Mat &Xp = part ? Xi : Xr;
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < nt; ++j) sc.X[i * NTMAX + j] = (T)((part ? -1.0 : 1.0) * Xp[i * nt + j]);
        KScope ks(h, ST_PROF_UPDATE, sizeof(T) * 3.0 * E, E * (2.0 * nt + 2.0));
        CK(launch_update<T>(u + s0 * sl, part ? Zi : Zr, sc, omega, h->g, ns, part ? 0 : overwrite,
                            s));
    }
    return ST_OK;
}

// Damped block-Jacobi step on slabs [s0, s0+ns) of level l with the inexact
// spatial solves of Sec. 3.5: w = (Y (x) I)(f - L u) (fused into the
// residual); Algorithm 1 on (Z (x) M_x + I (x) K_x) z = w over the
// standardised real Schur form Z, from the last diagonal block to the
// first: g_B = w_B - sum over the solved blocks j of Z_Bj M_x z_j (one
// operator application with those entries of Z), then a 1x1 block by one
// application of (K_x + Z_bb M_x)^{-1}, a 2x2 block by MinRes; finally
// u <- (overwrite ? 0 : u) + omega (X (x) I) z.
template <typename T>
int smooth_range_minres(st_handle h, int l, T *u, const T *f, T omega, int s0, int ns,
                        int overwrite) {
    Work<T> &w = work<T>(h);
    MrWork<T> &mw = mrwork<T>(h);
    if (ns > mw.cap)
        return fail(ST_ERR_INVALID_ARG, "MinRes batch of %d slabs exceeds its work space (%lld)",
                    ns, mw.cap);
    if (h->opt.variant != ST_RSCHUR)
        return smooth_range_minres_cplx<T>(h, l, u, f, omega, s0, ns, overwrite);
    const int nt = h->nt;
    const long long m = h->g.nxyz, sl = (long long)nt * m;
    const LevelHost &L = h->lv[l];
    const cudaStream_t s = h->stream;
    const double tol = h->opt.minres_tol;
    const int steps = h->opt.minres_maxit > 0 ? h->opt.minres_maxit : minres_bound_steps(tol);
    CKS(stencil<T>(h, l, u, f, w.w0, MODE_RES, true, s0, ns));
    T *W = w.w0 + s0 * sl, *G = w.w1 + s0 * sl, *Zs = mw.zs;
    {
        KScope ks(h, ST_PROF_MINRES, sizeof(T) * (double)ns * sl, 0.0);
        CK(launch_zero<T>(Zs, ns * sl, s));
    }
    double ob, of;
    op_counts(h, (double)ns * nt, nt, sizeof(T), &ob, &of);
    bool first = true;
    for (int i = nt - 1; i >= 0;) {
        const int c = (i >= 1 && L.blk[i]) ? 2 : 1;
        const int b = i - c + 1;
        const T *src = W;
        if (!first) {
            TimeCoefs<T> tc;
            std::memset(&tc, 0, sizeof tc);
            for (int r = b; r < b + c; ++r)
                for (int j = b + c; j < nt; ++j) tc.CK[r * NTMAX + j] = (T)L.Z[r * nt + j];
            tc.nt = nt;
            tc.fuse_y = 0;
            tc.mode = MODE_RES;
            KScope ks(h, cls_of<T>(ST_PROF_STENCIL64, ST_PROF_STENCIL32), ob * 1.5, of);
            CK(launch_stencil<T>(Zs, W, G, space<T>(h).bands, h->g, tc, 1, 0, ns, s));
            src = G;
        }
        first = false;
        const double Eb = (double)ns * c * m;
        if (c == 1) {
            {
                KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
                CK(launch_mr_gather<T>(src, b, src, b, mw.q, 1, nt, m, 1.0, 1.0, ns, s));
            }
            T *z = nullptr;
            CKS(precond_fd<T>(h, mw.q, mw.z0, mw.z1, &z, ns, 1, L.Z[b * nt + b], 1.0, 1.0));
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
            CK(launch_mr_scatter<T>(z, Zs, b, Zs, b, 1, nt, m, 1.0, 1.0, ns, s));
        } else {
            const BlockCoef bc{L.Z[b * nt + b], L.Z[b * nt + b + 1], L.Z[(b + 1) * nt + b]};
            {
                KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
                CK(launch_mr_gather<T>(src, b, src, b + 1, mw.q, 2, nt, m, std::fabs(bc.beta2),
                                       std::fabs(bc.beta1), ns, s));
            }
            CKS(block_minres<T>(h, mw, bc, ns, tol, steps, false));
            KScope ks(h, ST_PROF_MINRES, sizeof(T) * 2.0 * Eb, Eb);
            CK(launch_mr_scatter<T>(mw.x, Zs, b, Zs, b + 1, 2, nt, m, 1.0, -1.0, ns, s));
        }
        i = b - 1;
    }
    const SchurCoefs<T> sc = pack_schur<T>(h, l);
    const double E = (double)ns * sl;
    KScope ks(h, ST_PROF_UPDATE, sizeof(T) * (overwrite ? 2.0 : 3.0) * E, E * (2.0 * nt + 2.0));
    CK(launch_update<T>(u + s0 * sl, Zs, sc, omega, h->g, ns, overwrite, s));
    return ST_OK;
}

// Damped block-Jacobi step on slabs [s0, s0+ns) of level l:
// u <- (overwrite ? 0 : u) + omega A^{-1} (f - L u)  (A^{-1} by Eq. 3.1 + FD)
template <typename T>
int smooth_range(st_handle h, int l, T *u, const T *f, T omega, int s0, int ns, int overwrite) {
    if (h->opt.spatial_solver == ST_SPATIAL_MINRES)
        return smooth_range_minres<T>(h, l, u, f, omega, s0, ns, overwrite);
    Work<T> &w = work<T>(h);
    DevSpace<T> &ds = space<T>(h);
    const long long sl = (long long)h->nt * h->g.nxyz;  // elements per slab
    T *w0 = w.w0 + s0 * sl, *w1 = w.w1 + s0 * sl;
    const bool eig = h->opt.variant != ST_RSCHUR;
    // real Schur: Y fused into the residual, shift solve with Z, X in the
    // update; diagonalisation and complex Schur: the complex Y, the shifted
    // diagonal or triangular solve and X all per mode
    CKS(stencil<T>(h, l, u, f, w.w0, MODE_RES, !eig, s0, ns));
    T *fw = nullptr, *bz = nullptr;
    CKS(spatial<T>(h, w0, w1, w0, true, (long long)ns * h->nt, &fw));
    SchurCoefs<T> sc = pack_schur<T>(h, l);
    const double E = (double)ns * h->nt * h->g.nxyz;
    if (eig) {
        const SpecCoefs<T> c = pack_spec<T>(h, l);
        KScope ks(h, ST_PROF_SHIFT, sizeof(T) * 2.0 * E, E * (5.0 * h->nt + 4.0));
        CK(launch_mode_solve<T>(fw, ds.mu, h->g, c, ns, h->stream));
        for (int i = 0; i < NTMAX; ++i)
            for (int j = 0; j < NTMAX; ++j) sc.X[i * NTMAX + j] = (i == j) ? T(1) : T(0);
    } else {
        KScope ks(h, ST_PROF_SHIFT, sizeof(T) * 2.0 * E, E * (h->nt + 2.0));
        CK(launch_shift_solve<T>(fw, ds.lam[0], ds.lam[1], ds.lam[2], h->g, sc, ns, h->stream));
    }
    T *other = (fw == w0) ? w1 : w0;
    CKS(spatial<T>(h, fw, other, fw, false, (long long)ns * h->nt, &bz));
    {
        KScope ks(h, ST_PROF_UPDATE, sizeof(T) * (overwrite ? 2.0 : 3.0) * E, E * (2.0 * h->nt + 2.0));
        CK(launch_update<T>(u + s0 * sl, bz, sc, omega, h->g, ns, overwrite, h->stream));
    }
    return ST_OK;
}

template <typename T>
int smooth(st_handle h, int l, T *u, const T *f, T omega, int overwrite = 0) {
    return smooth_range<T>(h, l, u, f, omega, 0, h->lv[l].nslab * h->nrhs, overwrite);
}

// Exact solve on the coarsest level: block forward substitution over its
// slabs (a single damped step with omega = 1 when there is one slab).
template <typename T>
int coarse_solve(st_handle h, int l, T *u, const T *f) {
    const int Nl = h->lv[l].nslab;
    CK(launch_zero<T>(u, (long long)Nl * h->nrhs * h->nt * h->g.nxyz, h->stream));
    if (Nl == 1) return smooth<T>(h, l, u, f, T(1), 1);
    for (int r = 0; r < h->nrhs; ++r)
        for (int s = 0; s < Nl; ++s) CKS(smooth_range<T>(h, l, u, f, T(1), r * Nl + s, 1, 0));
    return ST_OK;
}

// One V-cycle on level l for L_l u = f starting from u (zero_init: u = 0).
// Makes level l's spatial grid and factors the handle's current ones for the
// scope (every operator, transform and smoother reads h->g and the DevSpace
// of its precision); restores the previous ones on exit.
struct LevelCtx {
    st_handle h;
    Grid g;
    DevSpace<double> s64;
    DevSpace<float> s32;
    LevelCtx(st_handle h_, int l) : h(h_), g(h_->g), s64(h_->s64), s32(h_->s32) {
        const LevelSpace &S = h->ls[h->lv[l].sp];
        h->g = S.g;
        h->s64 = S.s64;
        h->s32 = S.s32;
    }
    ~LevelCtx() {
        h->g = g;
        h->s64 = s64;
        h->s32 = s32;
    }
};

template <typename T>
const T *const *prolong_mats(const LevelSpace &S);
template <>
const double *const *prolong_mats<double>(const LevelSpace &S) { return S.P64; }
template <>
const float *const *prolong_mats<float>(const LevelSpace &S) { return S.P32; }

// Space transfer between level l (grid F) and level l + 1 (F's spans halved)
// for `planes` time planes: restriction out = (P_z^T (x) P_y^T (x) P_x^T) in
// (fine -> coarse), prolongation out = (P_z (x) P_y (x) P_x) in (coarse ->
// fine), with the 1D knot-insertion matrices P_a of F; one strided GEMM per
// axis, intermediates in t0 / t1, the last axis writes `out`.
template <typename T>
int space_transfer(st_handle h, int l, const T *in, T *t0, T *t1, T *out, bool restr,
                   long long planes) {
    const LevelSpace &F = h->ls[h->lv[l].sp], &Cs = h->ls[h->lv[l + 1].sp];
    const T *const *P = prolong_mats<T>(F);
    long long cur[3];
    for (int a = 0; a < 3; ++a) cur[a] = restr ? F.n[a] : Cs.n[a];
    const T *src = in;
    for (int a = 0; a < h->dim; ++a) {
        const int nf = F.n[a], nc = Cs.n[a];
        const int nin = restr ? nf : nc, nout = restr ? nc : nf;
        long long inner = 1, outer = planes;
        for (int b = 0; b < a; ++b) inner *= cur[b];
        for (int b = a + 1; b < 3; ++b) outer *= cur[b];
        T *dst = (a == h->dim - 1) ? out : ((a % 2 == 0) ? t0 : t1);
        const double E = (double)outer * inner * (nin + nout);
        KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * E, 2.0 * (double)outer * inner * nin * nout);
        if (a == 0) {
            // dst[o][j] = sum_k src[o][k] W[k][j]; W[k][j] = P[k][j] (restr), P[j][k] (prolong)
            CK(launch_gemm_strided<T>(1, (int)outer, nout, nin, src, 0, nin, 1, P[a], 0,
                                      restr ? nc : 1, restr ? 1 : nc, dst, 0, nout, 1, h->stream));
        } else {
            // dst[o][j][i] = sum_k W[k][j] src[o][k][i]
            CK(launch_gemm_strided<T>((int)outer, nout, (int)inner, nin, P[a], 0, restr ? 1 : nc,
                                      restr ? nc : 1, src, (long long)nin * inner, inner, 1, dst,
                                      (long long)nout * inner, inner, 1, h->stream));
        }
        cur[a] = nout;
        src = dst;
    }
    return ST_OK;
}

template <typename T>
int vcycle(st_handle h, int l, T *u, const T *f, bool zero_init) {
    LevelCtx ctx(h, l);
    const long long n_l = (long long)h->lv[l].nslab * h->nrhs * h->nt * h->g.nxyz;
    if (l == h->nlev - 1) return coarse_solve<T>(h, l, u, f);
    if (zero_init) CK(launch_zero<T>(u, n_l, h->stream));
    const T omega = (T)h->opt.omega;
    for (int k = 0; k < h->opt.nu1; ++k) CKS(smooth<T>(h, l, u, f, omega));
    Work<T> &w = work<T>(h);
    CKS(stencil<T>(h, l, u, f, w.w0, MODE_RES, false, 0, h->lv[l].nslab * h->nrhs));
    if (h->lv[l + 1].xstep) {  // space coarsening: same slabs, spans halved
        const long long planes = (long long)h->lv[l].nslab * h->nrhs * h->nt;
        T *xt = static_cast<T *>(h->xtmp);
        CKS(space_transfer<T>(h, l, w.w0, w.w1, xt, w.f[l + 1], true, planes));
        CKS(vcycle<T>(h, l + 1, w.u[l + 1], w.f[l + 1], true));
        CKS(space_transfer<T>(h, l, w.u[l + 1], w.w1, xt, w.w0, false, planes));
        KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * 3.0 * n_l, 1.0 * n_l);
        CK(launch_add<T>(u, w.w0, n_l, h->stream));
    } else if (h->part && l + 1 == h->gathered) {
        // the slab pair of this rank restricts to one coarse slab per rhs;
        // every rank gathers all ranks' coarse slabs, runs the rest of the
        // V-cycle on them and prolongates its own slab of the correction
        const ProlongCoefs<T> pc = pack_prolong<T>(h);
        const int R = h->nrhs, P = h->comm.size, rank = h->comm.rank;
        const long long se = (long long)h->nt * h->g.nxyz;  // one slab
        T *snd = static_cast<T *>(h->agg_send), *rcv = static_cast<T *>(h->agg_recv);
        const double Ec = (double)R * se;
        {
            KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * 3.0 * Ec, Ec * 4.0 * h->nt);
            CK(launch_restrict<T>(w.w0, snd, pc, h->g, R, h->stream));
        }
        CKS(comm_allgather(h, snd, rcv, sizeof(T) * R * se));  // [rank][rhs][slab]
        for (int q = 0; q < P; ++q)  // -> [rhs][rank's slab]
            CK(cudaMemcpy2DAsync(w.f[l + 1] + q * se, P * se * sizeof(T), rcv + q * R * se,
                                 se * sizeof(T), se * sizeof(T), R, cudaMemcpyDeviceToDevice,
                                 h->stream));
        CKS(vcycle<T>(h, l + 1, w.u[l + 1], w.f[l + 1], true));
        CK(cudaMemcpy2DAsync(snd, se * sizeof(T), w.u[l + 1] + rank * se, P * se * sizeof(T),
                             se * sizeof(T), R, cudaMemcpyDeviceToDevice, h->stream));
        {
            KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * 5.0 * Ec, Ec * 4.0 * h->nt);
            CK(launch_prolong_add<T>(snd, u, pc, h->g, R, h->stream));
        }
    } else {
        const ProlongCoefs<T> pc = pack_prolong<T>(h);
        const long long nc = (long long)h->lv[l + 1].nslab * h->nrhs;
        const double Ec = (double)nc * h->nt * h->g.nxyz;
        {
            KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * 3.0 * Ec, Ec * 4.0 * h->nt);
            CK(launch_restrict<T>(w.w0, w.f[l + 1], pc, h->g, nc, h->stream));
        }
        CKS(vcycle<T>(h, l + 1, w.u[l + 1], w.f[l + 1], true));
        {
            KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * 5.0 * Ec, Ec * 4.0 * h->nt);
            CK(launch_prolong_add<T>(w.u[l + 1], u, pc, h->g, nc, h->stream));
        }
    }
    for (int k = 0; k < h->opt.nu2; ++k) CKS(smooth<T>(h, l, u, f, omega));
    return ST_OK;
}

// y_r = post_r (y_r + sum_v coef[v*R + r] x_v), in chunks of MAXV vectors
GLaunch solo_launch(st_handle h);

template <typename T>
int vaxpy(st_handle h, int nv, const T *const *xs, const double *coef, T *y,
          const double *post = nullptr) {
    const int R = h->nrhs;
    GLaunch g = solo_launch(h);
    T *const y1[1] = {y};
    int v0 = 0;
    do {
        const int cnt = std::min(MAXV, nv - v0);
        const bool last = v0 + cnt >= nv;
        for (int r = 0; r < R; ++r) g.snv[r] = cnt;
        KScope ks(h, ST_PROF_VECTOR, sizeof(T) * (cnt + 2.0) * h->len * R, 2.0 * cnt * h->len * R);
        CK(launch_gaxpy<T>(g, cnt, xs ? xs + v0 : nullptr, coef ? coef + (size_t)v0 * R : nullptr,
                           y1, last ? post : nullptr, h->stream));
        ++h->n_vl;
        v0 += cnt;
    } while (v0 < nv);
    return ST_OK;
}

template <typename Tin, typename Tout>
int vconvert(st_handle h, const Tin *x, Tout *y) {
    const double n = (double)h->len * h->nrhs;
    KScope ks(h, ST_PROF_VECTOR, n * (sizeof(Tin) + sizeof(Tout)), 0.0);
    CK(launch_convert<Tin, Tout>(x, y, (long long)n, h->stream));
    return ST_OK;
}

template <typename T>
std::vector<T *> &inv_tabs(st_handle h);
template <>
std::vector<double *> &inv_tabs<double>(st_handle h) { return h->inv64; }
template <>
std::vector<float *> &inv_tabs<float>(st_handle h) { return h->inv32; }

// The per-mode slab inverses (K_t + mu_k M_t)^{-1} of every level (Eq. 3.1
// per spatial mode), formed once in FP64 and kept in precision T.
template <typename T>
int ensure_inv(st_handle h) {
    std::vector<T *> &tabs = inv_tabs<T>(h);
    if ((int)tabs.size() == h->nlev) return ST_OK;
    tabs.assign(h->nlev, nullptr);
    const size_t e = (size_t)h->nt * h->nt * (size_t)h->g.nxyz;
    for (int l = 0; l < h->nlev; ++l) {
        void *p;
        CKS(dalloc(h, e * sizeof(T), &p));
        tabs[l] = (T *)p;
        CK(launch_mode_inverse<T>(tabs[l], h->s64.mu, h->g, pack_spec<double>(h, l), h->stream));
    }
    return ST_OK;
}

// ---- the same V-cycle in the spatial eigenbasis -------------------------------
// u, f are eigenbasis coefficients of level l; tmp is a free buffer of at
// least the level's size.  Identical in exact arithmetic to vcycle() after
// the transforms (I (x) U^T) on the residual and (I (x) U) on the result.
template <typename T>
int svcycle(st_handle h, int l, T *u, const T *f, T *tmp, bool zero_init) {
    NvtxRange range(level_range_name(l));
    const int spp = h->lv[l].nslab;
    const long long ns = (long long)spp * h->nrhs;
    const double E = (double)ns * h->nt * h->g.nxyz;
    const SpecCoefs<T> c = pack_spec<T>(h, l);
    const T *lam = space<T>(h).mu;
    const int nt = h->nt;
    CKS(ensure_inv<T>(h));
    const T *inv = inv_tabs<T>(h)[l];
    // the coarse end of the cycle in one launch: up to 16 slabs per problem
    // (its level vectors in local memory) for a problem with few modes or
    // when no sweeping kernel applies; otherwise the sweeps go on down to 4
    // slabs and the tail's vectors fit in registers (with many modes the
    // local-memory tail spills out of L1: 2.3 ms per cycle for 48^3 x 16
    // right-hand sides at 16 slabs)
    const bool sweeps = h->opt.nu1 >= 2 && h->opt.nu1 <= 6 && h->opt.nu2 >= 2 && h->opt.nu2 <= 6;
    const bool many = (long long)h->g.nxyz * h->nrhs > 152LL * 256;
    const int tail_max = (sweeps && many) ? 4 : 16;
    if (zero_init && spp <= tail_max && l < h->nlev - 1) {
        const double nu = h->opt.nu1 + h->opt.nu2;
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * 2.0 * E, E * nu * (6.0 * nt + 6.0));
        const cudaError_t e = launch_spec_tail<T>(f, u, inv_tabs<T>(h).data() + l, h->nlev - l, h->g,
                                                  pack_prolong<T>(h), (T)h->opt.omega, spp,
                                                  h->nrhs, h->opt.nu1, h->opt.nu2, h->stream);
        if (e == cudaSuccess) return ST_OK;
        if (e != cudaErrorNotSupported) CK(e);
        cudaGetLastError();
    }
    if (l == h->nlev - 1) {
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * (2.0 * E + nt * nt * h->g.nxyz),
                  E * 2.0 * nt);
        CK(launch_spec_coarse<T>(u, f, inv, h->g, nt, spp, h->nrhs, h->stream));
        return ST_OK;
    }
    Work<T> &w = work<T>(h);
    const T omega = (T)h->opt.omega;
    T *cur = u, *oth = tmp;
    bool zero = zero_init;
    const ProlongCoefs<T> pc = pack_prolong<T>(h);
    const long long nc = (long long)h->lv[l + 1].nslab * h->nrhs;
    // nu1 = 2..4 from zero: all steps, the residual and the restriction in
    // one sweeping pass over the level
    bool swept = false;
    if (zero && h->opt.nu1 >= 2 && h->opt.nu1 <= 6) {
        const double nu = h->opt.nu1;
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * 2.5 * E, E * nu * (2.0 * nt + 4.0));
        const cudaError_t e = launch_spec_sweep_down<T>(f, oth, w.f[l + 1], inv, h->g, pc,
                                                        omega, spp, h->nrhs, h->opt.nu1, h->stream);
        if (e == cudaSuccess) {
            std::swap(cur, oth);
            zero = false;
            swept = true;
        } else {
            if (e != cudaErrorNotSupported) CK(e);
            cudaGetLastError();
            ks.cancel();
        }
    }
    // pre-smoothing; the last step runs fused with the residual and the
    // restriction (k_spec_down), the first post-smoothing step with the
    // prolongation (k_spec_up)
    for (int k = 0; !swept && k + 1 < h->opt.nu1; ++k) {
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * (zero ? 2.0 : 3.0) * E, E * (2.0 * nt + 3.0));
        CK(launch_spec_smooth<T>(cur, oth, f, inv, h->g, nt, omega, spp, ns, zero ? 1 : 0,
                                 h->stream));
        std::swap(cur, oth);
        zero = false;
    }
    if (swept) {
    } else if (h->opt.nu1 >= 1) {
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * (zero ? 2.5 : 3.5) * E,
                  E * (zero ? 4.0 * nt + 4.0 : 8.0 * nt + 8.0));
        CK(launch_spec_down<T>(zero ? nullptr : cur, oth, f, w.f[l + 1], inv, lam, h->g, c, pc,
                               omega, spp, nc, h->stream));
        std::swap(cur, oth);
    } else {
        if (zero) CK(launch_zero<T>(cur, (long long)E, h->stream));
        KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * 2.5 * E, E * (4.0 * nt + 2.0));
        CK(launch_spec_res_restrict<T>(cur, f, w.f[l + 1], lam, h->g, c, pc, spp, nc, h->stream));
    }
    CKS(svcycle<T>(h, l + 1, w.u[l + 1], w.f[l + 1], oth, true));
    bool swept_up = false;
    if (h->opt.nu2 >= 2 && h->opt.nu2 <= 6) {
        const double nu = h->opt.nu2;
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * 3.5 * E, E * nu * (2.0 * nt + 3.0));
        const cudaError_t e = launch_spec_sweep_up<T>(w.u[l + 1], cur, oth, f, inv, h->g, pc,
                                                      omega, spp, h->nrhs, h->opt.nu2, h->stream);
        if (e == cudaSuccess) {
            std::swap(cur, oth);
            swept_up = true;
        } else {
            if (e != cudaErrorNotSupported) CK(e);
            cudaGetLastError();
            ks.cancel();
        }
    }
    if (swept_up) {
    } else if (h->opt.nu2 >= 1) {
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * 3.5 * E, E * (4.0 * nt + 4.0));
        CK(launch_spec_up<T>(w.u[l + 1], cur, oth, f, inv, h->g, pc, omega, spp, nc, h->stream));
        std::swap(cur, oth);
    } else {
        const double Ec = (double)nc * nt * h->g.nxyz;
        KScope ks(h, ST_PROF_TRANSFER, sizeof(T) * 5.0 * Ec, Ec * 4.0 * nt);
        CK(launch_prolong_add<T>(w.u[l + 1], cur, pc, h->g, nc, h->stream));
    }
    for (int k = 1; !swept_up && k < h->opt.nu2; ++k) {
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * 3.0 * E, E * (2.0 * nt + 3.0));
        CK(launch_spec_smooth<T>(cur, oth, f, inv, h->g, nt, omega, spp, ns, 0, h->stream));
        std::swap(cur, oth);
    }
    if (cur != u)
        CK(cudaMemcpyAsync(u, cur, sizeof(T) * (size_t)E, cudaMemcpyDeviceToDevice, h->stream));
    return ST_OK;
}

template <typename T>
const SpecCoefs<T> *dev_lvc(st_handle h);
template <>
const SpecCoefs<double> *dev_lvc<double>(st_handle h) { return h->lvc64.data(); }
template <>
const SpecCoefs<float> *dev_lvc<float>(st_handle h) { return h->lvc32.data(); }

// Top of the eigenbasis V-cycle from zero: the whole V-cycle in one
// shared-memory kernel when a mode's levels fit (opt.fused_vcycle), else the
// level-by-level kernels.
template <typename T>
int svcycle_top(st_handle h, T *u, const T *f, T *tmp) {
    if (h->opt.fused_vcycle) {
        const double E = (double)h->len * h->nrhs;
        KScope ks(h, ST_PROF_SPEC, sizeof(T) * 2.0 * E,
                  E * 2.0 * (h->opt.nu1 + h->opt.nu2 + 1) * (7.0 * h->nt + 6.0));
        const cudaError_t e = launch_spec_vcycle<T>(f, u, dev_lvc<T>(h), space<T>(h).mu, h->g,
                                                    pack_prolong<T>(h), h->nlev, h->N, h->nrhs,
                                                    h->opt.nu1, h->opt.nu2, (T)h->opt.omega,
                                                    h->max_smem, h->nsm, h->stream);
        if (e == cudaSuccess) return ST_OK;
        if (e != cudaErrorNotSupported) CK(e);
        cudaGetLastError();
    }
    return svcycle<T>(h, 0, u, f, tmp, true);
}

// z = (I (x) U) V^( (I (x) U^T) v ), FP64 at the interface
template <typename T>
int precondition_spectral(st_handle h, const double *v, double *z);

template <>
int precondition_spectral<double>(st_handle h, const double *v, double *z) {
    Work<double> &w = h->w64;
    const long long planes = (long long)h->N * h->nrhs * h->nt;
    double *fh = nullptr, *e = nullptr;
    CKS(spatial<double>(h, v, w.w0, w.w1, true, planes, &fh));
    double *tmp = (fh == w.w0) ? w.w1 : w.w0;
    CKS(svcycle_top<double>(h, w.u[0], fh, tmp));
    double *t0 = (h->dim % 2 == 1) ? z : w.w0, *t1 = (h->dim % 2 == 1) ? w.w0 : z;
    CKS(spatial<double>(h, w.u[0], t0, t1, false, planes, &e));
    if (e != z) CK(cudaMemcpyAsync(z, e, sizeof(double) * h->len * h->nrhs, cudaMemcpyDeviceToDevice, h->stream));
    return ST_OK;
}

// z = V-cycle(v) with zero initial guess, FP64 at the interface
int precondition_spectral_f32(st_handle h, const double *v, double *z) {
    Work<float> &w = h->w32;
    const long long planes = (long long)h->N * h->nrhs * h->nt;
    CKS((vconvert<double, float>(h, v, w.w0)));
    float *fh = nullptr, *e = nullptr;
    CKS(spatial<float>(h, w.w0, w.w1, w.f[0], true, planes, &fh));
    float *tmp = (fh == w.w1) ? w.w0 : w.w1;
    CKS(svcycle_top<float>(h, w.u[0], fh, tmp));
    float *t0 = (fh == w.w0) ? w.w1 : w.w0;
    float *t1 = (fh == w.f[0]) ? ((t0 == w.w0) ? w.w1 : w.w0) : w.f[0];
    CKS(spatial<float>(h, w.u[0], t0, t1, false, planes, &e));
    CKS((vconvert<float, double>(h, e, z)));
    return ST_OK;
}

int precondition(st_handle h, const double *v, double *z) {
    const long long n0 = h->len * h->nrhs;
    if (h->opt.basis == ST_BASIS_SPECTRAL)
        return h->mixed ? precondition_spectral_f32(h, v, z) : precondition_spectral<double>(h, v, z);
    if (!h->mixed) return vcycle<double>(h, 0, z, v, true);
    Work<float> &w = h->w32;
    CKS((vconvert<double, float>(h, v, w.f[0])));
    CKS(vcycle<float>(h, 0, w.u[0], w.f[0], true));
    CKS((vconvert<float, double>(h, w.u[0], z)));
    (void)n0;
    return ST_OK;
}

int check_ptr(st_handle h, const void *p, const char *name) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (h->host_only) return fail(ST_ERR_INVALID_ARG, "handle was built host-only");
    if (!p) return fail(ST_ERR_INVALID_ARG, "null pointer '%s'", name);
    return ST_OK;
}

int ensure_krylov(st_handle h) {
    const int m = h->opt.gmres_restart;
    if (h->krylov_m == m && !h->V.empty()) return ST_OK;
    const size_t e0 = (size_t)h->len * h->nrhs;
    void *p;
    h->V.clear();
    h->Zk.clear();
    for (int i = 0; i <= m; ++i) {
        CKS(dalloc(h, e0 * sizeof(double), &p));
        h->V.push_back((double *)p);
    }
    for (int i = 0; i < m; ++i) {
        CKS(dalloc(h, e0 * sizeof(double), &p));
        h->Zk.push_back((double *)p);
    }
    h->krylov_m = m;
    return ST_OK;
}

// Run fn() (which enqueues on h->stream) as a CUDA graph keyed by (in, out):
// the first use runs eagerly, the second captures and instantiates a graph on
// a private stream, later uses launch it.  Eager while profiling is on.
template <typename Fn>
int run_graphed(st_handle h, const void *in, void *out, Fn fn) {
    NvtxRange range("preconditioner");
    if (h->prof_on || !h->opt.use_graphs) return fn();
    st_handle_s::GraphRec *g = nullptr;
    for (auto &r : h->graphs)
        if (r.in == in && r.out == out) g = &r;
    if (!g) {
        h->graphs.push_back({in, out, 0, nullptr});
        g = &h->graphs.back();
    }
    if (g->exec) {
        CK(cudaGraphLaunch(g->exec, h->stream));
        return ST_OK;
    }
    if (g->uses++ == 0) return fn();
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    // order the capture after prior work on the handle's stream
    CK(cudaStreamSynchronize(h->stream));
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = fn();
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
    h->stream = user;
    if (rc != ST_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CK(ec);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    g->exec = exec;
    CK(cudaGraphLaunch(g->exec, h->stream));
    return ST_OK;
}

// Small page-locked host blocks, kept for reuse by later handles instead of
// being freed (cudaFreeHost may wait for the whole device, which would stall
// every other stream of a serving process)
std::mutex g_pinned_mu;
std::multimap<size_t, void *> g_pinned_free;  // capacity in bytes -> block

void pinned_put(void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free.emplace(bytes, p);
}

// the page-locked host buffer for count reduced values (grown on demand; the
// stream is idle whenever this runs, every reader synchronises it first)
int host_dots(st_handle h, size_t count) {
    if (count <= h->dots_host_cap) return ST_OK;
    size_t bytes = 4096;
    while (bytes < count * sizeof(double)) bytes <<= 1;
    pinned_put(h->dots_host, h->dots_host_cap * sizeof(double));
    h->dots_host = nullptr;
    h->dots_host_cap = 0;
    void *p = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        auto it = g_pinned_free.lower_bound(bytes);
        if (it != g_pinned_free.end()) {
            bytes = it->first;
            p = it->second;
            g_pinned_free.erase(it);
        }
    }
    if (!p) CK(cudaHostAlloc(&p, bytes, cudaHostAllocPortable));
    h->dots_host = (double *)p;
    h->dots_host_cap = bytes / sizeof(double);
    return ST_OK;
}

// the handle's right-hand sides as a group launch of one member: every
// Krylov vector kernel of a single handle runs the group kernels, so a system
// gets the same arithmetic alone and in a group (st_solve_group)
GLaunch solo_launch(st_handle h) {
    GLaunch g;
    g.nmem = 1;
    g.nsys = h->nrhs;
    g.nblk = h->nblk_dot;
    g.len[0] = h->len;
    g.R[0] = h->nrhs;
    g.part[0] = h->partial;
    for (int r = 0; r < h->nrhs; ++r) g.sr[r] = r;
    return g;
}

// doubles per chunk of a solution copied back by st_solve_host (256 MB:
// about 1.3 ms of the host link, under one Krylov step of a large solve)
constexpr size_t kBgChunk = (size_t)32 << 20;

// Issue the next chunk of the pending solution copies if the previous one
// has completed (all: issue everything now).  Errors are kept for the caller
// of st_solve_host.
void bg_pump(st_handle h, bool all = false) {
    while (!h->bg.empty() && h->bg_err == cudaSuccess) {
        if (!all) {
            const cudaError_t q = cudaEventQuery(h->bg_ev);
            if (q == cudaErrorNotReady) return;
            if (q != cudaSuccess) {
                h->bg_err = q;
                return;
            }
        }
        auto &c = h->bg.front();
        const size_t n = all ? c.n - c.done : std::min(kBgChunk, c.n - c.done);
        cudaError_t e = cudaMemcpyAsync(c.dst + c.done, c.src + c.done, n * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->cp_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->bg_ev, h->cp_out);
        c.done += n;
        if (e == cudaSuccess && c.done == c.n) {
            e = cudaEventRecord(h->hs_out[c.slot], h->cp_out);
            h->bg.pop_front();
        }
        if (e != cudaSuccess) h->bg_err = e;
        if (!all) return;
    }
}

// per-rhs dots of vecs[0..nv) with w -> host out[v*nrhs + r] (FP64 sums)
template <typename T>
int dots(st_handle h, int nv, const T *const *vecs, const T *w, std::vector<double> &out) {
    const size_t cnt_all = (size_t)nv * h->nrhs;
    CKS(host_dots(h, cnt_all));
    const GLaunch g = solo_launch(h);
    const T *const w1[1] = {w};
    for (int v0 = 0; v0 < nv; v0 += MAXV) {
        const int cnt = std::min(MAXV, nv - v0);
        {
            KScope ks(h, ST_PROF_DOT, sizeof(T) * (cnt + 1.0) * h->len * h->nrhs,
                      2.0 * cnt * h->len * h->nrhs);
            CK(launch_gdot<T>(g, cnt, vecs + v0, w1, h->dots, h->stream));
        }
        ++h->n_vl;
        CK(cudaMemcpyAsync(h->dots_host + (size_t)v0 * h->nrhs, h->dots,
                           sizeof(double) * cnt * h->nrhs, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    ++h->n_sync;
    out.assign(h->dots_host, h->dots_host + cnt_all);
    bg_pump(h);
    if (h->part) CKS(comm_allreduce(h, out));
    if (h->recs.size() > 2048) prof_fold(h);
    return ST_OK;
}

template <typename T>
int norms(st_handle h, const T *x, std::vector<double> &nr) {
    std::vector<double> d;
    const T *v[1] = {x};
    CKS(dots<T>(h, 1, v, x, d));
    nr.resize(h->nrhs);
    // a NaN square sum stays NaN (std::max(0.0, NaN) would hide it as 0)
    for (int r = 0; r < h->nrhs; ++r)
        nr[r] = std::isnan(d[r]) ? d[r] : std::sqrt(std::max(0.0, d[r]));
    return ST_OK;
}

// out[(v * 2 + t) * nrhs + r]: dots of vecs[v] with t1 (t = 0) and t2 (t = 1)
template <typename T>
int gram2s(st_handle h, int nv, const T *const *vecs, const T *t1, const T *t2,
           std::vector<double> &out) {
    const size_t cnt_all = (size_t)2 * nv * h->nrhs;
    CKS(host_dots(h, cnt_all));
    const GLaunch g = solo_launch(h);
    const T *const a1[1] = {t1}, *const a2[1] = {t2};
    for (int v0 = 0; v0 < nv; v0 += MAXV) {
        const int cnt = std::min(MAXV, nv - v0);
        {
            KScope ks(h, ST_PROF_DOT, sizeof(T) * (cnt + 2.0) * h->len * h->nrhs,
                      4.0 * cnt * h->len * h->nrhs);
            CK(launch_ggram2<T>(g, cnt, vecs + v0, a1, a2, h->dots, h->stream));
        }
        ++h->n_vl;
        CK(cudaMemcpyAsync(h->dots_host + (size_t)2 * v0 * h->nrhs, h->dots,
                           sizeof(double) * 2 * cnt * h->nrhs, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    ++h->n_sync;
    out.assign(h->dots_host, h->dots_host + cnt_all);
    bg_pump(h);
    if (h->part) CKS(comm_allreduce(h, out));
    if (h->recs.size() > 2048) prof_fold(h);
    return ST_OK;
}

int residual64(st_handle h, const double *u, const double *f, double *r) {
    return stencil<double>(h, 0, u, f, r, MODE_RES, false, 0, h->N * h->nrhs);
}

// The refinement residual r = f - L u of the mixed modes on FP64 data in
// double-float arithmetic (about 48 significant bits, far below the FP32
// inner solve's error) instead of FP64, which runs at 1/64 of the FP32 rate.
int residual_df(st_handle h, const double *u, const double *f, double *r, int sch = 0) {
    NvtxRange range("FP64 residual");
    TimeCoefs<dfloat> tc = pack_time<dfloat>(h, 0, MODE_RES, false);
    CKS(exchange_halo<double>(h, 0, u, &tc.halo));
    // algorithmic work per dof: u and f read, r written (8 bytes each); flops
    // c_d 2(2p+1) for the banded 1D applications of M_x and K_x by sum
    // factorisation (c_1 = 2, c_2 = 5, c_3 = 9), 4 N_t for the time
    // coefficients, 3 for f and the coupling term
    const double E = (double)h->N * h->nrhs * h->nt * h->g.nxyz;
    const double cd = h->dim == 1 ? 2.0 : h->dim == 2 ? 5.0 : 9.0;
    const double fpd = cd * 2.0 * (2 * h->p + 1) + 4.0 * h->nt + 3.0;
    KScope ks(h, ST_PROF_STENCILDF, 8.0 * 3.0 * E, E * fpd);
    CK((launch_stencil<double, dfloat>(u, f, r, space<double>(h).bands, h->g, tc, h->lv[0].nslab,
                                       0, h->N * h->nrhs, h->stream, sch)));
    return ST_OK;
}

// A right-hand side whose norm is not finite (NaN or Inf entries) is an
// argument error: the iteration could never meet the tolerance.
int check_finite_rhs(const std::vector<double> &nf) {
    for (size_t q = 0; q < nf.size(); ++q)
        if (!std::isfinite(nf[q]))
            return fail(ST_ERR_INVALID_ARG, "right-hand side %zu is not finite", q);
    return ST_OK;
}

int solve_mg(st_handle h, const double *rhs, double tol, double *u, st_solve_info *info) {
    CKS(ensure_krylov(h));
    double *r = h->V[0], *e = h->Zk[0];
    std::vector<double> nf, nr;
    CKS(norms<double>(h, rhs, nf));
    CKS(check_finite_rhs(nf));
    int it = 0;
    double worst = 0.0;
    for (;;) {
        CKS(residual64(h, u, rhs, r));
        CKS(norms<double>(h, r, nr));
        worst = 0.0;
        for (int q = 0; q < h->nrhs; ++q) worst = std::max(worst, nf[q] > 0 ? nr[q] / nf[q] : 0.0);
        h->hist.emplace_back(it, worst);
        if (worst <= tol || it >= h->opt.max_it) break;
        CKS(precondition(h, r, e));
        std::vector<double> c(h->nrhs, 1.0);
        const double *xs[1] = {e};
        CKS(vaxpy<double>(h, 1, xs, c.data(), u));
        ++it;
    }
    info->iterations = it;
    info->rel_residual = worst;
    info->status = (worst <= tol) ? ST_OK : ST_ERR_NO_CONVERGENCE;
    return ST_OK;
}

// Flexible GMRES(m) on T vectors for L x = b (per right-hand side), right
// preconditioned by prec(v, z); x holds the initial guess.  Stops each rhs
// at ||b - L x|| <= tol ||b|| (true residual checked at every restart).
// skip[q] excludes rhs q (its x is left unchanged).  *its: iterations,
// *worst: largest relative true residual at exit.
template <typename T, typename Apply, typename Res, typename Prec>
int fgmres_core(st_handle h, const T *b, T *x, double tol, int maxit, std::vector<T *> &V,
                std::vector<T *> &Zk, Apply apply, Res resid, Prec prec, const std::vector<char> &skip,
                int *its, double *worst_out) {
    const int m = (int)Zk.size(), R = h->nrhs;
    std::vector<double> nb, beta, hcol;
    CKS(norms<T>(h, b, nb));
    CKS(check_finite_rhs(nb));
    int total = 0;
    double worst = 0.0;
    std::vector<char> done(R, 0);
    while (true) {
        CKS(resid(x, b, V[0]));
        CKS(norms<T>(h, V[0], beta));
        worst = 0.0;
        for (int q = 0; q < R; ++q) {
            const double rel = nb[q] > 0 ? beta[q] / nb[q] : 0.0;
            done[q] = skip[q] || !(nb[q] > 0) || rel <= tol;
            if (!skip[q]) worst = std::max(worst, rel);
        }
        if (h->record_hist) h->hist.emplace_back(total, worst);
        if (worst <= tol || total >= maxit) break;
        std::vector<double> sc(R);
        for (int q = 0; q < R; ++q) sc[q] = (!done[q] && beta[q] > 0) ? 1.0 / beta[q] : 0.0;
        CKS(vaxpy<T>(h, 0, nullptr, nullptr, V[0], sc.data()));
        // per-rhs Hessenberg (column-major (m+1) x m), Givens, rhs g
        std::vector<double> H((size_t)R * (m + 1) * m, 0.0), cs((size_t)R * m), sn((size_t)R * m),
            g((size_t)R * (m + 1), 0.0);
        std::vector<int> kq(R, 0);
        for (int q = 0; q < R; ++q) g[(size_t)q * (m + 1)] = done[q] ? 0.0 : beta[q];
        std::vector<char> act(R);
        for (int q = 0; q < R; ++q) act[q] = !done[q];
        for (int j = 0; j < m; ++j) {
            CKS(prec(V[j], Zk[j]));
            CKS(apply(Zk[j], V[j + 1]));
            // classical Gram-Schmidt: one fused pass gives V^T w and w.w; a
            // second pass runs only where ||w - V h||^2 < ||w||^2 / 2 (Kahan's
            // "twice is enough" criterion; a looser one lets the FGMRES
            // residual estimate drift from the true residual in FP32).  The
            // decision is taken per right-hand side (a rhs that needs no
            // second pass gets zero coefficients and keeps its first-pass
            // values), so a batch gives each rhs its single-rhs result.
            std::vector<const T *> vw(V.begin(), V.begin() + j + 1);
            vw.push_back(V[j + 1]);
            CKS(dots<T>(h, j + 2, vw.data(), V[j + 1], hcol));
            std::vector<double> hsum((size_t)(j + 1) * R), neg((size_t)(j + 1) * R), rem2(R), post(R);
            std::vector<char> rq(R, 0);
            bool reorth = false;
            for (int q = 0; q < R; ++q) {
                double hh = 0.0;
                for (int i = 0; i <= j; ++i) {
                    const double v = hcol[(size_t)i * R + q];
                    hsum[(size_t)i * R + q] = v;
                    hh += v * v;
                }
                const double ww = hcol[(size_t)(j + 1) * R + q];
                rem2[q] = ww - hh;
                rq[q] = act[q] && rem2[q] < 0.5 * ww;
                reorth = reorth || rq[q];
                for (int i = 0; i <= j; ++i)
                    neg[(size_t)i * R + q] = rq[q] ? -hsum[(size_t)i * R + q] : 0.0;
            }
            if (reorth) {
                CKS(vaxpy<T>(h, j + 1, V.data(), neg.data(), V[j + 1]));
                CKS(dots<T>(h, j + 2, vw.data(), V[j + 1], hcol));
                for (int q = 0; q < R; ++q) {
                    if (!rq[q]) continue;
                    double hh = 0.0;
                    for (int i = 0; i <= j; ++i) {
                        const double v = hcol[(size_t)i * R + q];
                        hsum[(size_t)i * R + q] += v;
                        hh += v * v;
                    }
                    rem2[q] = hcol[(size_t)(j + 1) * R + q] - hh;
                }
            }
            // the remaining projection: the second pass's coefficients where
            // it ran, else the first pass's
            for (int q = 0; q < R; ++q)
                for (int i = 0; i <= j; ++i)
                    neg[(size_t)i * R + q] = rq[q] ? -hcol[(size_t)i * R + q] : -hsum[(size_t)i * R + q];
            std::vector<double> hn(R);
            for (int q = 0; q < R; ++q) {
                hn[q] = std::sqrt(std::max(rem2[q], 0.0));
                post[q] = hn[q] > 0 ? 1.0 / hn[q] : 0.0;
            }
            CKS(vaxpy<T>(h, j + 1, V.data(), neg.data(), V[j + 1], post.data()));
            ++total;
            bool all = true;
            for (int q = 0; q < R; ++q) {
                if (!act[q]) continue;
                double *Hq = &H[(size_t)q * (m + 1) * m];
                double *col = Hq + (size_t)j * (m + 1);
                for (int i = 0; i <= j; ++i) col[i] = hsum[(size_t)i * R + q];
                col[j + 1] = hn[q];
                double *c = &cs[(size_t)q * m], *s = &sn[(size_t)q * m], *gq = &g[(size_t)q * (m + 1)];
                for (int i = 0; i < j; ++i) {
                    const double a = col[i], bb = col[i + 1];
                    col[i] = c[i] * a + s[i] * bb;
                    col[i + 1] = -s[i] * a + c[i] * bb;
                }
                const double a = col[j], bb = col[j + 1];
                const double rad = std::hypot(a, bb);
                c[j] = rad > 0 ? a / rad : 1.0;
                s[j] = rad > 0 ? bb / rad : 0.0;
                col[j] = rad;
                col[j + 1] = 0.0;
                gq[j + 1] = -s[j] * gq[j];
                gq[j] = c[j] * gq[j];
                kq[q] = j + 1;
                if (std::fabs(gq[j + 1]) <= tol * nb[q] || hn[q] == 0.0) act[q] = 0;
                if (act[q]) all = false;
            }
            if (all || total >= maxit) break;
        }
        // x += Z y per rhs
        const int kmax = *std::max_element(kq.begin(), kq.end());
        std::vector<double> coef((size_t)std::max(kmax, 1) * R, 0.0);
        for (int q = 0; q < R; ++q) {
            const int k = kq[q];
            const double *Hq = &H[(size_t)q * (m + 1) * m];
            const double *gq = &g[(size_t)q * (m + 1)];
            std::vector<double> y(k);
            for (int i = k - 1; i >= 0; --i) {
                double sacc = gq[i];
                for (int c2 = i + 1; c2 < k; ++c2) sacc -= Hq[(size_t)c2 * (m + 1) + i] * y[c2];
                y[i] = sacc / Hq[(size_t)i * (m + 1) + i];
            }
            for (int i = 0; i < k; ++i) coef[(size_t)i * R + q] = y[i];
        }
        if (kmax > 0) CKS(vaxpy<T>(h, kmax, Zk.data(), coef.data(), x));
    }
    *its = total;
    *worst_out = worst;
    return ST_OK;
}

// ---- groups of handles (st_solve_group; one handle = a group of one) -------
//
// Members keep their own vectors, operators and preconditioner graphs; the
// group runs their Krylov iterations in lockstep.  Per-member work (operator,
// V-cycle, transforms, residual) is issued on the member's stream; each
// Krylov vector operation of the members taking part is one group launch on
// the group stream (member 0's), ordered after the members' work by events;
// a reduction is read back once for the whole group.
struct Grp {
    std::vector<st_handle> hs;
    std::vector<int> first;            // first system of member k
    int S = 0;                         // systems (right-hand sides) in all
    cudaStream_t G = nullptr;          // group stream
    std::vector<cudaStream_t> own;     // members' streams before the call
    std::vector<cudaEvent_t> ev;       // member k's last work
    cudaEvent_t evg = nullptr;         // the group stream's last work
    bool forked = false;               // members 1.. run on streams of their own
};

// Streams and events the group fans out on, per host thread and device
// (created once, kept for the thread's later groups)
struct ForkPool {
    int dev = -1;
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> e;
};
thread_local ForkPool t_fork;

int fork_pool(int nstreams, int nevents) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (t_fork.dev != dev) {  // the old device's objects stay with it
        t_fork = ForkPool();
        t_fork.dev = dev;
    }
    while ((int)t_fork.s.size() < nstreams) {
        cudaStream_t st;
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        t_fork.s.push_back(st);
    }
    while ((int)t_fork.e.size() < nevents) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        t_fork.e.push_back(e);
    }
    return ST_OK;
}

// Members 1.. move to streams of their own (after the work already queued on
// their own and the group stream); a single member stays on its stream.
int grp_begin(Grp &g, bool fork) {
    const int M = (int)g.hs.size();
    g.first.assign(M, 0);
    g.S = 0;
    for (int k = 0; k < M; ++k) {
        g.first[k] = g.S;
        g.S += g.hs[k]->nrhs;
    }
    g.G = g.hs[0]->stream;
    g.own.resize(M);
    for (int k = 0; k < M; ++k) g.own[k] = g.hs[k]->stream;
    g.forked = fork && M > 1;
    if (!g.forked) return ST_OK;
    CKS(fork_pool(M - 1, M + 1));
    g.ev.assign(t_fork.e.begin(), t_fork.e.begin() + M);
    g.evg = t_fork.e[M];
    CK(cudaEventRecord(g.evg, g.G));
    for (int k = 1; k < M; ++k) {
        cudaStream_t st = t_fork.s[k - 1];
        CK(cudaStreamWaitEvent(st, g.evg, 0));
        CK(cudaEventRecord(g.ev[k], g.own[k]));
        CK(cudaStreamWaitEvent(st, g.ev[k], 0));
        g.hs[k]->stream = st;
    }
    return ST_OK;
}

// the group stream waits for the work of the members in mask
int grp_join(Grp &g, const std::vector<char> &mask) {
    if (!g.forked) return ST_OK;
    for (size_t k = 1; k < g.hs.size(); ++k)
        if (mask[k]) {
            CK(cudaEventRecord(g.ev[k], g.hs[k]->stream));
            CK(cudaStreamWaitEvent(g.G, g.ev[k], 0));
        }
    return ST_OK;
}

// the members in mask wait for the group stream's work
int grp_fork(Grp &g, const std::vector<char> &mask) {
    if (!g.forked) return ST_OK;
    CK(cudaEventRecord(g.evg, g.G));
    for (size_t k = 1; k < g.hs.size(); ++k)
        if (mask[k]) CK(cudaStreamWaitEvent(g.hs[k]->stream, g.evg, 0));
    return ST_OK;
}

// every member's work done, streams handed back, group stream synchronised
int grp_end(Grp &g) {
    std::vector<char> all(g.hs.size(), 1);
    const int rc = grp_join(g, all);
    for (size_t k = 0; k < g.hs.size(); ++k) g.hs[k]->stream = g.own[k];
    if (rc != ST_OK) return rc;
    CK(cudaStreamSynchronize(g.G));
    return ST_OK;
}

// the launch over the systems of the members in mask; sys[i] = the group
// system index of launch system i
GLaunch grp_launch(const Grp &g, const std::vector<char> &mask, std::vector<int> &sys) {
    GLaunch L;
    sys.clear();
    L.nblk = g.hs[0]->nblk_dot;
    for (size_t k = 0; k < g.hs.size(); ++k) {
        if (!mask[k]) continue;
        st_handle h = g.hs[k];
        const int kk = L.nmem++;
        L.len[kk] = h->len;
        L.R[kk] = h->nrhs;
        L.part[kk] = h->partial;
        for (int r = 0; r < h->nrhs; ++r) {
            L.sm[L.nsys] = kk;
            L.sr[L.nsys] = r;
            ++L.nsys;
            sys.push_back(g.first[k] + r);
        }
    }
    return L;
}

// Vector v of member k: vec(v, k).  Members outside mask get no entry.
template <typename T, class Vec>
std::vector<const T *> grp_vecs(const Grp &g, const std::vector<char> &mask, int v0, int nv,
                                Vec vec) {
    std::vector<const T *> out;
    int nm = 0;
    for (size_t k = 0; k < g.hs.size(); ++k) nm += mask[k] ? 1 : 0;
    out.resize((size_t)nv * nm);
    int kk = 0;
    for (size_t k = 0; k < g.hs.size(); ++k) {
        if (!mask[k]) continue;
        for (int v = 0; v < nv; ++v) out[(size_t)v * nm + kk] = vec(v0 + v, (int)k);
        ++kk;
    }
    return out;
}

// out[v * S + s] (group systems; zero for members outside mask) = dot of
// vector v with the target over system s (rows = 1), of vector v with itself
// (rows = 0: the targets are unused), or with rows = 2 the Gram pairs
// out[(2 v + t) * S + s] with targets t1, t2
template <typename T, class Vec, class Tgt1, class Tgt2>
int grp_reduce(Grp &g, const std::vector<char> &mask, int nv, Vec vec, Tgt1 t1, Tgt2 t2,
               int rows_in, std::vector<double> &out) {
    st_handle h0 = g.hs[0];
    const bool self = rows_in == 0;
    const int rows = self ? 1 : rows_in;  // output rows per vector
    std::vector<int> sys;
    const GLaunch L = grp_launch(g, mask, sys);
    out.assign((size_t)rows * nv * g.S, 0.0);
    if (L.nsys == 0) return ST_OK;
    CKS(grp_join(g, mask));
    CKS(host_dots(h0, (size_t)rows * nv * L.nsys));
    std::vector<const T *> a, b;
    for (size_t k = 0; k < g.hs.size(); ++k)
        if (mask[k] && !self) {
            a.push_back(t1((int)k));
            b.push_back(t2((int)k));
        }
    double bytes = 0.0;
    for (size_t k = 0; k < g.hs.size(); ++k)
        if (mask[k]) bytes += (double)g.hs[k]->len * g.hs[k]->nrhs;
    for (int v0 = 0; v0 < nv; v0 += MAXV) {
        const int cnt = std::min(MAXV, nv - v0);
        const std::vector<const T *> xs = grp_vecs<T>(g, mask, v0, cnt, vec);
        {
            KScope ks(h0, ST_PROF_DOT, sizeof(T) * (cnt + (self ? 0 : rows)) * bytes,
                      2.0 * rows * cnt * bytes);
            if (self)
                CK(launch_gnorm2<T>(L, cnt, xs.data(), h0->dots, g.G));
            else if (rows == 1)
                CK(launch_gdot<T>(L, cnt, xs.data(), a.data(), h0->dots, g.G));
            else
                CK(launch_ggram2<T>(L, cnt, xs.data(), a.data(), b.data(), h0->dots, g.G));
        }
        ++h0->n_vl;
        CK(cudaMemcpyAsync(h0->dots_host + (size_t)rows * v0 * L.nsys, h0->dots,
                           sizeof(double) * rows * cnt * L.nsys, cudaMemcpyDeviceToHost, g.G));
    }
    CK(cudaStreamSynchronize(g.G));
    ++h0->n_sync;
    for (int row = 0; row < rows * nv; ++row)
        for (int i = 0; i < L.nsys; ++i)
            out[(size_t)row * g.S + sys[i]] = h0->dots_host[(size_t)row * L.nsys + i];
    bg_pump(h0);
    // a slab-partitioned handle (only ever alone in its group): sum the
    // ranks' partial dots, as the single-handle reductions do
    if (h0->part) CKS(comm_allreduce(h0, out));
    if (h0->recs.size() > 2048) prof_fold(h0);
    return ST_OK;
}

// per-system norms of vector vec(0, k) (group systems of members in mask)
template <typename T, class Vec>
int grp_norms(Grp &g, const std::vector<char> &mask, Vec vec, std::vector<double> &nr) {
    std::vector<double> d;
    auto tgt = [&](int k) { return vec(0, k); };
    CKS((grp_reduce<T>(g, mask, 1, vec, tgt, tgt, 0, d)));
    nr.assign(g.S, 0.0);
    for (int q = 0; q < g.S; ++q) nr[q] = std::isnan(d[q]) ? d[q] : std::sqrt(std::max(0.0, d[q]));
    return ST_OK;
}

// y_s <- post_s (y_s + sum_{v < nvm[k]} coef[v * S + s] x_v) for the members
// in mask (nvm: vectors per member, <= nv; post may be NULL; y_zero: y_s is
// taken as zero and not read, nv <= MAXV)
template <typename T, class Vec, class Tgt>
int grp_axpy(Grp &g, const std::vector<char> &mask, int nv, const std::vector<int> &nvm, Vec vec,
             const double *coef, Tgt y, const double *post, bool y_zero = false) {
    st_handle h0 = g.hs[0];
    std::vector<int> sys;
    GLaunch L = grp_launch(g, mask, sys);
    if (L.nsys == 0) return ST_OK;
    CKS(grp_join(g, mask));
    std::vector<T *> ys;
    double bytes = 0.0;
    for (size_t k = 0; k < g.hs.size(); ++k)
        if (mask[k]) {
            ys.push_back(y((int)k));
            bytes += (double)g.hs[k]->len * g.hs[k]->nrhs;
        }
    std::vector<int> mk;  // group member of launch member kk
    for (size_t k = 0; k < g.hs.size(); ++k)
        if (mask[k]) mk.push_back((int)k);
    int v0 = 0;
    do {
        const int cnt = std::min(MAXV, nv - v0);
        const bool last = v0 + cnt >= nv;
        std::vector<double> c((size_t)std::max(cnt, 1) * L.nsys, 0.0), p(L.nsys, 1.0);
        for (int i = 0; i < L.nsys; ++i) {
            const int k = mk[L.sm[i]];
            L.snv[i] = std::max(0, std::min(cnt, nvm[k] - v0));
            for (int v = 0; v < L.snv[i]; ++v)
                c[(size_t)v * L.nsys + i] = coef[(size_t)(v0 + v) * g.S + sys[i]];
            if (post) p[i] = post[sys[i]];
        }
        const std::vector<const T *> xs = grp_vecs<T>(g, mask, v0, cnt, vec);
        {
            KScope ks(h0, ST_PROF_VECTOR, sizeof(T) * (cnt + 2.0) * bytes, 2.0 * cnt * bytes);
            CK(launch_gaxpy<T>(L, cnt, xs.data(), c.data(), ys.data(),
                               (last && post) ? p.data() : nullptr, g.G, y_zero && v0 == 0));
        }
        ++h0->n_vl;
        v0 += cnt;
    } while (v0 < nv);
    return grp_fork(g, mask);
}

// the delayed Gram-Schmidt two-output update for the members in mask
// (coefficients [v * S + s], scalars [s], group system order)
template <typename T, class Vec, class Tgt1, class Tgt2>
int grp_axpy2(Grp &g, const std::vector<char> &mask, int nv, Vec vec, const std::vector<double> &c1,
              const std::vector<double> &c2, const std::vector<double> &c21,
              const std::vector<double> &p1, const std::vector<double> &p2,
              const std::vector<int> &write1, Tgt1 y1, Tgt2 y2) {
    st_handle h0 = g.hs[0];
    std::vector<int> sys;
    const GLaunch L = grp_launch(g, mask, sys);
    if (L.nsys == 0) return ST_OK;
    CKS(grp_join(g, mask));
    std::vector<T *> a, b;
    double bytes = 0.0;
    for (size_t k = 0; k < g.hs.size(); ++k)
        if (mask[k]) {
            a.push_back(y1((int)k));
            b.push_back(y2((int)k));
            bytes += (double)g.hs[k]->len * g.hs[k]->nrhs;
        }
    const int n = L.nsys;
    std::vector<double> d1((size_t)std::max(nv, 1) * n), d2((size_t)std::max(nv, 1) * n), d21(n),
        q1(n), q2(n);
    std::vector<int> w1(n);
    for (int i = 0; i < n; ++i) {
        const int s = sys[i];
        for (int v = 0; v < nv; ++v) {
            d1[(size_t)v * n + i] = c1[(size_t)v * g.S + s];
            d2[(size_t)v * n + i] = c2[(size_t)v * g.S + s];
        }
        d21[i] = c21[s];
        q1[i] = p1[s];
        q2[i] = p2[s];
    }
    std::vector<int> mk;
    for (size_t k = 0; k < g.hs.size(); ++k)
        if (mask[k]) mk.push_back((int)k);
    for (int i = 0; i < n; ++i) w1[i] = write1[mk[L.sm[i]]];
    const std::vector<const T *> xs = grp_vecs<T>(g, mask, 0, nv, vec);
    {
        KScope ks(h0, ST_PROF_VECTOR, sizeof(T) * (nv + 4.0) * bytes, 4.0 * (nv + 1) * bytes);
        CK(launch_gaxpy2<T>(L, nv, xs.data(), d1.data(), d2.data(), d21.data(), q1.data(),
                            q2.data(), a.data(), b.data(), w1.data(), g.G));
    }
    ++h0->n_vl;
    return grp_fork(g, mask);
}

// Flexible GMRES(m) with classical Gram-Schmidt and DELAYED
// reorthogonalisation (the low-synchronisation scheme of Swirydowicz et al.,
// "Low synchronization Gram-Schmidt and GMRES algorithms", and Bielich et
// al., "Low-synch Gram-Schmidt with delayed reorthogonalization for Krylov
// solvers") on T vectors for every member k in mem, right-preconditioned by
// prec(k, v, z): basis vector j enters step j once-orthogonalised (q~_j); one
// Gram pass over [q_0 .. q_{j-1}, q~_j, w] with the two targets q~_j and
// w = A M^{-1} q~_j gives both the second pass of q~_j (a = Q^T q~_j,
// rho = sqrt(q~_j.q~_j - |a|^2), q_j = (q~_j - Q a) / rho) and the first pass
// of w (b = Q^T w, s_j = q_j^T w = (q~_j.w - a.b) / rho); one two-output
// update writes q_j and q~_{j+1} = (w - Q b - q_j s_j) / nu.  Column j - 1 of
// the Hessenberg matrix is completed one step late: w_{j-1}'s remainder
// nu q~_j = nu (Q a + rho q_j) adds nu a to its entries and nu rho below
// them.  Any vector may be preconditioned in FGMRES (A Z = Q H holds for the
// z actually used), so preconditioning q~_j instead of q_j is exact.  One
// host synchronisation and two passes over the basis per step (CGS2 takes
// two synchronisations and four passes).  Every decision is taken per
// right-hand side and every loop bound per member, so each system gets its
// single-handle (and single-rhs) result; a member that is done waits for the
// others without further work.  b(k), x(k): member k's right-hand side and
// iterate, x zero on entry; V(j, k), Z(j, k): its basis; tol, maxit, its,
// worst per member; skip per group system.
template <typename T, class VB, class VX, class VV, class VZ, class Apply, class Res, class Prec>
int fgmres_group(Grp &g, const std::vector<char> &mem, VB b, VX x, VV V, VZ Zk, int m,
                 const std::vector<double> &tolm, const std::vector<int> &maxit, Apply apply,
                 Res resid, Prec prec, const std::vector<char> &skip, std::vector<int> &its,
                 std::vector<double> &worst) {
    const int M = (int)g.hs.size(), S = g.S;
    const size_t ld = (size_t)m + 1;
    std::vector<int> mq(S);
    for (int k = 0; k < M; ++k)
        for (int r = 0; r < g.hs[k]->nrhs; ++r) mq[g.first[k] + r] = k;
    auto V0 = [&](int, int k) { return (const T *)V(0, k); };
    auto Bv = [&](int, int k) { return (const T *)b(k); };
    std::vector<double> nb, beta, G;
    CKS(grp_norms<T>(g, mem, Bv, nb));
    {
        std::vector<double> chk;
        for (int q = 0; q < S; ++q)
            if (mem[mq[q]]) chk.push_back(nb[q]);
        CKS(check_finite_rhs(chk));
    }
    std::vector<int> total(M, 0);
    worst.assign(M, 0.0);
    std::vector<char> live = mem, done(S, 0);
    // x is zero on entry: the first cycle's residual is b itself (b - L 0
    // has b's bits), so its norm is ||b|| and V_0 = b / ||b|| is formed from
    // b without the operator pass and the second norm
    for (bool first = true;; first = false) {
        NvtxRange range("FGMRES cycle");
        if (first) {
            beta = nb;
        } else {
            for (int k = 0; k < M; ++k)
                if (live[k]) CKS(resid(k, x(k), b(k), V(0, k)));
            CKS(grp_norms<T>(g, live, V0, beta));
        }
        for (int k = 0; k < M; ++k) {
            if (!live[k]) continue;
            double wk = 0.0;
            for (int q = g.first[k]; q < g.first[k] + g.hs[k]->nrhs; ++q) {
                const double rel = nb[q] > 0 ? beta[q] / nb[q] : 0.0;
                done[q] = skip[q] || !(nb[q] > 0) || rel <= tolm[k];
                if (!skip[q]) wk = std::max(wk, rel);
            }
            worst[k] = wk;
            if (g.hs[k]->record_hist) g.hs[k]->hist.emplace_back(total[k], wk);
            if (wk <= tolm[k] || total[k] >= maxit[k]) live[k] = 0;
        }
        bool anylive = false;
        for (int k = 0; k < M; ++k) anylive = anylive || live[k];
        if (!anylive) break;
        {
            std::vector<double> sc(S, 0.0);
            for (int q = 0; q < S; ++q)
                if (live[mq[q]]) sc[q] = (!done[q] && beta[q] > 0) ? 1.0 / beta[q] : 0.0;
            auto Vw = [&](int k) { return V(0, k); };
            if (first) {  // V_0 = sc b, V_0 not read
                std::vector<int> nv1(M, 1);
                CKS((grp_axpy<T>(g, live, 1, nv1, Bv, sc.data(), Vw, nullptr, true)));
            } else {
                std::vector<int> nv0(M, 0);
                CKS((grp_axpy<T>(g, live, 0, nv0, V0, nullptr, Vw, sc.data())));
            }
        }
        std::vector<double> H((size_t)S * ld * m, 0.0), cs((size_t)S * m), sn((size_t)S * m),
            gv((size_t)S * ld, 0.0), nu(S, 0.0);
        std::vector<int> kq(S, 0);
        std::vector<char> act(S, 0), pend(S, 0);
        for (int q = 0; q < S; ++q) {
            if (!live[mq[q]]) continue;
            gv[(size_t)q * ld] = done[q] ? 0.0 : beta[q];
            act[q] = !done[q];
        }
        // complete column col of rhs q with the second pass (a, rho) of the
        // vector below it, rotate it and update the residual estimate
        auto finish_col = [&](int q, int col, const double *a, double rho) {
            double *c = &H[(size_t)q * ld * m + (size_t)col * ld];
            for (int i = 0; i <= col; ++i) c[i] += nu[q] * a[i];
            c[col + 1] = nu[q] * rho;
            double *cq = &cs[(size_t)q * m], *sq = &sn[(size_t)q * m], *gq = &gv[(size_t)q * ld];
            for (int i = 0; i < col; ++i) {
                const double x0 = c[i], x1 = c[i + 1];
                c[i] = cq[i] * x0 + sq[i] * x1;
                c[i + 1] = -sq[i] * x0 + cq[i] * x1;
            }
            const double rad = std::hypot(c[col], c[col + 1]);
            cq[col] = rad > 0 ? c[col] / rad : 1.0;
            sq[col] = rad > 0 ? c[col + 1] / rad : 0.0;
            c[col] = rad;
            c[col + 1] = 0.0;
            gq[col + 1] = -sq[col] * gq[col];
            gq[col] = cq[col] * gq[col];
            kq[q] = col + 1;
            pend[q] = 0;
            if (std::fabs(gq[col + 1]) <= tolm[mq[q]] * nb[q] || rho == 0.0) act[q] = 0;
        };
        // residual estimate if the pending column were completed with a = 0, rho = 1
        auto provisional = [&](int q, int col) {
            std::vector<double> c(&H[(size_t)q * ld * m + (size_t)col * ld],
                                  &H[(size_t)q * ld * m + (size_t)col * ld] + col + 2);
            c[col + 1] = nu[q];
            const double *cq = &cs[(size_t)q * m], *sq = &sn[(size_t)q * m];
            for (int i = 0; i < col; ++i) {
                const double x0 = c[i], x1 = c[i + 1];
                c[i] = cq[i] * x0 + sq[i] * x1;
                c[i + 1] = -sq[i] * x0 + cq[i] * x1;
            }
            const double rad = std::hypot(c[col], c[col + 1]);
            const double s = rad > 0 ? c[col + 1] / rad : 0.0;
            return std::fabs(s * gv[(size_t)q * ld + col]);
        };
        std::vector<char> cyc = live;  // members still in this cycle
        for (int j = 0;; ++j) {
            // (A) rhs whose pending column already meets the tolerance (or
            // every pending rhs at the end of its member's cycle): second pass only
            std::vector<char> last(M, 0), fm(M, 0), fin(S, 0);
            for (int k = 0; k < M; ++k) last[k] = cyc[k] && ((j == m) || total[k] >= maxit[k]);
            bool anyfin = false;
            for (int q = 0; q < S; ++q) {
                const int k = mq[q];
                if (cyc[k] && act[q] && pend[q] &&
                    (last[k] || provisional(q, j - 1) <= tolm[k] * nb[q])) {
                    fin[q] = 1;
                    fm[k] = 1;
                    anyfin = true;
                }
            }
            if (anyfin) {
                auto Vj = [&](int, int k) { return (const T *)V(j, k); };
                auto Vi = [&](int i, int k) { return (const T *)V(i, k); };
                CKS((grp_reduce<T>(g, fm, j + 1, Vi, [&](int k) { return Vj(0, k); },
                                   [&](int k) { return Vj(0, k); }, 1, G)));
                std::vector<double> c1((size_t)std::max(j, 1) * S, 0.0), p1(S, 1.0), a(j);
                std::vector<char> cont(M, 0);  // members with a system that continues
                bool anycont = false;
                for (int q = 0; q < S; ++q) {
                    if (!fin[q]) continue;
                    double aa = 0.0;
                    for (int i = 0; i < j; ++i) {
                        a[i] = G[(size_t)i * S + q];
                        aa += a[i] * a[i];
                    }
                    const double rho = std::sqrt(std::max(G[(size_t)j * S + q] - aa, 0.0));
                    finish_col(q, j - 1, a.data(), rho);
                    if (act[q] && rho > 0) {  // continues: q~_j becomes q_j
                        for (int i = 0; i < j; ++i) c1[(size_t)i * S + q] = -a[i];
                        p1[q] = 1.0 / rho;
                        cont[mq[q]] = 1;
                        anycont = true;
                    }
                }
                // a system that stops here never reads q~_j again (x is
                // updated from the z vectors, a restart rebuilds q_0), so its
                // member's update is left out when none of its systems continues
                if (anycont) {
                    std::vector<int> nvj(M, j);
                    auto Vw = [&](int k) { return V(j, k); };
                    CKS((grp_axpy<T>(g, cont, j, nvj, Vi, c1.data(), Vw, p1.data())));
                }
            }
            bool anycyc = false;
            for (int k = 0; k < M; ++k) {
                if (!cyc[k]) continue;
                bool any = false;
                for (int q = g.first[k]; q < g.first[k] + g.hs[k]->nrhs; ++q) any = any || act[q];
                if (!any || last[k]) cyc[k] = 0;
                anycyc = anycyc || cyc[k];
            }
            if (!anycyc) break;
            // (B) the step: z_j = M^{-1} q~_j, w = A z_j
            for (int k = 0; k < M; ++k) {
                if (!cyc[k]) continue;
                CKS(prec(k, V(j, k), Zk(j, k)));
                CKS(apply(k, Zk(j, k), V(j + 1, k)));
            }
            // (C) one Gram pass, targets q~_j and w
            {
                auto Vi = [&](int i, int k) { return (const T *)V(i, k); };
                CKS((grp_reduce<T>(g, cyc, j + 2, Vi, [&](int k) { return (const T *)V(j, k); },
                                   [&](int k) { return (const T *)V(j + 1, k); }, 2, G)));
            }
            std::vector<double> c1((size_t)std::max(j, 1) * S, 0.0),
                c2((size_t)std::max(j, 1) * S, 0.0), c21(S, 0.0), p1(S, 1.0), p2(S, 1.0), a(j),
                bb(j);
            std::vector<int> write1(M, 0);
            for (int q = 0; q < S; ++q) {
                const int k = mq[q];
                if (!cyc[k] || !act[q]) continue;
                double aa = 0.0, ab = 0.0, b2 = 0.0;
                for (int i = 0; i < j; ++i) {
                    a[i] = pend[q] ? G[((size_t)2 * i) * S + q] : 0.0;
                    bb[i] = G[((size_t)2 * i + 1) * S + q];
                    aa += a[i] * a[i];
                    ab += a[i] * bb[i];
                    b2 += bb[i] * bb[i];
                }
                const double d = G[((size_t)2 * j) * S + q];
                const double cw = G[((size_t)2 * j + 1) * S + q];
                const double e = G[((size_t)2 * (j + 1) + 1) * S + q];
                double rho = 1.0;
                if (pend[q]) {
                    rho = std::sqrt(std::max(d - aa, 0.0));
                    finish_col(q, j - 1, a.data(), rho);
                    if (!act[q]) continue;  // converged at column j - 1
                    write1[k] = 1;
                    for (int i = 0; i < j; ++i) c1[(size_t)i * S + q] = -a[i];
                    p1[q] = 1.0 / rho;
                }
                const double sj = (cw - ab) / rho;
                double *col = &H[(size_t)q * ld * m + (size_t)j * ld];
                for (int i = 0; i < j; ++i) col[i] = bb[i];
                col[j] = sj;
                // |w - Q b - q_j s_j| by Pythagoras; only a scale, the exact
                // norm enters through the next second pass
                const double r2 = e - b2 - sj * sj;
                if (!(e > 0)) {  // w = 0: the Krylov space is invariant
                    nu[q] = 0.0;
                    kq[q] = j;
                    act[q] = 0;
                    continue;
                }
                const double nq = std::sqrt(std::max(r2, 1e-10 * e));
                for (int i = 0; i < j; ++i) c2[(size_t)i * S + q] = -(bb[i] - a[i] * sj / rho);
                c21[q] = -sj / rho;
                p2[q] = 1.0 / nq;
                nu[q] = nq;
                pend[q] = 1;
            }
            {
                auto Vi = [&](int i, int k) { return (const T *)V(i, k); };
                auto Y1 = [&](int k) { return V(j, k); };
                auto Y2 = [&](int k) { return V(j + 1, k); };
                CKS((grp_axpy2<T>(g, cyc, j, Vi, c1, c2, c21, p1, p2, write1, Y1, Y2)));
            }
            for (int k = 0; k < M; ++k) total[k] += cyc[k] ? 1 : 0;
        }
        // x += Z y per rhs, over the members of this cycle
        std::vector<int> kmax(M, 0);
        for (int q = 0; q < S; ++q)
            if (live[mq[q]]) kmax[mq[q]] = std::max(kmax[mq[q]], kq[q]);
        int kall = 0;
        std::vector<char> upd(M, 0);
        for (int k = 0; k < M; ++k) {
            upd[k] = live[k] && kmax[k] > 0;
            kall = std::max(kall, upd[k] ? kmax[k] : 0);
        }
        std::vector<double> coef((size_t)std::max(kall, 1) * S, 0.0);
        for (int q = 0; q < S; ++q) {
            if (!upd[mq[q]]) continue;
            const int k = kq[q];
            const double *Hq = &H[(size_t)q * ld * m];
            const double *gq = &gv[(size_t)q * ld];
            std::vector<double> y(k);
            for (int i = k - 1; i >= 0; --i) {
                double sacc = gq[i];
                for (int c2i = i + 1; c2i < k; ++c2i) sacc -= Hq[(size_t)c2i * ld + i] * y[c2i];
                y[i] = sacc / Hq[(size_t)i * ld + i];
            }
            for (int i = 0; i < k; ++i) coef[(size_t)i * S + q] = y[i];
        }
        if (kall > 0) {
            auto Zi = [&](int i, int k) { return (const T *)Zk(i, k); };
            auto Xw = [&](int k) { return x(k); };
            CKS((grp_axpy<T>(g, upd, kall, kmax, Zi, coef.data(), Xw, nullptr)));
        }
    }
    its = total;
    return ST_OK;
}

int solve_fgmres(st_handle h, const double *rhs, double tol, double *u, st_solve_info *info) {
    CKS(ensure_krylov(h));
    std::vector<double *> Z(h->Zk);
    std::vector<char> skip(h->nrhs, 0);
    int its = 0;
    double worst = 0.0;
    auto apply = [h](const double *z, double *w) {
        return stencil<double>(h, 0, z, nullptr, w, MODE_APPLY, false, 0, h->N * h->nrhs);
    };
    auto prec = [h](const double *v, double *z) {
        return run_graphed(h, v, z, [h, v, z] { return precondition(h, v, z); });
    };
    auto resid = [h](const double *x, const double *b, double *r) {
        return stencil<double>(h, 0, x, b, r, MODE_RES, false, 0, h->N * h->nrhs);
    };
    CKS(fgmres_core<double>(h, rhs, u, tol, h->opt.max_it, h->V, Z, apply, resid, prec, skip,
                            &its, &worst));
    info->iterations = its;
    info->rel_residual = worst;
    info->status = (worst <= tol) ? ST_OK : ST_ERR_NO_CONVERGENCE;
    return ST_OK;
}

// z = V-cycle(v) on FP32 vectors (the mixed modes' inner preconditioner)
int precondition32(st_handle h, const float *v, float *z) {
    Work<float> &w = h->w32;
    if (h->opt.basis != ST_BASIS_SPECTRAL) return vcycle<float>(h, 0, z, v, true);
    const long long planes = (long long)h->N * h->nrhs * h->nt;
    float *fh = nullptr, *e = nullptr;
    CKS(spatial<float>(h, v, w.w0, w.w1, true, planes, &fh));
    float *tmp = (fh == w.w0) ? w.w1 : w.w0;
    CKS(svcycle_top<float>(h, w.u[0], fh, tmp));
    float *t0 = (h->dim % 2 == 1) ? z : w.f[0], *t1 = (h->dim % 2 == 1) ? w.f[0] : z;
    CKS(spatial<float>(h, w.u[0], t0, t1, false, planes, &e));
    if (e != z) CK(cudaMemcpyAsync(z, e, sizeof(float) * h->len * h->nrhs, cudaMemcpyDeviceToDevice, h->stream));
    return ST_OK;
}

int ensure_krylov32(st_handle h) {
    const int m = h->opt.gmres_restart;
    if (h->krylov32_m == m && !h->V32.empty()) return ST_OK;
    const size_t e0 = (size_t)h->len * h->nrhs;
    void *p;
    h->V32.clear();
    h->Z32.clear();
    for (int i = 0; i <= m; ++i) {
        CKS(dalloc(h, e0 * sizeof(float), &p));
        h->V32.push_back((float *)p);
    }
    for (int i = 0; i < m; ++i) {
        CKS(dalloc(h, e0 * sizeof(float), &p));
        h->Z32.push_back((float *)p);
    }
    CKS(dalloc(h, e0 * sizeof(double), &p));
    h->r64 = (double *)p;
    CKS(dalloc(h, e0 * sizeof(float), &p));
    h->rhs32 = (float *)p;
    CKS(dalloc(h, e0 * sizeof(float), &p));
    h->e32 = (float *)p;
    h->krylov32_m = m;
    return ST_OK;
}

// Mixed-precision iterative refinement: FP64 residual r = f - L u and FP64
// update u += ||r|| e, where e solves L e = r / ||r|| approximately by FGMRES
// on FP32 vectors (FP32 operator, FP32 V-cycle) to inner_tol.
// Mixed-precision iterative refinement over a group of members (a single
// handle is the group of one): the refinement steps, FP64 residuals,
// transforms and updates run per member on its stream, the norms and the
// inner FGMRES's vector kernels as group launches.  Each member's loop
// bounds and each system's decisions are the single-handle ones, so every
// right-hand side gets the result st_solve gives it.
int solve_ir_group(Grp &g, const double *const *rhs, double tol, double *const *u,
                   bool guess, st_solve_info *info) {
    const int M = (int)g.hs.size(), S = g.S;
    for (st_handle h : g.hs) CKS(ensure_krylov32(h));
    std::vector<char> all(M, 1);
    std::vector<double> nf(S), nr(S), g0;
    // ||f||, and ||u|| of an initial guess, in one pass: from a zero initial
    // guess the first residual is f itself (without a guess u is not read)
    {
        auto FU = [&](int v, int k) { return v == 0 ? rhs[k] : (const double *)u[k]; };
        auto F = [&](int k) { return rhs[k]; };  // unused by the self dots
        CKS((grp_reduce<double>(g, all, guess ? 2 : 1, FU, F, F, 0, g0)));
    }
    std::vector<char> u_zero(M, 1);
    for (int k = 0; k < M; ++k)
        for (int q = g.first[k]; q < g.first[k] + g.hs[k]->nrhs; ++q) {
            const double f2 = g0[(size_t)0 * S + q];
            nf[q] = std::isfinite(f2) ? std::sqrt(std::max(0.0, f2)) : f2;
            if (guess) u_zero[k] = u_zero[k] && g0[(size_t)1 * S + q] == 0.0;
        }
    CKS(check_finite_rhs(nf));
    std::vector<int> total(M, 0), outer(M, 0);
    std::vector<double> worst(M, 0.0);
    std::vector<char> eig(M);
    std::vector<SpecCoefs<float>> c0(M);
    std::vector<long long> nsl(M);
    for (int k = 0; k < M; ++k) {
        eig[k] = g.hs[k]->opt.basis == ST_BASIS_SPECTRAL;
        c0[k] = pack_spec<float>(g.hs[k], 0);
        nsl[k] = (long long)g.hs[k]->N * g.hs[k]->nrhs;
    }
    // B-spline basis: FP32 stencil operator, V-cycle with its transforms;
    // eigenbasis: pointwise operator L^, V-cycle without transforms
    auto apply = [&](int k, const float *z, float *w) {
        st_handle h = g.hs[k];
        if (!eig[k]) return stencil<float>(h, 0, z, nullptr, w, MODE_APPLY, false, 0, (int)nsl[k]);
        const double E = (double)nsl[k] * h->nt * h->g.nxyz;
        KScope ks(h, ST_PROF_SPEC, 4.0 * 2.25 * E, E * (4.0 * h->nt + 2.0));
        CK(launch_spec_op<float>(z, nullptr, w, h->s32.mu, h->g, c0[k], h->N, nsl[k], 0,
                                 h->stream));
        return (int)ST_OK;
    };
    auto resid = [&](int k, const float *x, const float *b, float *r) {
        st_handle h = g.hs[k];
        if (!eig[k]) return stencil<float>(h, 0, x, b, r, MODE_RES, false, 0, (int)nsl[k]);
        const double E = (double)nsl[k] * h->nt * h->g.nxyz;
        KScope ks(h, ST_PROF_SPEC, 4.0 * 3.25 * E, E * (4.0 * h->nt + 2.0));
        CK(launch_spec_op<float>(x, b, r, h->s32.mu, h->g, c0[k], h->N, nsl[k], 1, h->stream));
        return (int)ST_OK;
    };
    auto prec = [&](int k, const float *v, float *z) {
        st_handle h = g.hs[k];
        if (!eig[k])
            return run_graphed(h, v, z, [h, v, z] { return precondition32(h, v, z); });
        return run_graphed(h, v, z, [h, v, z] { return svcycle_top<float>(h, z, v, h->w32.w0); });
    };
    auto R64 = [&](int, int k) { return (const double *)g.hs[k]->r64; };
    auto B32 = [&](int k) { return (const float *)g.hs[k]->rhs32; };
    auto X32 = [&](int k) { return g.hs[k]->e32; };
    auto VV = [&](int j, int k) { return g.hs[k]->V32[j]; };
    auto ZZ = [&](int j, int k) { return g.hs[k]->Z32[j]; };
    // without a guess u is not zeroed beforehand: a member's first update
    // stores u = 0 + ||r|| e (the bits of an update of a zero u), and a member
    // that never updates (or a solve that fails first) is zeroed on the way out
    struct ZeroUnset {
        Grp &g;
        double *const *u;
        std::vector<char> set;
        ~ZeroUnset() {
            for (size_t k = 0; k < set.size(); ++k)
                if (!set[k])
                    (void)launch_zero<double>(u[k], g.hs[k]->len * g.hs[k]->nrhs, g.hs[k]->stream);
        }
    } u_set{g, u, std::vector<char>(M, guess ? 1 : 0)};
    std::vector<char> run(M, 1);  // members still refining
    for (bool first = true;; first = false) {
        NvtxRange range("refinement step");
        std::vector<char> need(M, 0);
        for (int k = 0; k < M; ++k) {
            if (!run[k]) continue;
            st_handle h = g.hs[k];
            if (first && u_zero[k]) {  // the residual is f itself (read from f below)
                for (int q = g.first[k]; q < g.first[k] + h->nrhs; ++q) nr[q] = nf[q];
            } else {
                CKS(residual_df(h, u[k], rhs[k], h->r64));
                need[k] = 1;
            }
        }
        {
            std::vector<double> nn;
            CKS(grp_norms<double>(g, need, R64, nn));
            for (int k = 0; k < M; ++k)
                if (need[k])
                    for (int q = g.first[k]; q < g.first[k] + g.hs[k]->nrhs; ++q) nr[q] = nn[q];
        }
        std::vector<char> skip(S, 0);
        std::vector<double> sc(S, 0.0), back(S, 0.0);
        bool any = false;
        for (int k = 0; k < M; ++k) {
            if (!run[k]) continue;
            st_handle h = g.hs[k];
            double wk = 0.0;
            for (int q = g.first[k]; q < g.first[k] + h->nrhs; ++q) {
                const double rel = nf[q] > 0 ? nr[q] / nf[q] : 0.0;
                wk = std::max(wk, rel);
                skip[q] = !(nf[q] > 0) || rel <= tol || !(nr[q] > 0);
                sc[q] = skip[q] ? 0.0 : 1.0 / nr[q];
                back[q] = skip[q] ? 0.0 : nr[q];
            }
            worst[k] = wk;
            h->hist.emplace_back(total[k], wk);
            if (wk <= tol || total[k] >= h->opt.max_it || outer[k] >= 60) run[k] = 0;
            any = any || run[k];
        }
        if (!any) break;
        std::vector<double> itol(M, 0.0);
        std::vector<int> maxit(M, 0);
        for (int k = 0; k < M; ++k) {
            if (!run[k]) continue;
            st_handle h = g.hs[k];
            const long long n0 = h->len * h->nrhs;
            const long long planes = (long long)h->N * h->nrhs * h->nt;
            // FP32 right-hand side r / ||r|| in one pass (from f itself on the
            // first step from zero), straight into the buffer the forward
            // transform starts from: it ends in rhs32 (odd axis counts start in
            // w1, even ones in rhs32; no pass is in place)
            const double *src = (first && u_zero[k]) ? rhs[k] : h->r64;
            float *cv = (eig[k] && h->dim % 2 == 1) ? h->w32.w1 : h->rhs32;
            {
                KScope ks(h, ST_PROF_VECTOR, 12.0 * n0, 1.0 * n0);
                CK(launch_convert_scale(src, cv, &sc[g.first[k]], h->nrhs, h->len, h->stream));
            }
            // the two transforms around each inner solve run at full FP32
            // accuracy: their error bounds what one refinement step can gain
            if (eig[k]) {  // r^ = (I (x) U^T) r, into rhs32
                float *rh = nullptr;
                if (h->dim % 2 == 1)
                    CKS(spatial<float>(h, h->w32.w1, h->rhs32, h->w32.w0, true, planes, &rh, true));
                else
                    CKS(spatial<float>(h, h->rhs32, h->w32.w0, h->rhs32, true, planes, &rh, true));
                if (rh != h->rhs32) return fail(ST_ERR_CUDA, "forward transform landed elsewhere");
            }
            CK(launch_zero<float>(h->e32, n0, h->stream));
            itol[k] = std::max(h->opt.inner_tol, 1e-6);
            maxit[k] = h->opt.max_it - total[k];
        }
        std::vector<int> its;
        std::vector<double> w32;
        CKS((fgmres_group<float>(g, run, B32, X32, VV, ZZ, g.hs[0]->opt.gmres_restart, itol, maxit,
                                 apply, resid, prec, skip, its, w32)));
        for (int k = 0; k < M; ++k) {
            if (!run[k]) continue;
            st_handle h = g.hs[k];
            const long long n0 = h->len * h->nrhs;
            const long long planes = (long long)h->N * h->nrhs * h->nt;
            total[k] += its[k];
            ++outer[k];
            const float *corr = h->e32;
            if (eig[k]) {  // e = (I (x) U) e^
                float *eb = nullptr;
                CKS(spatial<float>(h, h->e32, h->w32.w0, h->w32.w1, false, planes, &eb, true));
                corr = eb;
            }
            KScope ks(h, ST_PROF_VECTOR, 12.0 * n0, 2.0 * n0);
            CK(launch_axpy_f32_f64(corr, u[k], &back[g.first[k]], h->nrhs, h->len, h->stream,
                                   !u_set.set[k]));
            u_set.set[k] = 1;
        }
    }
    for (int k = 0; k < M; ++k) {
        info[k].iterations = total[k];
        info[k].refinements = outer[k];
        info[k].rel_residual = worst[k];
        info[k].status = (worst[k] <= tol) ? ST_OK : ST_ERR_NO_CONVERGENCE;
    }
    return ST_OK;
}

int solve_ir(st_handle h, const double *rhs, double tol, double *u, bool guess,
             st_solve_info *info) {
    Grp g;
    g.hs = {h};
    CKS(grp_begin(g, false));
    return solve_ir_group(g, &rhs, tol, &u, guess, info);
}

// Slab partition plan: rank's first slab, its slab count, the first level
// held by every rank (ST_OK or INVALID_ARG).
int partition_plan(int slabs, int size, int rank, int *begin, int *local, int *gathered) {
    if (size < 1 || rank < 0 || rank >= size || slabs < 1 || slabs % size != 0)
        return fail(ST_ERR_INVALID_ARG, "%d slabs cannot be split evenly over %d ranks", slabs, size);
    const int n = slabs / size;
    if (n < 2 || (n & (n - 1)) != 0)
        return fail(ST_ERR_INVALID_ARG, "slabs per rank (%d) must be a power of two >= 2", n);
    int L = 0;
    while ((1 << L) < n) ++L;
    *begin = rank * n;
    *local = n;
    *gathered = L;
    return ST_OK;
}

int setup_impl(st_handle h, int geometry, int degree, const int *spans, int slabs,
               const st_options *opt, void *stream, const st_comm *comm = nullptr) {
    if (opt) h->opt = *opt; else st_options_default(&h->opt);
    st_options &o = h->opt;
    if (geometry < ST_INTERVAL || geometry > ST_CUBE) return fail(ST_ERR_INVALID_ARG, "geometry must be 1..3");
    if (degree < 1) return fail(ST_ERR_INVALID_ARG, "degree must be >= 1");
    if (degree > PMAX) return fail(ST_ERR_UNSUPPORTED, "degree %d > %d is not built", degree, PMAX);
    if (!spans) return fail(ST_ERR_INVALID_ARG, "null spans");
    if (slabs < 1) return fail(ST_ERR_INVALID_ARG, "slabs must be >= 1");
    if (o.ne_per_slab < 1 || o.ne_per_slab + degree > NTMAX)
        return fail(ST_ERR_UNSUPPORTED, "ne_per_slab + degree must be in [2, %d]", NTMAX);
    if (!(o.T > 0) || !(o.theta >= 0) || !(o.omega > 0))
        return fail(ST_ERR_INVALID_ARG, "T > 0, theta >= 0, omega > 0 required");
    if (o.nu1 < 0 || o.nu2 < 0 || o.gmres_restart < 1 || o.gmres_restart > 256 || o.max_it < 0 ||
        o.nrhs < 1 || o.nrhs > 32)
        return fail(ST_ERR_INVALID_ARG, "bad nu1/nu2/gmres_restart/max_it/nrhs");
    if (o.precision < ST_FP64 || o.precision > ST_MIXED_BF16)
        return fail(ST_ERR_INVALID_ARG, "bad precision");
    if (o.basis != ST_BASIS_NODAL && o.basis != ST_BASIS_SPECTRAL)
        return fail(ST_ERR_INVALID_ARG, "bad basis");
    if (o.variant != ST_RSCHUR && o.variant != ST_EIG && o.variant != ST_CSCHUR)
        return fail(ST_ERR_INVALID_ARG, "bad variant");
    if (o.outer < ST_OUTER_FGMRES || o.outer > ST_OUTER_IR)
        return fail(ST_ERR_INVALID_ARG, "bad outer iteration");
    if (!(o.inner_tol > 0) || o.inner_tol >= 1)
        return fail(ST_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
    if (o.spatial_solver != ST_SPATIAL_FD && o.spatial_solver != ST_SPATIAL_MINRES)
        return fail(ST_ERR_INVALID_ARG, "bad spatial_solver");
    if (!(o.space_ratio >= 0)) return fail(ST_ERR_INVALID_ARG, "space_ratio must be >= 0");
    if (o.space_ratio > 0 && o.basis != ST_BASIS_NODAL)
        return fail(ST_ERR_UNSUPPORTED, "space coarsening is built for the B-spline basis");
    if (o.spatial_solver == ST_SPATIAL_MINRES) {
        if (o.basis != ST_BASIS_NODAL)
            return fail(ST_ERR_UNSUPPORTED, "MinRes spatial solves are built for the B-spline basis");
        if (!(o.minres_tol > 0) || o.minres_tol >= 1 || o.minres_maxit < 0 || o.minres_maxit > 1000)
            return fail(ST_ERR_INVALID_ARG, "minres_tol must be in (0, 1), minres_maxit in [0, 1000]");
        if ((long long)slabs * o.nrhs > 32767)
            return fail(ST_ERR_UNSUPPORTED, "MinRes spatial solves take at most 32767 slabs x rhs");
    }
    h->dim = geometry;
    h->p = degree;
    h->N = slabs;
    h->nrhs = o.nrhs;
    h->nt = o.ne_per_slab + degree;
    h->mixed = o.precision != ST_FP64;
    h->stream = (cudaStream_t)stream;
    for (int a = 0; a < 3; ++a) {
        h->spans[a] = (a < h->dim) ? spans[a] : 1;
        if (a < h->dim && spans[a] < 2) return fail(ST_ERR_INVALID_ARG, "spans must be >= 2");
        h->n[a] = (a < h->dim) ? spans[a] + degree - 2 : 1;
        if (h->n[a] < 1) return fail(ST_ERR_INVALID_ARG, "no interior dofs on axis %d", a);
    }
    h->g.nx = h->n[0];
    h->g.ny = h->n[1];
    h->g.nz = h->n[2];
    h->g.dim = h->dim;
    h->g.p = degree;
    h->g.nxyz = (long long)h->n[0] * h->n[1] * h->n[2];
    h->len = (long long)slabs * h->nt * h->g.nxyz;
    if (slabs > 65535 / h->nrhs) return fail(ST_ERR_UNSUPPORTED, "too many slabs x rhs");

    // spatial factors of the finest grid (level 0); coarser grids are added
    // below when the hierarchy coarsens in space
    h->ls.clear();
    h->ls.emplace_back();
    CKS(build_space(h, h->spans, h->ls[0]));
    for (int a = 0; a < h->dim; ++a) {
        h->M1[a] = h->ls[0].M1[a];
        h->K1[a] = h->ls[0].K1[a];
        h->U[a] = h->ls[0].U[a];
        h->lam[a] = h->ls[0].lam[a];
    }
    // time factors per level (theta*h frozen at the finest value)
    const double tau0 = o.T / slabs;
    const double delta = o.theta * tau0 / o.ne_per_slab;
    int Nl = slabs;
    const int nt = h->nt;
    bool space_step = false;
    for (;;) {
        if (space_step) {  // same slabs and time factors, spatial grid halved
            LevelHost L = h->lv.back();
            L.sp = (int)h->ls.size() - 1;
            L.xstep = true;
            h->lv.push_back(L);
        } else {
            LevelHost L;
            L.nslab = Nl;
            L.sp = (int)h->ls.size() - 1;
            L.tau = o.T / Nl;
            host::time_matrices(L.tau, o.ne_per_slab, degree, delta, L.Kt, L.Mt);
            Mat G = L.Kt;  // G = M_t^{-1} K_t
            if (!host::lu_solve(nt, nt, L.Mt, G)) return fail(ST_ERR_NOT_POSITIVE, "M_t is singular");
            std::string err;
            if (!host::real_schur(nt, G, L.X, L.Z, L.blk, err))
                return fail(ST_ERR_ILL_CONDITIONED, "real Schur: %s", err.c_str());
            // MinRes block solves need the standard 2x2 blocks of Sec. 3.5
            if (o.spatial_solver == ST_SPATIAL_MINRES) host::standardize_schur(nt, L.X, L.Z, L.blk);
            // Re lambda > 0 check (Sec. 3.2: a posteriori control of positivity)
            for (int i = 0; i < nt; ++i) {
                double re;
                if (i + 1 < nt && L.blk[i + 1]) {
                    re = 0.5 * (L.Z[i * nt + i] + L.Z[(i + 1) * nt + i + 1]);
                    if (!(re > 0)) return fail(ST_ERR_NOT_POSITIVE, "Re lambda <= 0 on level with %d slabs (use a smaller theta)", Nl);
                    ++i;
                    continue;
                }
                re = L.Z[i * nt + i];
                if (!(re > 0)) return fail(ST_ERR_NOT_POSITIVE, "Re lambda <= 0 on level with %d slabs (use a smaller theta)", Nl);
            }
            // diagonalisation from the Schur form (Sec. 3.3): X, Y = (M_t X)^{-1}
            {
                std::string e2;
                L.eig_ok = host::schur_eigvecs(nt, L.X, L.Z, L.blk, L.lre, L.lim, L.Xre, L.Xim, e2);
                if (L.eig_ok) {
                    Mat MXr = host::matmul(nt, L.Mt, L.Xre), MXi = host::matmul(nt, L.Mt, L.Xim);
                    L.eig_ok = host::complex_inverse(nt, MXr, MXi, L.Yre, L.Yim);
                    L.condX = host::complex_cond2(nt, L.Xre, L.Xim);
                }
                if (o.variant == ST_EIG) {
                    if (!L.eig_ok) return fail(ST_ERR_ILL_CONDITIONED, "diagonalisation failed: %s", e2.c_str());
                    if (!(L.condX <= 1e8))
                        return fail(ST_ERR_ILL_CONDITIONED, "cond(X) = %.3e > 1e8 on the level with %d slabs "
                                    "(use the real Schur variant)", L.condX, Nl);
                }
            }
            // complex Schur form (Sec. 3.4) from the real one, Y_c = (M_t Q_c)^{-1}
            if (o.variant == ST_CSCHUR) {
                std::string e3;
                if (!host::complex_schur(nt, L.X, L.Z, L.blk, L.Qcre, L.Qcim, L.Tcre, L.Tcim, e3))
                    return fail(ST_ERR_ILL_CONDITIONED, "complex Schur: %s", e3.c_str());
                Mat MQr = host::matmul(nt, L.Mt, L.Qcre), MQi = host::matmul(nt, L.Mt, L.Qcim);
                if (!host::complex_inverse(nt, MQr, MQi, L.Ycre, L.Ycim))
                    return fail(ST_ERR_ILL_CONDITIONED, "M_t Q_c singular");
                // K_t Q_c = M_t Q_c T_c
                Mat KQr = host::matmul(nt, L.Kt, L.Qcre), KQi = host::matmul(nt, L.Kt, L.Qcim);
                Mat A1 = host::matmul(nt, MQr, L.Tcre), A2 = host::matmul(nt, MQi, L.Tcim);
                Mat B1 = host::matmul(nt, MQr, L.Tcim), B2 = host::matmul(nt, MQi, L.Tcre);
                double rc = 0.0;
                for (int i = 0; i < nt * nt; ++i)
                    rc = std::max(rc, std::max(std::fabs(KQr[i] - (A1[i] - A2[i])),
                                               std::fabs(KQi[i] - (B1[i] + B2[i]))));
                const double sc = host::frob(L.Kt) + host::frob(L.Mt) * (host::frob(L.Tcre) + host::frob(L.Tcim));
                if (!(rc <= 1e-12 * nt * sc))
                    return fail(ST_ERR_ILL_CONDITIONED, "complex Schur residual %.3e", rc);
            }
            // Y = (M_t X)^{-1}
            Mat MX = host::matmul(nt, L.Mt, L.X);
            L.Y.assign(nt * nt, 0.0);
            for (int i = 0; i < nt; ++i) L.Y[i * nt + i] = 1.0;
            if (!host::lu_solve(nt, nt, MX, L.Y)) return fail(ST_ERR_ILL_CONDITIONED, "M_t X singular");
            // check K_t X = M_t X Z
            Mat KX = host::matmul(nt, L.Kt, L.X), MXZ = host::matmul(nt, MX, L.Z);
            double rr = 0;
            for (int i = 0; i < nt * nt; ++i) rr = std::max(rr, std::fabs(KX[i] - MXZ[i]));
            // backward-error scale of K_t X = M_t X Z: ||K_t|| + ||M_t|| ||Z||
            const double scale = host::frob(L.Kt) + host::frob(L.Mt) * host::frob(L.Z);
            if (rr > 1e-12 * nt * scale)
                return fail(ST_ERR_ILL_CONDITIONED, "time factor residual %.2e (scale %.2e)", rr, scale);
            h->lv.push_back(L);
        }
        // next step: halve the spans while the slabs are diffusion-dominated
        // (tau / h_x^2 above opt.space_ratio; h_x = the largest element),
        // else merge slab pairs; stop at one slab
        const LevelSpace &S = h->ls.back();
        int smin = S.spans[0];
        bool halvable = true;
        for (int a = 0; a < h->dim; ++a) {
            smin = std::min(smin, S.spans[a]);
            if (S.spans[a] % 2 != 0 || S.spans[a] / 2 < 2) halvable = false;
        }
        const double ratio = (o.T / Nl) * (double)smin * smin;
        if (o.space_ratio > 0 && ratio > o.space_ratio && halvable) {
            int cs[3] = {1, 1, 1};
            for (int a = 0; a < h->dim; ++a) cs[a] = S.spans[a] / 2;
            LevelSpace C;
            CKS(build_space(h, cs, C));
            LevelSpace &F = h->ls.back();
            for (int a = 0; a < h->dim; ++a) host::space_prolongation(F.spans[a], degree, F.Pc[a]);
            h->ls.push_back(std::move(C));
            space_step = true;
            continue;
        }
        space_step = false;
        if (Nl % 2 != 0 || Nl == 1) break;
        Nl /= 2;
    }
    h->nlev = (int)h->lv.size();
    host::time_prolongation(tau0, o.ne_per_slab, degree, h->Pt);
    h->work_len = h->len;
    if (comm) {
        // keep the global hierarchy's time factors (they depend on the slab
        // length only); levels below the gathered one hold this rank's slabs
        int begin = 0, local = 0, gathered = 0;
        CKS(partition_plan(slabs, comm->size, comm->rank, &begin, &local, &gathered));
        if (gathered >= h->nlev) return fail(ST_ERR_INVALID_ARG, "partition deeper than the hierarchy");
        h->part = true;
        h->comm = *comm;
        h->slab_begin = begin;
        h->N_global = slabs;
        h->gathered = gathered;
        h->N = local;
        for (int l = 0; l < gathered; ++l) h->lv[l].nslab = local >> l;
        h->len = (long long)local * h->nt * h->g.nxyz;
        long long wl = 0;
        for (int l = 0; l < h->nlev; ++l)
            wl = std::max(wl, (long long)h->lv[l].nslab * h->nt * h->g.nxyz);
        h->work_len = wl;
        h->opt.use_graphs = 0;  // the exchanges run on the host
    }

    if (h->host_only) return ST_OK;

    // device data
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(ST_ERR_CUDA, "no CUDA device");
    }
    {
        int dev = 0, nsm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        h->nsm = nsm > 0 ? nsm : 1;
        void *pe;
        CKS(dalloc(h, sizeof(int), &pe));
        h->tc_err = (int *)pe;
        CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    for (size_t k = 0; k < h->ls.size(); ++k) {
        LevelSpace &S = h->ls[k];
        CKS(upload_space<double>(h, S.s64, S));
        if (h->mixed) CKS(upload_space<float>(h, S.s32, S));
        for (int a = 0; a < h->dim && k + 1 < h->ls.size(); ++a) {
            CKS(upload<double>(h, S.Pc[a], &S.P64[a]));
            if (h->mixed) CKS(upload<float>(h, S.Pc[a], &S.P32[a]));
        }
    }
    h->s64 = h->ls[0].s64;
    if (h->mixed) h->s32 = h->ls[0].s32;
    if (h->ls.size() > 1) {
        void *px;
        CKS(dalloc(h, (size_t)h->len * h->nrhs * (h->mixed ? sizeof(float) : sizeof(double)), &px));
        h->xtmp = px;
    }
    if (h->part) {
        const size_t plane = (size_t)h->nrhs * h->g.nxyz * sizeof(double);
        const size_t slab = (size_t)h->nrhs * h->nt * h->g.nxyz * sizeof(double);
        CKS(dalloc(h, plane, &h->send_plane));
        CKS(dalloc(h, plane, &h->halo));
        CKS(dalloc(h, slab, &h->agg_send));
        CKS(dalloc(h, slab * h->comm.size, &h->agg_recv));
        if (h->comm.host_buffers) {
            h->stage_bytes = slab * (h->comm.size + 1);
            if (cudaMallocHost(&h->stage, h->stage_bytes) != cudaSuccess) {
                cudaGetLastError();
                h->stage = nullptr;
                return fail(ST_ERR_OOM, "pinned staging buffer of %zu bytes", h->stage_bytes);
            }
        }
    }
    if (h->mixed) {
        CKS(alloc_work<float>(h, h->w32, true));
        // the FP64 outer residual needs no FP64 V-cycle buffers except scratch
        void *p;
        CKS(dalloc(h, (size_t)h->len * h->nrhs * sizeof(double), &p));
        h->w64.w0 = (double *)p;
    } else {
        CKS(alloc_work<double>(h, h->w64, true));
    }
    if (o.spatial_solver == ST_SPATIAL_MINRES) {
        auto budgeted = [h](size_t b, void **p) { return dalloc(h, b, p); };
        const long long cap = (long long)slabs * o.nrhs;
        CKS(h->mixed ? alloc_mr<float>(h, h->mr32, cap, true, budgeted)
                     : alloc_mr<double>(h, h->mr64, cap, true, budgeted));
    }
    {
        int dev = 0, ms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&ms, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        h->max_smem = ms > 0 ? ms : 48 * 1024;
        h->lvc64.resize(h->nlev);
        h->lvc32.resize(h->nlev);
        for (int l = 0; l < h->nlev; ++l) {
            h->lvc64[l] = pack_spec<double>(h, l);
            h->lvc32[l] = pack_spec<float>(h, l);
        }
    }
    // the eigenbasis V-cycle's per-mode inverses, in its working precision
    if (o.basis == ST_BASIS_SPECTRAL) CKS(h->mixed ? ensure_inv<float>(h) : ensure_inv<double>(h));
    h->nblk_dot = 3 * h->nsm;  // the dot kernels are register-limited to 3 CTAs per SM
    void *p;
    CKS(dalloc(h, sizeof(double) * 2 * MAXV * h->nrhs * h->nblk_dot, &p));
    h->partial = (double *)p;
    // room for a group launch of up to NSYS_MAX systems (st_solve_group)
    CKS(dalloc(h, sizeof(double) * 2 * MAXV * NSYS_MAX, &p));
    h->dots = (double *)p;
    CKS(host_dots(h, (size_t)2 * MAXV * NSYS_MAX));
    return ST_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free smoothing: work vectors and 1D factors in static device
// memory (see st_smooth_static in include/st_iga.h).
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticFactorPerAxis =
    2 * (size_t)ST_STATIC_MAX_N * (2 * PMAX + 1) + 2 * (size_t)ST_STATIC_MAX_N * ST_STATIC_MAX_N +
    ST_STATIC_MAX_N;
constexpr size_t kStaticDoubles = 2 * (size_t)ST_STATIC_MAX_DOFS + 3 * kStaticFactorPerAxis;

// Shared by every call on a device and kept until the process exits.  Host
// code must not use this name as an address: it only stands for the device
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];
// the public size constant hard-codes the band width 2 * PMAX + 1 = 7
static_assert(2 * PMAX + 1 == 7, "ST_STATIC_SCRATCH_BYTES assumes PMAX = 3");
static_assert(sizeof(g_static_scratch) == (size_t)ST_STATIC_SCRATCH_BYTES,
              "static scratch array and ST_STATIC_SCRATCH_BYTES disagree");

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
double *g_static_addr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device; looked up once
// per device, with that device current.
int static_scratch_addr(double **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(ST_ERR_INVALID_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(ST_ERR_CUDA, "cudaGetSymbolAddress(static scratch) failed: %s",
                        cudaGetErrorString(e));
        g_static_addr[dev] = static_cast<double *>(p);
    }
    *out = g_static_addr[dev];
    return ST_OK;
}

}  // namespace

namespace {
// ST_ERR_TIMEOUT if a tensor-core kernel's bounded wait ran out since the
// last check (the flag is cleared); synchronises the handle's stream.
int check_waits(st_handle h) {
    int err = 0;
    CK(cudaMemcpyAsync(&err, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (err) {
        CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
        return fail(ST_ERR_TIMEOUT, "a tensor-core transform's bounded wait ran out");
    }
    return ST_OK;
}
int vcycle_entry(st_handle h, double *u, const double *f);
}  // namespace

int st::prepare_solve(st_handle_s *h) {
    if (!h || h->host_only) return ST_ERR_INVALID_ARG;
    if (h->opt.outer == ST_OUTER_IR && h->mixed) return ensure_krylov32(h);
    return ensure_krylov(h);
}

extern "C" {

void st_options_default(st_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->T = 1.0;
    o->theta = 1.0;
    o->omega = 0.5;
    o->ne_per_slab = 2;
    o->nu1 = 1;
    o->nu2 = 1;
    o->precision = ST_FP64;
    o->outer = ST_OUTER_FGMRES;
    o->gmres_restart = 20;
    o->max_it = 200;
    o->nrhs = 1;
    o->hbm_budget = 0;
    o->basis = ST_BASIS_NODAL;
    o->inner_tol = 1e-4;
    o->use_graphs = 1;
    o->variant = ST_RSCHUR;
    o->autotune = 1;
    o->fused_vcycle = 0;
    o->spatial_solver = ST_SPATIAL_FD;
    o->minres_tol = 1e-4;
    o->minres_maxit = 0;
    o->space_ratio = 0.0;
}

const char *st_last_error(void) { return g_err.c_str(); }

static int setup_entry(st_handle *out, int geometry, int degree, const int *spans, int slabs,
                       const st_options *opt, void *stream, bool host_only,
                       cudaMemPool_t pool = nullptr, const st_comm *comm = nullptr) {
    if (!out) return fail(ST_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    st_handle h = nullptr;
    try {
        h = new st_handle_s();
        h->host_only = host_only;
        h->pool = pool;
        const int rc = setup_impl(h, geometry, degree, spans, slabs, opt, stream, comm);
        if (rc != ST_OK) {
            st_destroy(h);
            return rc;
        }
    } catch (...) {
        if (h) st_destroy(h);
        return fail(ST_ERR_OOM, "host exception during setup");
    }
    *out = h;
    g_err.clear();
    return ST_OK;
}

int st_setup(st_handle *out, int geometry, int degree, const int *spans, int slabs,
             const st_options *opt, void *stream) {
    NvtxRange range("st_setup");
    return setup_entry(out, geometry, degree, spans, slabs, opt, stream, false);
}

int st_setup_host(st_handle *out, int geometry, int degree, const int *spans, int slabs,
                  const st_options *opt) {
    NvtxRange range("st_setup_host");
    return setup_entry(out, geometry, degree, spans, slabs, opt, nullptr, true);
}

int st_setup_partitioned(st_handle *out, int geometry, int degree, const int *spans,
                         int slabs_global, const st_options *opt, const st_comm *comm,
                         void *stream) {
    NvtxRange range("st_setup_partitioned");
    if (out) *out = nullptr;
    if (!comm || !comm->sendrecv || !comm->allgather || !comm->allreduce_sum || comm->size < 1 ||
        comm->rank < 0 || comm->rank >= comm->size)
        return fail(ST_ERR_INVALID_ARG, "bad communicator");
    st_options o;
    if (opt) o = *opt; else st_options_default(&o);
    if (o.basis != ST_BASIS_NODAL || o.spatial_solver != ST_SPATIAL_FD || o.space_ratio != 0 ||
        o.fused_vcycle)
        return fail(ST_ERR_UNSUPPORTED, "a partitioned handle runs the B-spline-basis V-cycle with "
                    "exact spatial solves and time coarsening only");
    return setup_entry(out, geometry, degree, spans, slabs_global, &o, stream, false, nullptr, comm);
}

int st_partition_plan(int slabs_global, int size, int rank, int *slab_begin, int *slabs_local,
                      int *gathered_level) {
    int b = 0, n = 0, g = 0;
    CKS(partition_plan(slabs_global, size, rank, &b, &n, &g));
    if (slab_begin) *slab_begin = b;
    if (slabs_local) *slabs_local = n;
    if (gathered_level) *gathered_level = g;
    return ST_OK;
}

void st_destroy(st_handle h) {
    if (!h) return;
    for (auto &g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (void *p : h->allocs) {
        if (h->pool)
            cudaFreeAsync(p, h->stream);  // stream-ordered: no device-wide synchronisation
        else
            cudaFree(p);
    }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (int s = 0; s < 2; ++s)
        for (cudaEvent_t e : {h->hs_in[s], h->hs_solved[s], h->hs_out[s]})
            if (e) cudaEventDestroy(e);
    if (h->bg_ev) cudaEventDestroy(h->bg_ev);
    if (h->cp_in) cudaStreamDestroy(h->cp_in);
    if (h->cp_out) cudaStreamDestroy(h->cp_out);
    if (h->stage) cudaFreeHost(h->stage);
    pinned_put(h->dots_host, h->dots_host_cap * sizeof(double));
    delete h;
}

int st_set_stream(st_handle h, void *stream) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    h->stream = (cudaStream_t)stream;
    return ST_OK;
}

int st_sizes(st_handle h, int64_t *n_dofs, int *n_t, int *n_x, int *n_levels, size_t *bytes) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (n_dofs) *n_dofs = h->len * h->nrhs;
    if (n_t) *n_t = h->nt;
    if (n_x)
        for (int a = 0; a < 3; ++a) n_x[a] = h->n[a];
    if (n_levels) *n_levels = h->nlev;
    if (bytes) *bytes = h->bytes;
    return ST_OK;
}

int st_apply(st_handle h, const double *x, double *y) {
    NvtxRange range("st_apply");
    CKS(check_ptr(h, x, "x"));
    CKS(check_ptr(h, y, "y"));
    if ((const void *)x == (void *)y) return fail(ST_ERR_INVALID_ARG, "x and y alias");
    return stencil<double>(h, 0, x, nullptr, y, MODE_APPLY, false, 0, h->N * h->nrhs);
}

int st_residual(st_handle h, const double *u, const double *f, double *r) {
    CKS(check_ptr(h, u, "u"));
    CKS(check_ptr(h, f, "f"));
    CKS(check_ptr(h, r, "r"));
    if ((const void *)u == (void *)r) return fail(ST_ERR_INVALID_ARG, "u and r alias");
    return residual64(h, u, f, r);
}

int st_residual_df(st_handle h, const double *u, const double *f, double *r, int slabs_per_cta) {
    CKS(check_ptr(h, u, "u"));
    CKS(check_ptr(h, f, "f"));
    CKS(check_ptr(h, r, "r"));
    if ((const void *)u == (void *)r) return fail(ST_ERR_INVALID_ARG, "u and r alias");
    if (slabs_per_cta != 0 && slabs_per_cta != 1 && slabs_per_cta != 2 && slabs_per_cta != 4 &&
        slabs_per_cta != 8)
        return fail(ST_ERR_INVALID_ARG, "slabs_per_cta must be 0, 1, 2, 4 or 8");
    return residual_df(h, u, f, r, slabs_per_cta);
}

int st_load_coeffs(st_handle h, const double *c, double *f) {
    CKS(check_ptr(h, c, "c"));
    CKS(check_ptr(h, f, "f"));
    if ((const void *)c == (void *)f) return fail(ST_ERR_INVALID_ARG, "c and f alias");
    return stencil<double>(h, 0, c, nullptr, f, MODE_MASS, false, 0, h->N * h->nrhs);
}

int st_load_gaussians(st_handle h, int nbumps, const double *centers, const double *widths,
                      const double *amps, double *f) {
    CKS(check_ptr(h, f, "f"));
    if (nbumps < 0 || (nbumps > 0 && (!centers || !widths || !amps)))
        return fail(ST_ERR_INVALID_ARG, "bad bump arrays");
    const int d = h->dim, nt = h->nt, N = h->N, ne = h->opt.ne_per_slab, p = h->p;
    const long long nst = (long long)N * nt;
    const long long per = nst + h->n[0] + h->n[1] + h->n[2];
    if ((long long)nbumps * per > h->len * h->nrhs)
        return fail(ST_ERR_INVALID_ARG, "too many bumps for the work space");
    // slabs of a partitioned handle start at global slab slab_begin
    const double tau = h->opt.T / (h->part ? h->N_global : N), delta = h->opt.theta * tau / ne;
    const int npts = 2 * p + 4;
    std::vector<double> g((size_t)nbumps * per, 0.0);
    for (int k = 0; k < nbumps; ++k) {
        const double w = widths[k], a = amps[k];
        if (!(w > 0)) return fail(ST_ERR_INVALID_ARG, "bump width must be > 0");
        double *gk = g.data() + (size_t)k * per;
        const double ct = centers[k * (d + 1) + d];
        auto ft = [=](double t) { return a * std::exp(-(t - ct) * (t - ct) / (2 * w * w)); };
        for (int n = 0; n < N; ++n) {
            const int ng = n + h->slab_begin;
            const std::vector<double> gt = host::load_1d(ng * tau, (ng + 1) * tau, ne, p, delta, false, npts, ft);
            for (int j = 0; j < nt; ++j) gk[(size_t)n * nt + j] = gt[j];
        }
        long long off = nst;
        for (int ax = 0; ax < 3; ++ax) {
            if (ax < d) {
                const double c = centers[k * (d + 1) + ax];
                auto fx = [=](double x) { return std::exp(-(x - c) * (x - c) / (2 * w * w)); };
                const std::vector<double> gx = host::load_1d(0.0, 1.0, h->spans[ax], p, 0.0, true, npts, fx);
                for (int i = 0; i < h->n[ax]; ++i) gk[off + i] = gx[i];
            } else {
                gk[off] = 1.0;
            }
            off += h->n[ax];
        }
    }
    if (nbumps == 0) {
        CK(launch_zero<double>(f, h->len * h->nrhs, h->stream));
        return ST_OK;
    }
    double *dg = h->w64.w0;  // the handle's FP64 scratch holds the 1D loads
    CK(cudaMemcpyAsync(dg, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    for (int r = 0; r < h->nrhs; ++r)
        CK(launch_separable_sum(f + r * h->len, dg, nbumps, nst, h->n[0], h->n[1], h->n[2], h->stream));
    CK(cudaStreamSynchronize(h->stream));  // g (host) must outlive the copy
    return ST_OK;
}

int st_smooth(st_handle h, double *u, const double *f, int nsteps) {
    NvtxRange range("st_smooth");
    CKS(check_ptr(h, u, "u"));
    CKS(check_ptr(h, f, "f"));
    if (nsteps < 0) return fail(ST_ERR_INVALID_ARG, "nsteps < 0");
    if (!h->mixed) {
        for (int k = 0; k < nsteps; ++k) CKS(smooth<double>(h, 0, u, f, h->opt.omega));
        return ST_OK;
    }
    const long long n0 = h->len * h->nrhs;
    CK(launch_convert<double, float>(u, h->w32.u[0], n0, h->stream));
    CK(launch_convert<double, float>(f, h->w32.f[0], n0, h->stream));
    for (int k = 0; k < nsteps; ++k)
        CKS(smooth<float>(h, 0, h->w32.u[0], h->w32.f[0], (float)h->opt.omega));
    CK(launch_convert<float, double>(h->w32.u[0], u, n0, h->stream));
    return ST_OK;
}

int st_block_minres(st_handle h, double alpha, double beta1, double beta2, const double *f,
                    double *u, int nsys, double tol, int maxit, int *iters, double *relres) {
    CKS(check_ptr(h, f, "f"));
    CKS(check_ptr(h, u, "u"));
    if ((const void *)f == (const void *)u) return fail(ST_ERR_INVALID_ARG, "f and u alias");
    if (nsys < 1 || nsys > 32767) return fail(ST_ERR_INVALID_ARG, "nsys must be in [1, 32767]");
    if (!(alpha > 0) || !(beta1 * beta2 < 0))
        return fail(ST_ERR_INVALID_ARG, "need alpha > 0 and beta1 * beta2 < 0 (a complex pair)");
    if (!(tol > 0) || tol >= 1 || maxit < 0 || maxit > 100000)
        return fail(ST_ERR_INVALID_ARG, "tol must be in (0, 1), maxit in [0, 100000]");
    const int steps = maxit > 0 ? maxit : minres_bound_steps(tol);
    // one-off work space in plain device memory, released on every return
    struct Tmp {
        std::vector<void *> p;
        ~Tmp() {
            for (void *q : p) cudaFree(q);
        }
    } tmp;
    auto plain = [&tmp](size_t b, void **out) {
        void *q = nullptr;
        const cudaError_t e = cudaMalloc(&q, b ? b : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ST_ERR_OOM, "cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
        }
        tmp.p.push_back(q);
        *out = q;
        return ST_OK;
    };
    MrWork<double> w;
    CKS(alloc_mr<double>(h, w, nsys, false, plain));
    const long long m = h->g.nxyz;
    const BlockCoef bc{alpha, beta1, beta2};
    CK(launch_mr_gather<double>(f, 0, f, 1, w.q, 2, 2, m, std::fabs(beta2), std::fabs(beta1), nsys,
                                h->stream));
    CKS(block_minres<double>(h, w, bc, nsys, tol, steps, true));
    CK(launch_mr_scatter<double>(w.x, u, 0, u, 1, 2, 2, m, 1.0, -1.0, nsys, h->stream));
    std::vector<MrState> hs(nsys);
    CK(cudaMemcpyAsync(hs.data(), w.st, sizeof(MrState) * nsys, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    bool ok = true;
    for (int i = 0; i < nsys; ++i) {
        if (iters) iters[i] = hs[i].iters;
        if (relres) relres[i] = hs[i].relres;
        if (!(hs[i].relres <= tol)) ok = false;
    }
    if (!ok) return fail(ST_ERR_NO_CONVERGENCE, "MinRes stopped at %d steps above tol %.3e", steps, tol);
    return ST_OK;
}

int st_vcycle(st_handle h, double *u, const double *f) {
    NvtxRange range("st_vcycle");
    CKS(check_ptr(h, u, "u"));
    CKS(check_ptr(h, f, "f"));
    const int rc = vcycle_entry(h, u, f);
    if (rc != ST_OK) return rc;
    return check_waits(h);
}

int st_solve_history(st_handle h, int cap, int *its, double *res, int *n) {
    if (!h || cap < 0) return fail(ST_ERR_INVALID_ARG, "null handle or negative capacity");
    const int k = std::min(cap, (int)h->hist.size());
    for (int i = 0; i < k; ++i) {
        if (its) its[i] = h->hist[i].first;
        if (res) res[i] = h->hist[i].second;
    }
    if (n) *n = (int)h->hist.size();
    return ST_OK;
}

int st_set_wait_limit(st_handle h, double seconds) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (!(seconds >= 0) || seconds > 60) return fail(ST_ERR_INVALID_ARG, "wait limit must be in [0, 60] s");
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    return ST_OK;
}

}  // extern "C"

namespace {
int vcycle_entry(st_handle h, double *u, const double *f) {
    if (h->opt.basis == ST_BASIS_SPECTRAL) {
        // the V-cycle is the affine iteration u + B (f - L u)
        CKS(ensure_krylov(h));
        CKS(residual64(h, u, f, h->V[0]));
        CKS(precondition(h, h->V[0], h->Zk[0]));
        const double one[1] = {1.0};
        std::vector<double> c(h->nrhs, 1.0);
        const double *xs[1] = {h->Zk[0]};
        (void)one;
        return vaxpy<double>(h, 1, xs, c.data(), u);
    }
    if (!h->mixed) return vcycle<double>(h, 0, u, f, false);
    const long long n0 = h->len * h->nrhs;
    CK(launch_convert<double, float>(u, h->w32.u[0], n0, h->stream));
    CK(launch_convert<double, float>(f, h->w32.f[0], n0, h->stream));
    CKS(vcycle<float>(h, 0, h->w32.u[0], h->w32.f[0], false));
    CK(launch_convert<float, double>(h->w32.u[0], u, n0, h->stream));
    return ST_OK;
}
}  // namespace

extern "C" {

int st_solve(st_handle h, const double *rhs, double tol, double *u, int use_guess,
             st_solve_info *info) {
    NvtxRange range("st_solve");
    CKS(check_ptr(h, rhs, "rhs"));
    CKS(check_ptr(h, u, "u"));
    if ((const void *)rhs == (void *)u) return fail(ST_ERR_INVALID_ARG, "rhs and u alias");
    if (!(tol > 0)) return fail(ST_ERR_INVALID_ARG, "tol must be > 0");
    st_solve_info local;
    if (!info) info = &local;
    std::memset(info, 0, sizeof *info);
    if (h->opt.autotune && !h->tuned) CKS(autotune(h));
    const auto t0 = std::chrono::steady_clock::now();
    try {
        const bool ir = h->opt.outer == ST_OUTER_IR && h->mixed;
        if (!use_guess && !ir) CK(launch_zero<double>(u, h->len * h->nrhs, h->stream));
        h->hist.clear();
        h->n_sync = h->n_vl = 0;
        if (h->opt.outer == ST_OUTER_MG) {
            CKS(solve_mg(h, rhs, tol, u, info));
        } else if (ir) {  // writes u itself without a guess; records its refinement steps
            CKS(solve_ir(h, rhs, tol, u, use_guess != 0, info));
        } else {
            h->record_hist = true;
            const int rc = solve_fgmres(h, rhs, tol, u, info);
            h->record_hist = false;
            if (rc != ST_OK) return rc;
        }
        CKS(check_waits(h));
    } catch (...) {
        return fail(ST_ERR_OOM, "host exception during solve");
    }
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->host_syncs = (int)h->n_sync;
    info->vector_launches = (int)h->n_vl;
    if (info->status != ST_OK)
        return fail(info->status, "no convergence: rel. residual %.3e after %d iterations",
                    info->rel_residual, info->iterations);
    return ST_OK;
}

int st_solve_group(int n, const st_handle *hs, const double *const *rhs, double tol,
                   double *const *u, int use_guess, st_solve_info *info) {
    NvtxRange range("st_solve_group");
    if (n < 1 || n > GH) return fail(ST_ERR_INVALID_ARG, "a group has 1 to %d handles", GH);
    if (!hs || !rhs || !u) return fail(ST_ERR_INVALID_ARG, "null array");
    if (!(tol > 0)) return fail(ST_ERR_INVALID_ARG, "tol must be > 0");
    int S = 0;
    for (int k = 0; k < n; ++k) {
        st_handle h = hs[k];
        CKS(check_ptr(h, rhs[k], "rhs"));
        CKS(check_ptr(h, u[k], "u"));
        if ((const void *)rhs[k] == (void *)u[k])
            return fail(ST_ERR_INVALID_ARG, "rhs and u of member %d alias", k);
        for (int j = 0; j < k; ++j)
            if (hs[j] == h) return fail(ST_ERR_INVALID_ARG, "handle %d appears twice", k);
        if (h->part) return fail(ST_ERR_UNSUPPORTED, "member %d is slab-partitioned", k);
        if (!h->mixed || h->opt.outer != ST_OUTER_IR)
            return fail(ST_ERR_UNSUPPORTED,
                        "st_solve_group solves mixed-precision handles with ST_OUTER_IR");
        if (h->opt.gmres_restart != hs[0]->opt.gmres_restart)
            return fail(ST_ERR_INVALID_ARG, "members differ in gmres_restart");
        S += h->nrhs;
    }
    if (S > NSYS_MAX)
        return fail(ST_ERR_INVALID_ARG, "%d right-hand sides in the group (at most %d)", S, NSYS_MAX);
    std::vector<st_solve_info> local(n);
    if (!info) info = local.data();
    std::memset(info, 0, sizeof(st_solve_info) * n);
    for (int k = 0; k < n; ++k)
        if (hs[k]->opt.autotune && !hs[k]->tuned) CKS(autotune(hs[k]));
    const auto t0 = std::chrono::steady_clock::now();
    Grp g;
    g.hs.assign(hs, hs + n);
    CKS(grp_begin(g, true));
    int rc = ST_OK;
    try {
        for (int k = 0; k < n && rc == ST_OK; ++k) {
            st_handle h = hs[k];  // the refinement writes u itself without a guess
            h->hist.clear();
            h->n_sync = h->n_vl = 0;
        }
        if (rc == ST_OK) rc = solve_ir_group(g, rhs, tol, u, use_guess != 0, info);
    } catch (...) {
        rc = fail(ST_ERR_OOM, "host exception during solve");
    }
    const int rc_end = grp_end(g);  // the members' streams handed back in every case
    if (rc != ST_OK) return rc;
    if (rc_end != ST_OK) return rc_end;
    for (int k = 0; k < n; ++k) CKS(check_waits(hs[k]));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    long long ns = 0, nl = 0;
    for (int k = 0; k < n; ++k) {
        ns += hs[k]->n_sync;
        nl += hs[k]->n_vl;
    }
    for (int k = 0; k < n; ++k) {
        info[k].seconds = secs;
        info[k].host_syncs = (int)ns;
        info[k].vector_launches = (int)nl;
    }
    for (int k = 0; k < n; ++k)
        if (info[k].status != ST_OK)
            return fail(info[k].status, "member %d: no convergence: rel. residual %.3e after %d iterations",
                        k, info[k].rel_residual, info[k].iterations);
    return ST_OK;
}

int st_solve_host(st_handle h, int nbatch, const double *rhs, double tol, double *u,
                  int use_guess, st_solve_info *info) {
    NvtxRange range("st_solve_host");
    CKS(check_ptr(h, rhs, "rhs"));
    CKS(check_ptr(h, u, "u"));
    if (nbatch < 1) return fail(ST_ERR_INVALID_ARG, "nbatch must be >= 1");
    if ((const void *)rhs == (void *)u) return fail(ST_ERR_INVALID_ARG, "rhs and u alias");
    if (!(tol > 0)) return fail(ST_ERR_INVALID_ARG, "tol must be > 0");
    for (const void *p : {(const void *)rhs, (const void *)u}) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
        } else if (a.type == cudaMemoryTypeDevice) {
            return fail(ST_ERR_INVALID_ARG, "st_solve_host takes host buffers (use st_solve)");
        }
    }
    const size_t e = (size_t)h->len * h->nrhs;  // doubles per batch
    if (!h->hs_f[0]) {
        void *p;
        for (int s = 0; s < 2; ++s) {
            CKS(dalloc(h, e * sizeof(double), &p));
            h->hs_f[s] = (double *)p;
            CKS(dalloc(h, e * sizeof(double), &p));
            h->hs_u[s] = (double *)p;
        }
    }
    if (!h->cp_in) {
        // non-blocking: no implicit ordering with a legacy-default compute stream
        CK(cudaStreamCreateWithFlags(&h->cp_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->cp_out, cudaStreamNonBlocking));
        for (int s = 0; s < 2; ++s) {
            CK(cudaEventCreateWithFlags(&h->hs_in[s], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->hs_solved[s], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->hs_out[s], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&h->bg_ev, cudaEventDisableTiming));
    }
    st_solve_info local;
    if (!info) info = &local;
    std::memset(info, 0, sizeof *info);
    const auto t0 = std::chrono::steady_clock::now();
    h->bg.clear();
    h->bg_err = cudaSuccess;
    // the pending copy of slot s (two batches back) issued in full
    auto flush_slot = [&](int s) {
        if (h->bg.empty() || h->bg.front().slot != s) return;
        auto &c = h->bg.front();
        cudaError_t e = cudaMemcpyAsync(c.dst + c.done, c.src + c.done,
                                        (c.n - c.done) * sizeof(double), cudaMemcpyDeviceToHost,
                                        h->cp_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->bg_ev, h->cp_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->hs_out[s], h->cp_out);
        if (e != cudaSuccess && h->bg_err == cudaSuccess) h->bg_err = e;
        h->bg.pop_front();
    };
    // batch k uses slot k & 1; a slot is refilled only after the solve two
    // batches back has finished with it and its solution has been copied out
    auto copy_in = [&](int k) -> cudaError_t {
        const int s = k & 1;
        if (use_guess) flush_slot(s);
        cudaError_t c = cudaStreamWaitEvent(h->cp_in, h->hs_solved[s], 0);
        if (c == cudaSuccess && use_guess) c = cudaStreamWaitEvent(h->cp_in, h->hs_out[s], 0);
        if (c == cudaSuccess)
            c = cudaMemcpyAsync(h->hs_f[s], rhs + (size_t)k * e, e * sizeof(double),
                                cudaMemcpyHostToDevice, h->cp_in);
        if (c == cudaSuccess && use_guess)
            c = cudaMemcpyAsync(h->hs_u[s], u + (size_t)k * e, e * sizeof(double),
                                cudaMemcpyHostToDevice, h->cp_in);
        if (c == cudaSuccess) c = cudaEventRecord(h->hs_in[s], h->cp_in);
        return c;
    };
    // every solution of the batches solved so far issued, and no copy left in
    // flight on the staging slots, whatever happened
    auto drain = [&](int rc) {
        bg_pump(h, true);
        cudaStreamSynchronize(h->cp_in);
        cudaStreamSynchronize(h->cp_out);
        cudaStreamSynchronize(h->stream);
        h->bg.clear();
        return rc;
    };
    cudaError_t c = copy_in(0);
    for (int k = 0; k < nbatch && c == cudaSuccess; ++k) {
        const int s = k & 1;
        if (k + 1 < nbatch) c = copy_in(k + 1);  // overlaps this batch's solve
        flush_slot(s);
        if (c == cudaSuccess) c = cudaStreamWaitEvent(h->stream, h->hs_in[s], 0);
        if (c == cudaSuccess) c = cudaStreamWaitEvent(h->stream, h->hs_out[s], 0);
        if (c != cudaSuccess) break;
        st_solve_info bi;
        // batch k - 1's solution is copied back in chunks during this solve
        const int rc = st_solve(h, h->hs_f[s], tol, h->hs_u[s], use_guess, &bi);
        info->iterations = std::max(info->iterations, bi.iterations);
        info->refinements = std::max(info->refinements, bi.refinements);
        info->rel_residual = std::max(info->rel_residual, bi.rel_residual);
        info->host_syncs += bi.host_syncs;
        info->vector_launches += bi.vector_launches;
        if (rc != ST_OK) {
            info->status = rc;
            return drain(rc);
        }
        c = cudaEventRecord(h->hs_solved[s], h->stream);
        if (c == cudaSuccess) c = cudaStreamWaitEvent(h->cp_out, h->hs_solved[s], 0);
        if (c == cudaSuccess) {
            h->bg.push_back({u + (size_t)k * e, h->hs_u[s], e, 0, s});
            bg_pump(h);
        }
    }
    if (c == cudaSuccess) {
        bg_pump(h, true);
        c = h->bg_err;
    }
    if (c == cudaSuccess) c = cudaStreamSynchronize(h->cp_out);
    if (c != cudaSuccess) {
        cudaGetLastError();
        return drain(fail(ST_ERR_CUDA, "st_solve_host: %s", cudaGetErrorString(c)));
    }
    CK(cudaStreamSynchronize(h->cp_in));
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return ST_OK;
}

int st_profile(st_handle h, int enable) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (h->host_only) return fail(ST_ERR_INVALID_ARG, "handle was built host-only");
    CK(cudaStreamSynchronize(h->stream));
    prof_fold(h);
    if (enable) {
        for (int c = 0; c < ST_PROF_NCLASS; ++c) {
            h->prof_n[c] = 0;
            h->prof_ms[c] = h->prof_bytes[c] = h->prof_flops[c] = 0.0;
        }
    }
    h->prof_on = enable != 0;
    return ST_OK;
}

int st_profile_read(st_handle h, int cls, int64_t *launches, double *ms, double *bytes,
                    double *flops) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (cls < 0 || cls >= ST_PROF_NCLASS) return fail(ST_ERR_INVALID_ARG, "bad kernel class");
    if (!h->host_only) {
        CK(cudaStreamSynchronize(h->stream));
        prof_fold(h);
    }
    if (launches) *launches = h->prof_n[cls];
    if (ms) *ms = h->prof_ms[cls];
    if (bytes) *bytes = h->prof_bytes[cls];
    if (flops) *flops = h->prof_flops[cls];
    return ST_OK;
}

int st_smooth_static(st_handle h, double *u, const double *f, int nsteps, void *stream) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (!u || !f) return fail(ST_ERR_INVALID_ARG, "null vector pointer");
    if ((const void *)u == (const void *)f) return fail(ST_ERR_INVALID_ARG, "u and f alias");
    if (nsteps < 0) return fail(ST_ERR_INVALID_ARG, "nsteps < 0");
    // only the real Schur form with exact spatial solves keeps everything it
    // needs in the static array (the other variants need the per-mode shift
    // table or the MinRes work space); refuse them before any upload or launch
    if (h->opt.variant != ST_RSCHUR)
        return fail(ST_ERR_UNSUPPORTED, "st_smooth_static supports only the real Schur variant");
    if (h->opt.spatial_solver != ST_SPATIAL_FD)
        return fail(ST_ERR_UNSUPPORTED, "st_smooth_static supports only exact spatial solves");
    const long long total = h->len * h->nrhs;
    if (total > ST_STATIC_MAX_DOFS)
        return fail(ST_ERR_INVALID_ARG, "%lld dofs exceed the static work space of %d dofs", total,
                    (int)ST_STATIC_MAX_DOFS);
    for (int a = 0; a < h->dim; ++a)
        if (h->n[a] > ST_STATIC_MAX_N)
            return fail(ST_ERR_INVALID_ARG, "%d dofs on axis %d exceed the static limit %d", h->n[a],
                        a, (int)ST_STATIC_MAX_N);
    double *base = nullptr;
    CKS(static_scratch_addr(&base));
    try {
        // a view of the handle's host factors that runs on the static memory
        st_handle_s v;
        v.dim = h->dim; v.p = h->p; v.N = h->N; v.nt = h->nt; v.nrhs = h->nrhs; v.nlev = h->nlev;
        for (int a = 0; a < 3; ++a) { v.spans[a] = h->spans[a]; v.n[a] = h->n[a]; }
        v.opt = h->opt;
        v.g = h->g;
        v.len = h->len;
        v.lv = h->lv;
        v.stream = (cudaStream_t)stream;
        v.w64.w0 = base;
        v.w64.w1 = base + ST_STATIC_MAX_DOFS;
        const cudaStream_t s = v.stream;
        const int W = 2 * h->p + 1;
        for (int a = 0; a < h->dim; ++a) {
            const int n = h->n[a];
            double *fa = base + 2 * (size_t)ST_STATIC_MAX_DOFS + a * kStaticFactorPerAxis;
            double *bm = fa, *bk = bm + (size_t)ST_STATIC_MAX_N * W;
            double *U = bk + (size_t)ST_STATIC_MAX_N * W, *Ut = U + (size_t)ST_STATIC_MAX_N * ST_STATIC_MAX_N;
            double *lam = Ut + (size_t)ST_STATIC_MAX_N * ST_STATIC_MAX_N;
            std::vector<double> hbm((size_t)n * W, 0.0), hbk((size_t)n * W, 0.0), hut((size_t)n * n);
            for (int i = 0; i < n; ++i)
                for (int o = -h->p; o <= h->p; ++o) {
                    const int j = i + o;
                    if (j < 0 || j >= n) continue;
                    hbm[(size_t)i * W + o + h->p] = h->M1[a][(size_t)i * n + j];
                    hbk[(size_t)i * W + o + h->p] = h->K1[a][(size_t)i * n + j];
                }
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < n; ++k) hut[(size_t)k * n + i] = h->U[a][(size_t)i * n + k];
            // pageable sources: each copy has consumed its host buffer on return
            CK(cudaMemcpyAsync(bm, hbm.data(), hbm.size() * 8, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(bk, hbk.data(), hbk.size() * 8, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(U, h->U[a].data(), (size_t)n * n * 8, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(Ut, hut.data(), hut.size() * 8, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(lam, h->lam[a].data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
            v.s64.bands.M[a] = bm;
            v.s64.bands.K[a] = bk;
            v.s64.U[a] = U;
            v.s64.Ut[a] = Ut;
            v.s64.lam[a] = lam;
        }
        // nothing in the static work space has to start at zero: every step
        // writes both work vectors before it reads them
        for (int k = 0; k < nsteps; ++k) CKS(smooth<double>(&v, 0, u, f, v.opt.omega));
    } catch (...) {
        return fail(ST_ERR_OOM, "host exception in st_smooth_static");
    }
    return ST_OK;
}

int st_time_factors(st_handle h, int lvl, int *nt, double *Kt, double *Mt, double *X, double *Z,
                    double *Y) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (lvl < 0 || lvl >= h->nlev) return fail(ST_ERR_INVALID_ARG, "level out of range");
    const LevelHost &L = h->lv[lvl];
    const size_t b = sizeof(double) * h->nt * h->nt;
    if (nt) *nt = h->nt;
    if (Kt) std::memcpy(Kt, L.Kt.data(), b);
    if (Mt) std::memcpy(Mt, L.Mt.data(), b);
    if (X) std::memcpy(X, L.X.data(), b);
    if (Z) std::memcpy(Z, L.Z.data(), b);
    if (Y) std::memcpy(Y, L.Y.data(), b);
    return ST_OK;
}

int st_space_factors(st_handle h, int axis, int *n, double *M1, double *K1, double *U, double *lam) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (axis < 0 || axis >= h->dim) return fail(ST_ERR_INVALID_ARG, "axis out of range");
    const int nn = h->n[axis];
    const size_t b = sizeof(double) * nn * nn;
    if (n) *n = nn;
    if (M1) std::memcpy(M1, h->M1[axis].data(), b);
    if (K1) std::memcpy(K1, h->K1[axis].data(), b);
    if (U) std::memcpy(U, h->U[axis].data(), b);
    if (lam) std::memcpy(lam, h->lam[axis].data(), sizeof(double) * nn);
    return ST_OK;
}

int st_autotune(st_handle h, int *choice, double *ms) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (h->host_only) return fail(ST_ERR_INVALID_ARG, "handle was built host-only");
    CKS(autotune(h));
    for (int a = 0; a < 3; ++a) {
        if (choice) choice[a] = a < h->dim ? h->tune[a] : -1;
        if (ms) ms[a] = a < h->dim ? h->tune_ms[a] : 0.0;
    }
    return ST_OK;
}

int st_time_spectrum(st_handle h, int lvl, double *lam_re, double *lam_im, double *cond_x) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (lvl < 0 || lvl >= h->nlev) return fail(ST_ERR_INVALID_ARG, "level out of range");
    const LevelHost &L = h->lv[lvl];
    if (!L.eig_ok) return fail(ST_ERR_ILL_CONDITIONED, "no eigen-decomposition on this level");
    if (lam_re) std::memcpy(lam_re, L.lre.data(), sizeof(double) * h->nt);
    if (lam_im) std::memcpy(lam_im, L.lim.data(), sizeof(double) * h->nt);
    if (cond_x) *cond_x = L.condX;
    return ST_OK;
}

int st_time_prolongation(st_handle h, int *nt, double *Pt) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (nt) *nt = h->nt;
    if (Pt) std::memcpy(Pt, h->Pt.data(), sizeof(double) * 2 * h->nt * h->nt);
    return ST_OK;
}

int st_space_prolongation(st_handle h, int lvl, int axis, int *nf, int *nc, double *P) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (lvl < 0 || lvl + 1 >= h->nlev || !h->lv[lvl + 1].xstep)
        return fail(ST_ERR_INVALID_ARG, "level %d is not followed by a space step", lvl);
    if (axis < 0 || axis >= h->dim) return fail(ST_ERR_INVALID_ARG, "bad axis %d", axis);
    const LevelSpace &F = h->ls[h->lv[lvl].sp], &C = h->ls[h->lv[lvl + 1].sp];
    if (nf) *nf = F.n[axis];
    if (nc) *nc = C.n[axis];
    if (P) std::memcpy(P, F.Pc[axis].data(), sizeof(double) * F.Pc[axis].size());
    return ST_OK;
}

int st_level_shape(st_handle h, int lvl, int *slabs, int *spans, int *space_step) {
    if (!h) return fail(ST_ERR_INVALID_ARG, "null handle");
    if (lvl < 0 || lvl >= h->nlev) return fail(ST_ERR_INVALID_ARG, "level %d out of range", lvl);
    const LevelHost &L = h->lv[lvl];
    if (slabs) *slabs = L.nslab;
    if (spans)
        for (int a = 0; a < 3; ++a) spans[a] = h->ls[L.sp].spans[a];
    if (space_step) *space_step = L.xstep ? 1 : 0;
    return ST_OK;
}

}  // extern "C"

int st::setup_pooled(st_handle_s **out, int geometry, int degree, const int *spans, int slabs,
                     const st_options *opt, cudaStream_t stream, cudaMemPool_t pool) {
    return setup_entry(out, geometry, degree, spans, slabs, opt, stream, false, pool);
}

// Vector kernels of the FP64 outer iteration (FGMRES, Sec. 3.1 outer solver
// of arXiv:1802.09277) and precision conversion for the mixed V-cycle.
// Reductions are deterministic: fixed-size per-block partial sums, then one
// fixed-order pass.
#include "pdl.cuh"
#include "st_internal.h"

namespace st {

constexpr int NRHS_MAX = 32;

// Device view of a group launch (see GLaunch): per member its length, rhs
// count, wide-load flag and partial-sum buffer; per system its member and
// rhs index and (multi-axpy) its vector count.
struct GMemD {
    long long len[GH];
    int R[GH];
    int vec[GH];
    double *part[GH];
};
struct GSysD {
    int m[NSYS_MAX], r[NSYS_MAX], nv[NSYS_MAX];
};
// vector v of member k
template <typename T>
struct GVecD {
    const T *v[MAXV][GH];
};
// one target vector per member
template <typename T>
struct GTgtD {
    T *p[GH];
};
template <typename T>
struct GAxpyD {
    T coef[MAXV * NSYS_MAX];  // rounded to T on the host
    T post[NSYS_MAX];         // y <- post_s * (y + sum_v coef x_v)
};
// two outputs sharing the vectors x_v (the delayed Gram-Schmidt step):
//   y1 <- post1_s * (y1 + sum_v c1 x_v)
//   y2 <- post2_s * (y2 + c21_s * y1_old + sum_v c2 x_v)
template <typename T>
struct GAxpy2D {
    T c1[MAXV * NSYS_MAX];
    T c2[MAXV * NSYS_MAX];
    T c21[NSYS_MAX];
    T post1[NSYS_MAX], post2[NSYS_MAX];
    int write1[NSYS_MAX];  // 0: y1 of system s is left untouched
};

static GMemD mem_of(const GLaunch &g) {
    GMemD m{};
    for (int k = 0; k < g.nmem; ++k) {
        m.len[k] = g.len[k];
        m.R[k] = g.R[k];
        m.part[k] = g.part[k];
    }
    return m;
}
static GSysD sys_of(const GLaunch &g) {
    GSysD s{};
    for (int i = 0; i < g.nsys; ++i) {
        s.m[i] = g.sm[i];
        s.r[i] = g.sr[i];
        s.nv[i] = g.snv[i];
    }
    return s;
}
static bool group_ok(const GLaunch &g, int nv) {
    if (g.nmem < 1 || g.nmem > GH || g.nsys < 1 || g.nsys > NSYS_MAX || nv < 0 || nv > MAXV)
        return false;
    for (int i = 0; i < g.nsys; ++i)
        if (g.sm[i] < 0 || g.sm[i] >= g.nmem || g.sr[i] < 0 || g.sr[i] >= g.R[g.sm[i]])
            return false;
    return true;
}

// two consecutive elements as one 8- (float) or 16-byte (double) access
template <typename T>
struct Pair;
template <>
struct Pair<double> {
    using V = double2;
};
template <>
struct Pair<float> {
    using V = float2;
};

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin *__restrict__ x, Tout *__restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (Tout)x[i];
}

template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin *x, Tout *y, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_convert<Tin, Tout><<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_zero(T *x, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = T(0);
}

template <typename T>
cudaError_t launch_zero(T *x, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_zero<T><<<(unsigned)blocks, 256, 0, s>>>(x, n);
    return cudaGetLastError();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-thread accumulator of a dot product: FP64 for FP64 vectors; for FP32
// vectors an FP32 sum with Kahan compensation (GB300's FP64 pipe is ~60x
// slower than its FP32 pipe, so FP64 products would make the kernel
// ALU-bound); partial sums are combined in FP64.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add1(double p) { s += p; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float y = fmaf(a, b, -c);
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ void add1(float p) {  // add p (Kahan)
        const float y = p - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Reduction of the per-thread accumulators across a warp and the CTA.  For
// FP32 data the Kahan pairs (s, -c) are summed as double-float numbers (FP32
// operations only): an FP64 shuffle tree per accumulator costs more than the
// whole streaming loop on GB300's FP64 pipe.
template <typename T>
struct Red;
template <>
struct Red<double> {
    using V = double;
    static __device__ __forceinline__ V of(const DotAcc<double> &a) { return a.value(); }
    static __device__ __forceinline__ V zero() { return 0.0; }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V warp(V v) { return warp_sum(v); }
    static __device__ __forceinline__ double out(V v) { return v; }
};
template <>
struct Red<float> {
    using V = dfloat;
    static __device__ __forceinline__ V of(const DotAcc<float> &a) { return dfloat(a.s, -a.c); }
    static __device__ __forceinline__ V zero() { return dfloat(0.f, 0.f); }
    static __device__ __forceinline__ V add(V a, V b) { return df_add(a, b); }
    static __device__ __forceinline__ V warp(V v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = df_add(v, dfloat(__shfl_xor_sync(0xffffffffu, v.hi, o),
                                 __shfl_xor_sync(0xffffffffu, v.lo, o)));
        return v;
    }
    static __device__ __forceinline__ double out(V v) { return (double)v; }
};

// One thread's share of the dots of CNT vectors with the target w (SELF: of
// each vector with itself, w unused), elements in grid-stride order.  The
// count is a compile-time constant and the loop takes two strides at a time,
// so every load of both is issued before the products that use them: with
// the count a run-time value (predicated loads) the loads of the next stride
// waited for the arithmetic of this one, and the FP64 dots ran at a sixth of
// HBM bandwidth.  Each accumulator sees its elements in the order of the
// plain grid-stride loop.
template <typename T, int CNT, bool SELF>
__device__ __forceinline__ void gdot_body(const T *const *x, const T *__restrict__ w,
                                          long long len, int vec2, DotAcc<T> *acc) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec2) {
        using P2 = typename Pair<T>::V;
        const long long np = len / 2;
        const P2 *w2 = reinterpret_cast<const P2 *>(w);
        long long i = i0;
        for (; i + stride < np; i += 2 * stride) {
            P2 a[2][CNT], b[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (!SELF) b[u] = w2[i + u * stride];
#pragma unroll
                for (int k = 0; k < CNT; ++k)
                    a[u][k] = reinterpret_cast<const P2 *>(x[k])[i + u * stride];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int k = 0; k < CNT; ++k) {
                    const P2 c = SELF ? a[u][k] : b[u];
                    acc[k].add(a[u][k].x, c.x);
                    acc[k].add(a[u][k].y, c.y);
                }
        }
        if (i < np) {
            P2 a[CNT], b;
            if (!SELF) b = w2[i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) a[k] = reinterpret_cast<const P2 *>(x[k])[i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) {
                const P2 c = SELF ? a[k] : b;
                acc[k].add(a[k].x, c.x);
                acc[k].add(a[k].y, c.y);
            }
        }
    } else {
        long long i = i0;
        for (; i + stride < len; i += 2 * stride) {
            T a[2][CNT], b[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (!SELF) b[u] = w[i + u * stride];
#pragma unroll
                for (int k = 0; k < CNT; ++k) a[u][k] = x[k][i + u * stride];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int k = 0; k < CNT; ++k) acc[k].add(a[u][k], SELF ? a[u][k] : b[u]);
        }
        if (i < len) {
            T a[CNT], b = T(0);
            if (!SELF) b = w[i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) a[k] = x[k][i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) acc[k].add(a[k], SELF ? a[k] : b);
        }
    }
}

// grid (nblk, nsys, ceil(nv / GV)), 256 threads; member k's partial sums at
// part[k][(v * R[k] + r) * nblk + blk].  Block (b, s, g) accumulates the dots
// of vectors GV g .. GV g + GV - 1 of system s with its target (SELF: with
// themselves) over a grid-stride loop, two elements per load when the member
// allows it.  The target is re-read by every group from L2.
template <typename T, int GV, bool SELF>
__global__ void __launch_bounds__(256)
    k_gdot_partial(int nv, const __grid_constant__ GVecD<T> vl, const __grid_constant__ GTgtD<T> tw,
                   const __grid_constant__ GMemD gm, const __grid_constant__ GSysD gs) {
    griddep_wait();
    griddep_launch();
    __shared__ typename Red<T>::V red[8][GV];
    const int s = blockIdx.y, nblk = gridDim.x;
    const int mk = gs.m[s], r = gs.r[s];
    const long long len = gm.len[mk];
    const long long off = (long long)r * len;
    const int vec2 = gm.vec[mk];
    const T *w = SELF ? nullptr : tw.p[mk] + off;
    const int v0 = GV * blockIdx.z;
    const int cnt = (nv - v0 < GV) ? nv - v0 : GV;
    const T *x[GV];
#pragma unroll
    for (int k = 0; k < GV; ++k) x[k] = vl.v[(k < cnt) ? v0 + k : v0][mk] + off;
    DotAcc<T> acc[GV];
    static_assert(GV == 2 || GV == 4, "the count dispatch below covers GV = 2 and 4");
    switch (cnt) {  // uniform across the grid row
        case 1: gdot_body<T, 1, SELF>(x, w, len, vec2, acc); break;
        case 2: gdot_body<T, 2, SELF>(x, w, len, vec2, acc); break;
        case 3: gdot_body<T, (GV > 2 ? 3 : 2), SELF>(x, w, len, vec2, acc); break;
        default: gdot_body<T, GV, SELF>(x, w, len, vec2, acc); break;
    }
    using RD = Red<T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < GV; ++k) {
        if (k >= cnt) break;
        const typename RD::V t = RD::warp(RD::of(acc[k]));
        if (lane == 0) red[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        typename RD::V t = RD::zero();
        for (int q = 0; q < 8; ++q) t = RD::add(t, red[q][threadIdx.x]);
        gm.part[mk][((long long)(v0 + threadIdx.x) * gm.R[mk] + r) * nblk + blockIdx.x] = RD::out(t);
    }
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// one warp per output out[row * nsys + s]: lane-strided partial sums of that
// row and system, then a fixed shuffle tree
__global__ void k_greduce(const __grid_constant__ GMemD gm, const __grid_constant__ GSysD gs,
                          int nsys, int count, int nblk, double *__restrict__ out) {
    griddep_wait();
    griddep_launch();
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= count) return;
    const int row = i / nsys, s = i % nsys;
    const int mk = gs.m[s];
    const double *p = gm.part[mk] + ((long long)row * gm.R[mk] + gs.r[s]) * nblk;
    double t = 0.0;
    for (int b = lane; b < nblk; b += 32) t += p[b];
    t = warp_sum(t);
    if (lane == 0) out[i] = t;
}

template <typename T>
static bool al2(const void *p) {
    return sizeof(T) == 8 ? aligned16(p) : ((reinterpret_cast<uintptr_t>(p) & 7u) == 0);
}

// shared by launch_gdot and launch_gnorm2 (self = 1: w unused)
template <typename T>
static cudaError_t gdot_run(const GLaunch &g, int nv, const T *const *xs, const T *const *w,
                            bool self, double *out, cudaStream_t s) {
    if (!group_ok(g, nv) || nv < 1) return cudaErrorInvalidValue;
    GVecD<T> vl{};
    GTgtD<T> tw{};
    GMemD gm = mem_of(g);
    for (int k = 0; k < g.nmem; ++k) {
        tw.p[k] = self ? nullptr : const_cast<T *>(w[k]);
        int vec2 = (g.len[k] % 2 == 0) && (self || al2<T>(w[k]));
        for (int v = 0; v < nv; ++v) {
            vl.v[v][k] = xs[(size_t)v * g.nmem + k];
            vec2 = vec2 && al2<T>(vl.v[v][k]);
        }
        gm.vec[k] = vec2;
    }
    const GSysD gs = sys_of(g);
    cudaError_t e;
    if (self)  // norms come one or two at a time: the two-vector kernel keeps its registers low
        e = launch_pdl(k_gdot_partial<T, 2, true>, dim3(g.nblk, g.nsys, (nv + 1) / 2), dim3(256),
                       0, s, nv, vl, tw, gm, gs);
    else
        e = launch_pdl(k_gdot_partial<T, 4, false>, dim3(g.nblk, g.nsys, (nv + 3) / 4), dim3(256),
                       0, s, nv, vl, tw, gm, gs);
    if (e != cudaSuccess) return e;
    const int count = nv * g.nsys;
    e = launch_pdl(k_greduce, dim3((count + 3) / 4), dim3(128), 0, s, gm, gs, g.nsys, count,
                   g.nblk, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_gdot(const GLaunch &g, int nv, const T *const *xs, const T *const *w,
                        double *out, cudaStream_t s) {
    bool self = nv == 1;  // a vector with itself: one load per element
    for (int k = 0; self && k < g.nmem; ++k) self = xs[k] == w[k];
    return gdot_run<T>(g, nv, xs, w, self, out, s);
}

template <typename T>
cudaError_t launch_gnorm2(const GLaunch &g, int nv, const T *const *xs, double *out,
                          cudaStream_t s) {
    return gdot_run<T>(g, nv, xs, nullptr, true, out, s);
}

// grid (blocks, nsys): block row s updates system s (its member's vector at
// offset r * len) with the first nv[s] vectors
template <typename T>
__global__ void __launch_bounds__(256)
    k_gaxpy(const __grid_constant__ GVecD<T> vl, const __grid_constant__ GTgtD<T> ty,
            const __grid_constant__ GAxpyD<T> aa, const __grid_constant__ GMemD gm,
            const __grid_constant__ GSysD gs, int yz) {
    griddep_wait();
    griddep_launch();
    using P2 = typename Pair<T>::V;
    const int s = blockIdx.y;
    const int mk = gs.m[s], nv = gs.nv[s];
    const long long len = gm.len[mk];
    const long long off = (long long)gs.r[s] * len;
    T *__restrict__ y = ty.p[mk];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const T post = aa.post[s];
    if (gm.vec[mk]) {  // off is even because len is
        const long long n = len / 2;
        P2 *y2 = reinterpret_cast<P2 *>(y + off);
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            P2 acc;
            if (yz) {  // -0 + p = p for every p, signed zeros included
                acc.x = -T(0);
                acc.y = -T(0);
            } else {
                acc = y2[i];
            }
            for (int v = 0; v < nv; ++v) {
                const T c = aa.coef[v * NSYS_MAX + s];
                const P2 x = reinterpret_cast<const P2 *>(vl.v[v][mk] + off)[i];
                acc.x += c * x.x;
                acc.y += c * x.y;
            }
            acc.x *= post;
            acc.y *= post;
            y2[i] = acc;
        }
        return;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        T acc = yz ? -T(0) : y[off + i];
        for (int v = 0; v < nv; ++v) acc += aa.coef[v * NSYS_MAX + s] * vl.v[v][mk][off + i];
        y[off + i] = post * acc;
    }
}

// Two-output update of system s, CNT vectors fixed at compile time (CNT < 0:
// the run-time count nv).  With a fixed count the coefficients sit in
// registers and every load of an element pair (y1, y2, the vectors) is
// issued before its arithmetic; each output sees the same operations in the
// same order in every instance.
template <typename T, int CNT>
__global__ void __launch_bounds__(256)
    k_gaxpy2(int nv, const __grid_constant__ GVecD<T> vl, const __grid_constant__ GTgtD<T> t1,
             const __grid_constant__ GTgtD<T> t2, const __grid_constant__ GAxpy2D<T> aa,
             const __grid_constant__ GMemD gm, const __grid_constant__ GSysD gs) {
    griddep_wait();
    griddep_launch();
    const int s = blockIdx.y;
    const int mk = gs.m[s];
    const long long len = gm.len[mk];
    const long long off = (long long)gs.r[s] * len;
    T *__restrict__ y1 = t1.p[mk];
    T *__restrict__ y2 = t2.p[mk];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const T p1 = aa.post1[s], p2 = aa.post2[s], c21 = aa.c21[s];
    const int write1 = aa.write1[s];
    if constexpr (CNT < 0) {
        for (long long i = i0; i < len; i += stride) {
            const T a1o = y1[off + i];
            T a1 = a1o, a2 = y2[off + i] + c21 * a1o;
            for (int v = 0; v < nv; ++v) {
                const T x = vl.v[v][mk][off + i];
                a1 += aa.c1[v * NSYS_MAX + s] * x;
                a2 += aa.c2[v * NSYS_MAX + s] * x;
            }
            if (write1) y1[off + i] = p1 * a1;
            y2[off + i] = p2 * a2;
        }
    } else {
        constexpr int NV = CNT > 0 ? CNT : 1;
        T k1[NV], k2[NV];
        const T *x[NV];
#pragma unroll
        for (int v = 0; v < CNT; ++v) {
            k1[v] = aa.c1[v * NSYS_MAX + s];
            k2[v] = aa.c2[v * NSYS_MAX + s];
            x[v] = vl.v[v][mk] + off;
        }
        if (gm.vec[mk]) {  // off is even because len is
            using P2 = typename Pair<T>::V;
            const long long np = len / 2;
            P2 *q1 = reinterpret_cast<P2 *>(y1 + off);
            P2 *q2 = reinterpret_cast<P2 *>(y2 + off);
            for (long long i = i0; i < np; i += stride) {
                const P2 u1 = q1[i], u2 = q2[i];
                P2 xv[NV];
#pragma unroll
                for (int v = 0; v < CNT; ++v) xv[v] = reinterpret_cast<const P2 *>(x[v])[i];
                T a1x = u1.x, a1y = u1.y, a2x = u2.x + c21 * u1.x, a2y = u2.y + c21 * u1.y;
#pragma unroll
                for (int v = 0; v < CNT; ++v) {
                    a1x += k1[v] * xv[v].x;
                    a2x += k2[v] * xv[v].x;
                    a1y += k1[v] * xv[v].y;
                    a2y += k2[v] * xv[v].y;
                }
                if (write1) {
                    P2 o1;
                    o1.x = p1 * a1x;
                    o1.y = p1 * a1y;
                    q1[i] = o1;
                }
                P2 o2;
                o2.x = p2 * a2x;
                o2.y = p2 * a2y;
                q2[i] = o2;
            }
        } else {
            for (long long i = i0; i < len; i += stride) {
                const T a1o = y1[off + i], b2 = y2[off + i];
                T xv[NV];
#pragma unroll
                for (int v = 0; v < CNT; ++v) xv[v] = x[v][i];
                T a1 = a1o, a2 = b2 + c21 * a1o;
#pragma unroll
                for (int v = 0; v < CNT; ++v) {
                    a1 += k1[v] * xv[v];
                    a2 += k2[v] * xv[v];
                }
                if (write1) y1[off + i] = p1 * a1;
                y2[off + i] = p2 * a2;
            }
        }
    }
}

template <typename T>
struct Quad;
template <>
struct Quad<float> {
    using V = float4;
};
template <>
struct Quad<double> {
    using V = double4_32a;
};

// one CTA's share of the Gram products for CNT vectors (compile-time count:
// every load of an iteration is issued before the arithmetic that uses it)
template <typename T, int CNT>
__device__ __forceinline__ void gram2_body(const T *const *x, const T *__restrict__ t1,
                                           const T *__restrict__ t2, long long len, int vec4,
                                           DotAcc<T> *a1, DotAcc<T> *a2) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec4) {
        using Q = typename Quad<T>::V;
        const long long nq = len / 4;
        const Q *q1 = reinterpret_cast<const Q *>(t1);
        const Q *q2 = reinterpret_cast<const Q *>(t2);
#pragma unroll 2
        for (long long i = i0; i < nq; i += stride) {
            Q xv[CNT];
            const Q u1 = q1[i], u2 = q2[i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) xv[k] = reinterpret_cast<const Q *>(x[k])[i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) {
                a1[k].add1(xv[k].x * u1.x + xv[k].y * u1.y + xv[k].z * u1.z + xv[k].w * u1.w);
                a2[k].add1(xv[k].x * u2.x + xv[k].y * u2.y + xv[k].z * u2.z + xv[k].w * u2.w);
            }
        }
    } else {
        for (long long i = i0; i < len; i += stride) {
            T xv[CNT];
            const T u1 = t1[i], u2 = t2[i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) xv[k] = x[k][i];
#pragma unroll
            for (int k = 0; k < CNT; ++k) {
                a1[k].add(xv[k], u1);
                a2[k].add(xv[k], u2);
            }
        }
    }
}

// grid (nblk, nsys, ceil(nv / GV)): the dots of vectors GV g .. GV g + GV - 1
// with two targets t1, t2 in one pass; member k's partial sums at
// part[k][((v * 2 + t) * R[k] + r) * nblk + blk].  vec4: 16-byte loads (len a
// multiple of 4, 16-byte aligned vectors); each thread forms the 4-term
// products of a chunk in T and adds them into its accumulator
// (Kahan-compensated in FP32), so the compensation runs once per 4 elements.
template <typename T, int GV>
__global__ void __launch_bounds__(256)
    k_ggram2_partial(int nv, const __grid_constant__ GVecD<T> vl,
                     const __grid_constant__ GTgtD<T> tt1, const __grid_constant__ GTgtD<T> tt2,
                     const __grid_constant__ GMemD gm, const __grid_constant__ GSysD gs) {
    griddep_wait();
    griddep_launch();
    __shared__ typename Red<T>::V red[8][2 * GV];
    const int s = blockIdx.y, nblk = gridDim.x;
    const int mk = gs.m[s], r = gs.r[s];
    const long long len = gm.len[mk];
    const long long off = (long long)r * len;
    const int vec4 = gm.vec[mk];
    const T *t1 = tt1.p[mk] + off, *t2 = tt2.p[mk] + off;
    const int v0 = GV * blockIdx.z;
    const int cnt = (nv - v0 < GV) ? nv - v0 : GV;
    const T *x[GV];
#pragma unroll
    for (int k = 0; k < GV; ++k) x[k] = vl.v[(k < cnt) ? v0 + k : v0][mk] + off;
    DotAcc<T> a1[GV], a2[GV];
    static_assert(GV == 4, "the count dispatch below covers GV = 4");
    switch (cnt) {  // uniform across the grid row
        case 1: gram2_body<T, 1>(x, t1, t2, len, vec4, a1, a2); break;
        case 2: gram2_body<T, 2>(x, t1, t2, len, vec4, a1, a2); break;
        case 3: gram2_body<T, 3>(x, t1, t2, len, vec4, a1, a2); break;
        default: gram2_body<T, 4>(x, t1, t2, len, vec4, a1, a2); break;
    }
    using RD = Red<T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < GV; ++k) {
        if (k >= cnt) break;
        const typename RD::V s1 = RD::warp(RD::of(a1[k])), s2 = RD::warp(RD::of(a2[k]));
        if (lane == 0) {
            red[warp][2 * k] = s1;
            red[warp][2 * k + 1] = s2;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * cnt) {
        typename RD::V t = RD::zero();
        for (int q = 0; q < 8; ++q) t = RD::add(t, red[q][threadIdx.x]);
        const int v = v0 + threadIdx.x / 2, which = threadIdx.x % 2;
        gm.part[mk][((long long)(2 * v + which) * gm.R[mk] + r) * nblk + blockIdx.x] = RD::out(t);
    }
}

template <typename T>
cudaError_t launch_ggram2(const GLaunch &g, int nv, const T *const *xs, const T *const *t1,
                          const T *const *t2, double *out, cudaStream_t s) {
    if (!group_ok(g, nv) || nv < 1) return cudaErrorInvalidValue;
    GVecD<T> vl{};
    GTgtD<T> a{}, b{};
    GMemD gm = mem_of(g);
    // 4-element loads need the vectors aligned to 4 elements (16 or 32 bytes)
    const uintptr_t am = 4 * sizeof(T) - 1;
    auto al4 = [am](const void *p) { return (reinterpret_cast<uintptr_t>(p) & am) == 0; };
    for (int k = 0; k < g.nmem; ++k) {
        a.p[k] = const_cast<T *>(t1[k]);
        b.p[k] = const_cast<T *>(t2[k]);
        int vec4 = (g.len[k] % 4 == 0) && al4(t1[k]) && al4(t2[k]);
        for (int v = 0; v < nv; ++v) {
            vl.v[v][k] = xs[(size_t)v * g.nmem + k];
            vec4 = vec4 && al4(vl.v[v][k]);
        }
        gm.vec[k] = vec4;
    }
    const GSysD gs = sys_of(g);
    constexpr int GV = 4;
    cudaError_t e = launch_pdl(k_ggram2_partial<T, GV>, dim3(g.nblk, g.nsys, (nv + GV - 1) / GV),
                               dim3(256), 0, s, nv, vl, a, b, gm, gs);
    if (e != cudaSuccess) return e;
    const int count = 2 * nv * g.nsys;
    e = launch_pdl(k_greduce, dim3((count + 3) / 4), dim3(128), 0, s, gm, gs, g.nsys, count,
                   g.nblk, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

static unsigned axpy_blocks(const GLaunch &g, long long per_block) {
    long long len = 1;
    for (int k = 0; k < g.nmem; ++k) len = g.len[k] > len ? g.len[k] : len;
    long long bx = (len + per_block - 1) / per_block;
    const long long cap = (152LL * 16 + g.nsys - 1) / g.nsys;
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    return (unsigned)bx;
}

template <typename T>
cudaError_t launch_gaxpy2(const GLaunch &g, int nv, const T *const *xs, const double *c1,
                          const double *c2, const double *c21, const double *post1,
                          const double *post2, T *const *y1, T *const *y2, const int *write1,
                          cudaStream_t s) {
    if (!group_ok(g, nv)) return cudaErrorInvalidValue;
    GVecD<T> vl{};
    GTgtD<T> a{}, b{};
    GAxpy2D<T> aa{};
    for (int k = 0; k < g.nmem; ++k) {
        a.p[k] = y1[k];
        b.p[k] = y2[k];
        for (int v = 0; v < nv; ++v) vl.v[v][k] = xs[(size_t)v * g.nmem + k];
    }
    for (int i = 0; i < g.nsys; ++i) {
        for (int v = 0; v < nv; ++v) {
            aa.c1[v * NSYS_MAX + i] = (T)c1[(size_t)v * g.nsys + i];
            aa.c2[v * NSYS_MAX + i] = (T)c2[(size_t)v * g.nsys + i];
        }
        aa.c21[i] = (T)c21[i];
        aa.post1[i] = (T)post1[i];
        aa.post2[i] = (T)post2[i];
        aa.write1[i] = write1[i];
    }
    GMemD gm = mem_of(g);
    for (int k = 0; k < g.nmem; ++k) {  // pair loads: every vector aligned to two elements
        int vec2 = (g.len[k] % 2 == 0) && al2<T>(y1[k]) && al2<T>(y2[k]);
        for (int v = 0; v < nv; ++v) vec2 = vec2 && al2<T>(vl.v[v][k]);
        gm.vec[k] = vec2;
    }
    const dim3 grid(axpy_blocks(g, 256), g.nsys);
    const GSysD gs = sys_of(g);
    cudaError_t e;
    switch (nv) {
#define ST_GAXPY2_CASE(C) \
    case C: e = launch_pdl(k_gaxpy2<T, C>, grid, dim3(256), 0, s, nv, vl, a, b, aa, gm, gs); break;
        ST_GAXPY2_CASE(0)
        ST_GAXPY2_CASE(1)
        ST_GAXPY2_CASE(2)
        ST_GAXPY2_CASE(3)
        ST_GAXPY2_CASE(4)
        ST_GAXPY2_CASE(5)
        ST_GAXPY2_CASE(6)
        ST_GAXPY2_CASE(7)
        ST_GAXPY2_CASE(8)
#undef ST_GAXPY2_CASE
        default: e = launch_pdl(k_gaxpy2<T, -1>, grid, dim3(256), 0, s, nv, vl, a, b, aa, gm, gs);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_gaxpy(const GLaunch &g, int nv, const T *const *xs, const double *coef,
                         T *const *y, const double *post, cudaStream_t s, bool y_zero) {
    if (!group_ok(g, nv)) return cudaErrorInvalidValue;
    for (int i = 0; i < g.nsys; ++i)
        if (g.snv[i] < 0 || g.snv[i] > nv) return cudaErrorInvalidValue;
    if (nv == 0 && !post) return cudaSuccess;
    GVecD<T> vl{};
    GTgtD<T> ty{};
    GAxpyD<T> aa{};
    GMemD gm = mem_of(g);
    for (int k = 0; k < g.nmem; ++k) {
        ty.p[k] = y[k];
        int nvk = 0;  // vectors member k's systems use
        for (int i = 0; i < g.nsys; ++i)
            if (g.sm[i] == k && g.snv[i] > nvk) nvk = g.snv[i];
        int vec2 = (g.len[k] % 2 == 0) && al2<T>(y[k]);
        for (int v = 0; v < nv; ++v) {
            vl.v[v][k] = xs[(size_t)v * g.nmem + k];
            if (v < nvk) vec2 = vec2 && al2<T>(vl.v[v][k]);
        }
        gm.vec[k] = vec2;
    }
    for (int i = 0; i < g.nsys; ++i) {
        for (int v = 0; v < nv; ++v) aa.coef[v * NSYS_MAX + i] = (T)coef[(size_t)v * g.nsys + i];
        aa.post[i] = post ? (T)post[i] : T(1);
    }
    const cudaError_t e = launch_pdl(k_gaxpy<T>, dim3(axpy_blocks(g, 512), g.nsys), dim3(256), 0,
                                     s, vl, ty, aa, gm, sys_of(g), y_zero ? 1 : 0);
    return e != cudaSuccess ? e : cudaGetLastError();
}

struct ScaleArgs {
    double a[NRHS_MAX];
};

// y (FP64) += a_r * x (FP32), per rhs r: the refinement update
// y_r += a_r x_r (store: y_r = 0 + a_r x_r, y not read), one grid row per
// right-hand side r
__global__ void k_axpy_f32_f64(const float *__restrict__ x, double *__restrict__ y,
                               const __grid_constant__ ScaleArgs sa, long long len, int store) {
    const long long off = (long long)blockIdx.y * len;
    const double a = sa.a[blockIdx.y];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        y[off + i] = (store ? 0.0 : y[off + i]) + a * (double)x[off + i];
}

cudaError_t launch_axpy_f32_f64(const float *x, double *y, const double *a, int nrhs,
                                long long len, cudaStream_t s, bool store) {
    if (nrhs > NRHS_MAX) return cudaErrorInvalidValue;
    if (nrhs <= 0 || len <= 0) return cudaSuccess;
    ScaleArgs sa;
    for (int r = 0; r < nrhs; ++r) sa.a[r] = a[r];
    long long bx = (len + 255) / 256;
    const long long cap = (152LL * 16 + nrhs - 1) / nrhs;
    if (bx > cap) bx = cap;
    k_axpy_f32_f64<<<dim3((unsigned)bx, (unsigned)nrhs), 256, 0, s>>>(x, y, sa, len, store ? 1 : 0);
    return cudaGetLastError();
}

__global__ void k_scale(const double *__restrict__ x, double *y, const __grid_constant__ ScaleArgs sa,
                        long long len, int nrhs) {
    const long long n = (long long)nrhs * len;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = sa.a[i / len] * x[i];
}

cudaError_t launch_scale(const double *x, double *y, const double *a, int nrhs, long long len,
                         cudaStream_t s) {
    if (nrhs > NRHS_MAX) return cudaErrorInvalidValue;
    ScaleArgs sa;
    for (int r = 0; r < nrhs; ++r) sa.a[r] = a[r];
    long long blocks = ((long long)nrhs * len + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks <= 0) return cudaSuccess;
    k_scale<<<(unsigned)blocks, 256, 0, s>>>(x, y, sa, len, nrhs);
    return cudaGetLastError();
}

struct ScaleArgsF {
    float a[NRHS_MAX];
};

// y (FP32) = float(x) * s_r per rhs r: the refinement's scaled FP32 right-hand
// side in one pass (the rounding of a conversion followed by an FP32 scaling)
__global__ void k_convert_scale(const double *__restrict__ x, float *__restrict__ y,
                                const __grid_constant__ ScaleArgsF sa, long long len, int vec2) {
    const int r = blockIdx.y;
    const long long off = (long long)r * len;
    const float s = sa.a[r];
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (vec2) {  // off is even because len is
        const double2 *x2 = reinterpret_cast<const double2 *>(x + off);
        float2 *y2 = reinterpret_cast<float2 *>(y + off);
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len / 2; i += stride) {
            const double2 v = x2[i];
            y2[i] = make_float2(__fmul_rn((float)v.x, s), __fmul_rn((float)v.y, s));
        }
        return;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride)
        y[off + i] = __fmul_rn((float)x[off + i], s);
}

cudaError_t launch_convert_scale(const double *x, float *y, const double *scale, int nrhs,
                                 long long len, cudaStream_t s) {
    if (nrhs > NRHS_MAX || nrhs < 1) return cudaErrorInvalidValue;
    if (len <= 0) return cudaSuccess;
    ScaleArgsF sa;
    for (int r = 0; r < nrhs; ++r) sa.a[r] = (float)scale[r];
    const int vec2 = (len % 2 == 0) && aligned16(x) && ((reinterpret_cast<uintptr_t>(y) & 7u) == 0);
    long long bx = (len / 2 + 255) / 256;
    const long long cap = (152LL * 16 + nrhs - 1) / nrhs;
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    k_convert_scale<<<dim3((unsigned)bx, (unsigned)nrhs), 256, 0, s>>>(x, y, sa, len, vec2);
    return cudaGetLastError();
}

// f[slab][t][z][y][x] = sum_k gt[k][slab][t] gz[k][z] gy[k][y] gx[k][x]
__global__ void k_separable_sum(double *__restrict__ f, const double *__restrict__ g, int K,
                                long long nslab_t, int nx, int ny, int nz, long long total) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const long long nxyz = (long long)nx * ny * nz;
    const long long st = idx / nxyz, sp = idx % nxyz;
    const int x = (int)(sp % nx), y = (int)((sp / nx) % ny), z = (int)(sp / ((long long)nx * ny));
    const long long per = nslab_t + nx + ny + nz;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        const double *gk = g + k * per;
        acc += gk[st] * gk[nslab_t + x] * gk[nslab_t + nx + y] * gk[nslab_t + nx + ny + z];
    }
    f[idx] = acc;
}

cudaError_t launch_separable_sum(double *f, const double *g, int K, long long nslab_t, int nx,
                                 int ny, int nz, cudaStream_t s) {
    const long long total = nslab_t * nx * ny * nz;
    if (total <= 0) return cudaSuccess;
    k_separable_sum<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(f, g, K, nslab_t, nx, ny, nz,
                                                                    total);
    return cudaGetLastError();
}

template cudaError_t launch_convert<double, float>(const double *, float *, long long, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float *, double *, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_zero<double>(double *, long long, cudaStream_t);
template cudaError_t launch_zero<float>(float *, long long, cudaStream_t);
#define ST_GVEC(T)                                                                             \
    template cudaError_t launch_gdot<T>(const GLaunch &, int, const T *const *, const T *const *, \
                                        double *, cudaStream_t);                                  \
    template cudaError_t launch_gnorm2<T>(const GLaunch &, int, const T *const *, double *,       \
                                          cudaStream_t);                                          \
    template cudaError_t launch_ggram2<T>(const GLaunch &, int, const T *const *,                \
                                          const T *const *, const T *const *, double *,           \
                                          cudaStream_t);                                          \
    template cudaError_t launch_gaxpy<T>(const GLaunch &, int, const T *const *, const double *,  \
                                         T *const *, const double *, cudaStream_t, bool);         \
    template cudaError_t launch_gaxpy2<T>(const GLaunch &, int, const T *const *, const double *, \
                                          const double *, const double *, const double *,         \
                                          const double *, T *const *, T *const *, const int *,    \
                                          cudaStream_t);
ST_GVEC(float)
ST_GVEC(double)
#undef ST_GVEC

}  // namespace st

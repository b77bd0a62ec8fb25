// Vector kernels of the FP64 outer iteration (FGMRES, Sec. 3.1 outer solver
// of arXiv:1802.09277) and precision conversion for the mixed V-cycle.
// Reductions are deterministic: fixed-size per-block partial sums, then one
// fixed-order pass.
#include "pdl.cuh"
#include "st_internal.h"

namespace st {

constexpr int NRHS_MAX = 32;

template <typename T>
struct VecList {
    const T *v[MAXV];
};
template <typename T>
struct AxpyArgs {
    const T *x[MAXV];
    T coef[MAXV * NRHS_MAX];  // rounded to T on the host
    T post[NRHS_MAX];         // y <- post_r * (y + sum_v coef x_v)
};

// two outputs sharing the vectors x_v (the delayed Gram-Schmidt step):
//   y1 <- post1_r * (y1 + sum_v c1 x_v)
//   y2 <- post2_r * (y2 + c21_r * y1_old + sum_v c2 x_v)
template <typename T>
struct Axpy2Args {
    const T *x[MAXV];
    T c1[MAXV * NRHS_MAX];
    T c2[MAXV * NRHS_MAX];
    T c21[NRHS_MAX];
    T post1[NRHS_MAX], post2[NRHS_MAX];
};

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

// grid (nblk, nrhs, ceil(nv / 4)), 256 threads; partial[(v*nrhs + r)*nblk + blk].
// Block (b, r, g) accumulates the dots of w with vectors 4g .. 4g+3 over a
// grid-stride loop, two elements per load when vec2 is set.  w is re-read
// by every group from L2.
template <typename T>
__global__ void __launch_bounds__(256)
    k_multidot_partial(int nv, const __grid_constant__ VecList<T> vl, const T *__restrict__ w,
                       long long len, double *__restrict__ partial, int vec2) {
    griddep_wait();
    griddep_launch();
    using P2 = typename Pair<T>::V;
    __shared__ typename Red<T>::V red[8][4];
    const int r = blockIdx.y, nblk = gridDim.x, nrhs = gridDim.y;
    const int v0 = 4 * blockIdx.z;
    const int cnt = (nv - v0 < 4) ? nv - v0 : 4;
    const long long off = (long long)r * len;
    const T *x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = vl.v[(k < cnt) ? v0 + k : v0] + off;
    DotAcc<T> acc[4];
    const long long stride = (long long)nblk * blockDim.x;
    if (vec2) {
        const P2 *w2 = reinterpret_cast<const P2 *>(w + off);
        const long long np = len / 2;
#pragma unroll 2
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
            const P2 wi = w2[i];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < cnt) {
                    const P2 a = reinterpret_cast<const P2 *>(x[k])[i];
                    acc[k].add(a.x, wi.x);
                    acc[k].add(a.y, wi.y);
                }
        }
    } else {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
            const T wi = w[off + i];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < cnt) acc[k].add(x[k][i], wi);
        }
    }
    using RD = Red<T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= cnt) break;
        const typename RD::V t = RD::warp(RD::of(acc[k]));
        if (lane == 0) red[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        typename RD::V t = RD::zero();
        for (int q = 0; q < 8; ++q) t = RD::add(t, red[q][threadIdx.x]);
        partial[((long long)(v0 + threadIdx.x) * nrhs + r) * nblk + blockIdx.x] = RD::out(t);
    }
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// one warp per output; lane-strided partial sums, then a fixed shuffle tree
__global__ void k_reduce_partials(const double *__restrict__ partial, int nblk, int count,
                                  double *__restrict__ out) {
    griddep_wait();
    griddep_launch();
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= count) return;
    double t = 0.0;
    for (int b = lane; b < nblk; b += 32) t += partial[(long long)i * nblk + b];
    t = warp_sum(t);
    if (lane == 0) out[i] = t;
}

template <typename T>
cudaError_t launch_multidot(int nv, const T *const *vecs, const T *w, int nrhs, long long len,
                            double *partial, int nblk, double *out, cudaStream_t s) {
    if (nv > MAXV || nrhs > 65535 || nv <= 0) return cudaErrorInvalidValue;
    VecList<T> vl;
    auto al = [](const void *p) {
        return sizeof(T) == 8 ? aligned16(p) : ((reinterpret_cast<uintptr_t>(p) & 7u) == 0);
    };
    int vec2 = (len % 2 == 0) && al(w);
    for (int i = 0; i < nv; ++i) {
        vl.v[i] = vecs[i];
        vec2 = vec2 && al(vecs[i]);
    }
    cudaError_t e = launch_pdl(k_multidot_partial<T>, dim3(nblk, nrhs, (nv + 3) / 4), dim3(256),
                               0, s, nv, vl, w, len, partial, vec2);
    if (e != cudaSuccess) return e;
    const int count = nv * nrhs;
    e = launch_pdl(k_reduce_partials, dim3((count + 3) / 4), dim3(128), 0, s, partial, nblk,
                   count, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// grid (blocks, nrhs): block row r handles right-hand side r (no index division)
template <typename T>
__global__ void __launch_bounds__(256)
    k_multiaxpy(int nv, const __grid_constant__ AxpyArgs<T> aa, long long len,
                T *__restrict__ y, int vec2) {
    griddep_wait();
    griddep_launch();
    using P2 = typename Pair<T>::V;
    const int r = blockIdx.y;
    const long long off = (long long)r * len;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const T post = aa.post[r];
    if (vec2) {  // off is even because len is
        const long long n = len / 2;
        P2 *y2 = reinterpret_cast<P2 *>(y + off);
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            P2 acc = y2[i];
            for (int v = 0; v < nv; ++v) {
                const T c = aa.coef[v * NRHS_MAX + r];
                const P2 x = reinterpret_cast<const P2 *>(aa.x[v] + off)[i];
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
        T acc = y[off + i];
        for (int v = 0; v < nv; ++v) acc += aa.coef[v * NRHS_MAX + r] * aa.x[v][off + i];
        y[off + i] = post * acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_axpy2(int nv, const __grid_constant__ Axpy2Args<T> aa, long long len, T *__restrict__ y1,
            T *__restrict__ y2, int write1) {
    griddep_wait();
    griddep_launch();
    const int r = blockIdx.y;
    const long long off = (long long)r * len;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const T p1 = aa.post1[r], p2 = aa.post2[r], c21 = aa.c21[r];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const T a1o = y1[off + i];
        T a1 = a1o, a2 = y2[off + i] + c21 * a1o;
        for (int v = 0; v < nv; ++v) {
            const T x = aa.x[v][off + i];
            a1 += aa.c1[v * NRHS_MAX + r] * x;
            a2 += aa.c2[v * NRHS_MAX + r] * x;
        }
        if (write1) y1[off + i] = p1 * a1;
        y2[off + i] = p2 * a2;
    }
}

// grid (nblk, nrhs, ceil(nv / GV)): the dots of vectors GV g .. GV g + GV - 1
// with two targets t1, t2 in one pass; partial[((v * 2 + t) * nrhs + r) * nblk + blk].
// vec4: 16-byte loads (len a multiple of 4, 16-byte aligned vectors); each
// thread forms the 4-term products of a chunk in T and adds them into its
// accumulator (Kahan-compensated in FP32), so the compensation runs once per
// 4 elements.
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

template <typename T, int GV>
__global__ void __launch_bounds__(256)
    k_gram2_partial(int nv, const __grid_constant__ VecList<T> vl, const T *__restrict__ t1,
                    const T *__restrict__ t2, long long len, double *__restrict__ partial,
                    int vec4) {
    griddep_wait();
    griddep_launch();
    __shared__ typename Red<T>::V red[8][2 * GV];
    const int r = blockIdx.y, nblk = gridDim.x, nrhs = gridDim.y;
    const int v0 = GV * blockIdx.z;
    const int cnt = (nv - v0 < GV) ? nv - v0 : GV;
    const long long off = (long long)r * len;
    const T *x[GV];
#pragma unroll
    for (int k = 0; k < GV; ++k) x[k] = vl.v[(k < cnt) ? v0 + k : v0] + off;
    DotAcc<T> a1[GV], a2[GV];
    static_assert(GV == 4, "the count dispatch below covers GV = 4");
    switch (cnt) {  // uniform across the grid row
        case 1: gram2_body<T, 1>(x, t1 + off, t2 + off, len, vec4, a1, a2); break;
        case 2: gram2_body<T, 2>(x, t1 + off, t2 + off, len, vec4, a1, a2); break;
        case 3: gram2_body<T, 3>(x, t1 + off, t2 + off, len, vec4, a1, a2); break;
        default: gram2_body<T, 4>(x, t1 + off, t2 + off, len, vec4, a1, a2); break;
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
        partial[((long long)(2 * v + which) * nrhs + r) * nblk + blockIdx.x] = RD::out(t);
    }
}

template <typename T>
cudaError_t launch_gram2(int nv, const T *const *vecs, const T *t1, const T *t2, int nrhs,
                         long long len, double *partial, int nblk, double *out, cudaStream_t s) {
    if (nv > MAXV || nrhs > 65535 || nv <= 0) return cudaErrorInvalidValue;
    VecList<T> vl;
    // 4-element loads need the vectors aligned to 4 elements (16 or 32 bytes)
    const uintptr_t am = 4 * sizeof(T) - 1;
    auto al4 = [am](const void *p) { return (reinterpret_cast<uintptr_t>(p) & am) == 0; };
    int vec4 = (len % 4 == 0) && al4(t1) && al4(t2);
    for (int i = 0; i < nv; ++i) {
        vl.v[i] = vecs[i];
        vec4 = vec4 && al4(vecs[i]);
    }
    constexpr int GV = 4;
    cudaError_t e = launch_pdl(k_gram2_partial<T, GV>, dim3(nblk, nrhs, (nv + GV - 1) / GV),
                               dim3(256), 0, s, nv, vl, t1, t2, len, partial, vec4);
    if (e != cudaSuccess) return e;
    const int count = 2 * nv * nrhs;
    e = launch_pdl(k_reduce_partials, dim3((count + 3) / 4), dim3(128), 0, s, partial, nblk,
                   count, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpy2(int nv, const T *const *xs, const double *c1, const double *c2,
                         const double *c21, const double *post1, const double *post2, int nrhs,
                         long long len, T *y1, T *y2, int write1, cudaStream_t s) {
    if (nv > MAXV || nrhs > NRHS_MAX || nv < 0) return cudaErrorInvalidValue;
    Axpy2Args<T> aa;
    for (int v = 0; v < nv; ++v) {
        aa.x[v] = xs[v];
        for (int r = 0; r < nrhs; ++r) {
            aa.c1[v * NRHS_MAX + r] = (T)c1[v * nrhs + r];
            aa.c2[v * NRHS_MAX + r] = (T)c2[v * nrhs + r];
        }
    }
    for (int r = 0; r < nrhs; ++r) {
        aa.c21[r] = (T)c21[r];
        aa.post1[r] = (T)post1[r];
        aa.post2[r] = (T)post2[r];
    }
    long long bx = (len + 255) / 256;
    const long long cap = (152LL * 16 + nrhs - 1) / nrhs;
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    const cudaError_t e = launch_pdl(k_axpy2<T>, dim3((unsigned)bx, (unsigned)nrhs), dim3(256), 0,
                                     s, nv, aa, len, y1, y2, write1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_multiaxpy(int nv, const T *const *xs, const double *coef, int nrhs,
                             long long len, T *y, cudaStream_t s, const double *post) {
    if (nv > MAXV || nrhs > NRHS_MAX || nv < 0) return cudaErrorInvalidValue;
    if (nv == 0 && !post) return cudaSuccess;
    AxpyArgs<T> aa;
    for (int v = 0; v < nv; ++v) {
        aa.x[v] = xs[v];
        for (int r = 0; r < nrhs; ++r) aa.coef[v * NRHS_MAX + r] = (T)coef[v * nrhs + r];
    }
    for (int r = 0; r < nrhs; ++r) aa.post[r] = post ? (T)post[r] : T(1);
    const bool al = sizeof(T) == 8 ? aligned16(y) : ((reinterpret_cast<uintptr_t>(y) & 7u) == 0);
    int vec2 = (len % 2 == 0) && al;
    for (int v = 0; v < nv; ++v)
        vec2 = vec2 && (sizeof(T) == 8 ? aligned16(xs[v])
                                       : ((reinterpret_cast<uintptr_t>(xs[v]) & 7u) == 0));
    long long bx = (len + 511) / 512;
    const long long cap = (152LL * 16 + nrhs - 1) / nrhs;
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    const cudaError_t e = launch_pdl(k_multiaxpy<T>, dim3((unsigned)bx, (unsigned)nrhs),
                                     dim3(256), 0, s, nv, aa, len, y, vec2);
    return e != cudaSuccess ? e : cudaGetLastError();
}

struct ScaleArgs {
    double a[NRHS_MAX];
};

// y (FP64) += a_r * x (FP32), per rhs r: the refinement update
__global__ void k_axpy_f32_f64(const float *__restrict__ x, double *__restrict__ y,
                               const __grid_constant__ ScaleArgs sa, long long len, int nrhs) {
    const long long n = (long long)nrhs * len;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] += sa.a[i / len] * (double)x[i];
}

cudaError_t launch_axpy_f32_f64(const float *x, double *y, const double *a, int nrhs,
                                long long len, cudaStream_t s) {
    if (nrhs > NRHS_MAX) return cudaErrorInvalidValue;
    ScaleArgs sa;
    for (int r = 0; r < nrhs; ++r) sa.a[r] = a[r];
    long long blocks = ((long long)nrhs * len + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks <= 0) return cudaSuccess;
    k_axpy_f32_f64<<<(unsigned)blocks, 256, 0, s>>>(x, y, sa, len, nrhs);
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
template cudaError_t launch_multidot<double>(int, const double *const *, const double *, int,
                                             long long, double *, int, double *, cudaStream_t);
template cudaError_t launch_multidot<float>(int, const float *const *, const float *, int,
                                            long long, double *, int, double *, cudaStream_t);
template cudaError_t launch_multiaxpy<double>(int, const double *const *, const double *, int,
                                              long long, double *, cudaStream_t, const double *);
template cudaError_t launch_multiaxpy<float>(int, const float *const *, const double *, int,
                                             long long, float *, cudaStream_t, const double *);
template cudaError_t launch_zero<float>(float *, long long, cudaStream_t);
template cudaError_t launch_gram2<float>(int, const float *const *, const float *, const float *,
                                         int, long long, double *, int, double *, cudaStream_t);
template cudaError_t launch_gram2<double>(int, const double *const *, const double *,
                                          const double *, int, long long, double *, int,
                                          double *, cudaStream_t);
template cudaError_t launch_axpy2<float>(int, const float *const *, const double *,
                                         const double *, const double *, const double *,
                                         const double *, int, long long, float *, float *, int,
                                         cudaStream_t);
template cudaError_t launch_axpy2<double>(int, const double *const *, const double *,
                                          const double *, const double *, const double *,
                                          const double *, int, long long, double *, double *,
                                          int, cudaStream_t);

}  // namespace st

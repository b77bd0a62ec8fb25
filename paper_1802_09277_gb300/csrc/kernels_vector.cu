// Vector kernels of the FP64 outer iteration (FGMRES, Sec. 3.1 outer solver
// of arXiv:1802.09277) and precision conversion for the mixed V-cycle.
// Reductions are deterministic: fixed-size per-block partial sums, then one
// fixed-order pass.
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
    double coef[MAXV * NRHS_MAX];
    double post[NRHS_MAX];  // y <- post_r * (y + sum_v coef x_v)
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
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// grid (nblk, nrhs, ceil(nv / 4)), 256 threads; partial[(v*nrhs + r)*nblk + blk].
// Block (b, r, g) accumulates the dots of w with vectors 4g .. 4g+3 over a
// grid-stride loop, two elements per load when vec2 is set.  w is re-read
// by every group from L2.
template <typename T>
__global__ void __launch_bounds__(256)
    k_multidot_partial(int nv, const __grid_constant__ VecList<T> vl, const T *__restrict__ w,
                       long long len, double *__restrict__ partial, int vec2) {
    using P2 = typename Pair<T>::V;
    __shared__ double red[8][4];
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double t = warp_sum(acc[k].value());
        if (lane == 0) red[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
        partial[((long long)(v0 + threadIdx.x) * nrhs + r) * nblk + blockIdx.x] = t;
    }
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// one warp per output; lane-strided partial sums, then a fixed shuffle tree
__global__ void k_reduce_partials(const double *__restrict__ partial, int nblk, int count,
                                  double *__restrict__ out) {
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
    k_multidot_partial<T><<<dim3(nblk, nrhs, (nv + 3) / 4), 256, 0, s>>>(nv, vl, w, len, partial,
                                                                        vec2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int count = nv * nrhs;
    k_reduce_partials<<<(count + 3) / 4, 128, 0, s>>>(partial, nblk, count, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_multiaxpy(int nv, const __grid_constant__ AxpyArgs<T> aa, int nrhs,
                            long long len, T *__restrict__ y, int vec2) {
    using P2 = typename Pair<T>::V;
    if (vec2) {  // pairs never straddle two rhs because len is even
        const long long n = (long long)nrhs * len / 2;
        P2 *y2 = reinterpret_cast<P2 *>(y);
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const int r = (int)((2 * i) / len);
            P2 acc = y2[i];
            for (int v = 0; v < nv; ++v) {
                const T c = (T)aa.coef[v * NRHS_MAX + r];
                const P2 x = reinterpret_cast<const P2 *>(aa.x[v])[i];
                acc.x += c * x.x;
                acc.y += c * x.y;
            }
            acc.x *= (T)aa.post[r];
            acc.y *= (T)aa.post[r];
            y2[i] = acc;
        }
        return;
    }
    const long long n = (long long)nrhs * len;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / len);
        T acc = y[i];
        for (int v = 0; v < nv; ++v) acc += (T)aa.coef[v * NRHS_MAX + r] * aa.x[v][i];
        y[i] = (T)aa.post[r] * acc;
    }
}

template <typename T>
cudaError_t launch_multiaxpy(int nv, const T *const *xs, const double *coef, int nrhs,
                             long long len, T *y, cudaStream_t s, const double *post) {
    if (nv > MAXV || nrhs > NRHS_MAX || nv < 0) return cudaErrorInvalidValue;
    if (nv == 0 && !post) return cudaSuccess;
    AxpyArgs<T> aa;
    for (int v = 0; v < nv; ++v) {
        aa.x[v] = xs[v];
        for (int r = 0; r < nrhs; ++r) aa.coef[v * NRHS_MAX + r] = coef[v * nrhs + r];
    }
    for (int r = 0; r < nrhs; ++r) aa.post[r] = post ? post[r] : 1.0;
    const bool al = sizeof(T) == 8 ? aligned16(y) : ((reinterpret_cast<uintptr_t>(y) & 7u) == 0);
    int vec2 = (len % 2 == 0) && al;
    for (int v = 0; v < nv; ++v)
        vec2 = vec2 && (sizeof(T) == 8 ? aligned16(xs[v])
                                       : ((reinterpret_cast<uintptr_t>(xs[v]) & 7u) == 0));
    long long blocks = ((long long)nrhs * len + 511) / 512;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_multiaxpy<T><<<(unsigned)blocks, 256, 0, s>>>(nv, aa, nrhs, len, y, vec2);
    return cudaGetLastError();
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

}  // namespace st

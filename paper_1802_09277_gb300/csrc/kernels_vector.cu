// Vector kernels of the FP64 outer iteration (FGMRES, Sec. 3.1 outer solver
// of arXiv:1802.09277) and precision conversion for the mixed V-cycle.
// Reductions are deterministic: fixed-size per-block partial sums, then one
// fixed-order pass.
#include "st_internal.h"

namespace st {

constexpr int NRHS_MAX = 32;

struct VecList {
    const double *v[MAXV];
};
struct AxpyArgs {
    const double *x[MAXV];
    double coef[MAXV * NRHS_MAX];
    double post[NRHS_MAX];  // y <- post_r * (y + sum_v coef x_v)
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

// grid (nblk, nrhs), 256 threads; partial[(v*nrhs + r)*nblk + blk].
// One pass over w: every thread keeps the nv running sums in registers.
__global__ void __launch_bounds__(256)
    k_multidot_partial(int nv, const __grid_constant__ VecList vl, const double *__restrict__ w,
                       long long len, double *__restrict__ partial) {
    __shared__ double red[8][MAXV];
    const int r = blockIdx.y, nblk = gridDim.x, nrhs = gridDim.y;
    const long long chunk = (len + nblk - 1) / nblk;
    const long long lo = blockIdx.x * chunk;
    const long long hi = (lo + chunk < len) ? lo + chunk : len;
    const long long off = (long long)r * len;
    double acc[MAXV];
#pragma unroll
    for (int v = 0; v < MAXV; ++v) acc[v] = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double wi = w[off + i];
#pragma unroll
        for (int v = 0; v < MAXV; ++v)
            if (v < nv) acc[v] += vl.v[v][off + i] * wi;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < MAXV; ++v) {
        if (v >= nv) break;
        const double t = warp_sum(acc[v]);
        if (lane == 0) red[warp][v] = t;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
        partial[((long long)threadIdx.x * nrhs + r) * nblk + blockIdx.x] = t;
    }
}

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

cudaError_t launch_multidot(int nv, const double *const *vecs, const double *w, int nrhs,
                            long long len, double *partial, int nblk, double *out,
                            cudaStream_t s) {
    if (nv > MAXV || nrhs > 65535 || nv <= 0) return cudaErrorInvalidValue;
    VecList vl;
    for (int i = 0; i < nv; ++i) vl.v[i] = vecs[i];
    k_multidot_partial<<<dim3(nblk, nrhs), 256, 0, s>>>(nv, vl, w, len, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int count = nv * nrhs;
    k_reduce_partials<<<(count + 3) / 4, 128, 0, s>>>(partial, nblk, count, out);
    return cudaGetLastError();
}

__global__ void k_multiaxpy(int nv, const __grid_constant__ AxpyArgs aa, int nrhs, long long len,
                            double *__restrict__ y) {
    const long long n = (long long)nrhs * len;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / len);
        double acc = y[i];
        for (int v = 0; v < nv; ++v) acc += aa.coef[v * NRHS_MAX + r] * aa.x[v][i];
        y[i] = aa.post[r] * acc;
    }
}

cudaError_t launch_multiaxpy(int nv, const double *const *xs, const double *coef, int nrhs,
                             long long len, double *y, cudaStream_t s, const double *post) {
    if (nv > MAXV || nrhs > NRHS_MAX || nv < 0) return cudaErrorInvalidValue;
    if (nv == 0 && !post) return cudaSuccess;
    AxpyArgs aa;
    for (int v = 0; v < nv; ++v) {
        aa.x[v] = xs[v];
        for (int r = 0; r < nrhs; ++r) aa.coef[v * NRHS_MAX + r] = coef[v * nrhs + r];
    }
    for (int r = 0; r < nrhs; ++r) aa.post[r] = post ? post[r] : 1.0;
    long long blocks = ((long long)nrhs * len + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_multiaxpy<<<(unsigned)blocks, 256, 0, s>>>(nv, aa, nrhs, len, y);
    return cudaGetLastError();
}

struct ScaleArgs {
    double a[NRHS_MAX];
};

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

template cudaError_t launch_convert<double, float>(const double *, float *, long long, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float *, double *, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_zero<double>(double *, long long, cudaStream_t);
template cudaError_t launch_zero<float>(float *, long long, cudaStream_t);

}  // namespace st

// Device helpers shared by the eigenbasis kernels (arXiv:1802.09277, Sec.
// 3.1 smoother with the slab inverse of Eq. 3.1 per spatial mode).
#pragma once
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
    if (c.variant == 2) {  // complex Schur (Sec. 3.4, Algorithm 1): complex triangular Z
        T wr[NTMAX], wi[NTMAX], zr[NTMAX], zi[NTMAX];
#pragma unroll
        for (int i = 0; i < NTMAX; ++i) {
            T ar = T(0), ai = T(0);
#pragma unroll
            for (int j = 0; j < NTMAX; ++j)
                if (j < nt) {
                    ar += c.Y[i * NTMAX + j] * r[j];
                    ai += c.Yi[i * NTMAX + j] * r[j];
                }
            wr[i] = ar;
            wi[i] = ai;
            zr[i] = T(0);
            zi[i] = T(0);
        }
        // back substitution (Z + mu I) z = w, complex
#pragma unroll
        for (int i = NTMAX - 1; i >= 0; --i) {
            if (i >= nt) continue;
            T gr = wr[i], gi = wi[i];
#pragma unroll
            for (int j = i + 1; j < NTMAX; ++j)
                if (j < nt) {
                    gr -= c.Z[i * NTMAX + j] * zr[j] - c.Zi[i * NTMAX + j] * zi[j];
                    gi -= c.Z[i * NTMAX + j] * zi[j] + c.Zi[i * NTMAX + j] * zr[j];
                }
            const T dr = c.Z[i * NTMAX + i] + mu, di = c.Zi[i * NTMAX + i];
            const T rden = recip(dr * dr + di * di);
            zr[i] = (gr * dr + gi * di) * rden;
            zi[i] = (gi * dr - gr * di) * rden;
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

inline ModeLaunch mode_launch(long long nmodes, long long nslabs) {
    ModeLaunch L;
    const int th = nmodes >= 256 ? 256 : (int)((nmodes + 31) / 32 * 32);
    L.block = dim3((unsigned)th);
    const long long gy = nslabs < 65535 ? nslabs : 65535;
    L.grid = dim3((unsigned)((nmodes + th - 1) / th), (unsigned)gy,
                  (unsigned)((nslabs + gy - 1) / gy));
    return L;
}

}  // namespace st

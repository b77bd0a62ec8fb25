// Matrix-free slab operator of the space-time system (Eq. 2.4, Eq. 2.5 of
// arXiv:1802.09277), sum-factorised over the banded 1D B-spline matrices.
//
// For every slab n and spatial point, with m_j = M_x u_{n,j} and
// k_j = K_x u_{n,j} (M_x = M1z(x)M1y(x)M1x, K_x = sum over axes of K1 in one
// slot) and the coupling plane m_prev = M_x u_{n-1,nt-1} (B_n = N_t (x) M_x,
// N_t = e_1 e_nt^T for open knots):
//   MODE_RES  : r_i = f_i - sum_j (Kt[i][j] m_j + Mt[i][j] k_j) + [i==0] m_prev
//   MODE_APPLY: y_i =       sum_j (Kt[i][j] m_j + Mt[i][j] k_j) - [i==0] m_prev
//   MODE_MASS : y_i =       sum_j  Mt[i][j] m_j                  (load vector)
// optionally followed by the forward time transform w = Y r (the first step
// of applying A_n^{-1} through Eq. 3.1).
//
// One CTA owns one spatial tile (all time planes) of `sch` consecutive slabs.
// Each plane tile plus a halo of p is staged in shared memory, then reduced
// axis by axis: x-pass (M1x, K1x), y-pass, z-pass; the 2p+1 band
// coefficients of the tile's rows are staged once per CTA.
//
// In double-float the coupling term enters the accumulator of time plane 0
// as one more Dot2 term (-m_prev), ahead of the slab's own terms, and a CTA
// with several slabs keeps M_x u of each slab's last time plane for the next
// one: B_n u_{n-1} is then never recomputed inside a CTA (one mass-only plane
// of staging and three passes saved per slab; 8 % of the multiply-adds at
// N_t = 4).  The carried value has the bits a recomputation would give (the
// mass passes are the same operation sequence), so the result does not
// depend on `sch`.  FP64 and FP32 run one slab per CTA and add the coupling
// term in the epilogue.
//
// Storage type T (FP64 or FP32 in HBM) and compute type C are separate: the
// FP64-accurate residual of the mixed-precision refinement computes in
// double-float (C = dfloat) on FP64 data, converting on load and store.
#pragma once
#include <type_traits>

#include "st_internal.h"

namespace st {

template <typename C, typename T>
__device__ __forceinline__ C to_c(T x) {
    return C(x);
}
template <typename T, typename C>
__device__ __forceinline__ T from_c(C x) {
    return (T)x;
}
// acc + x * y: contracted to one FMA in FP32 / FP64, the fused double-float
// multiply-add for dfloat
template <typename C>
__device__ __forceinline__ C madd(C acc, C x, C y) {
    return acc + x * y;
}
template <>
__device__ __forceinline__ dfloat madd<dfloat>(dfloat acc, dfloat x, dfloat y) {
    return df_fma(acc, x, y);
}

// Accumulator of a sum of products: a plain FMA chain in FP32 / FP64.  In
// double-float it is the compensated dot product Dot2 of Ogita, Rump and
// Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005): the
// leading products are summed by the error-free TwoSum into s, every
// rounding error (TwoSum's, the leading product's exact error from FMA, the
// cross terms with the operands' low parts) is summed in FP32 into t, and
// s + t is renormalised once when the value is read -- about 12 FP32
// instructions per term instead of 15, and one add on the loop-carried path
// instead of a full renormalisation.
template <typename C>
struct Acc {
    C v;
    __device__ __forceinline__ Acc() : v(C(0)) {}
    __device__ __forceinline__ void add(C c, C x) { v = madd(v, c, x); }
    __device__ __forceinline__ C get() const { return v; }
};
template <>
struct Acc<dfloat> {
    float s, t;
    __device__ __forceinline__ Acc() : s(0.f), t(0.f) {}
    __device__ __forceinline__ void add(dfloat c, dfloat x) {
        const float p = __fmul_rn(c.hi, x.hi);
        float e = __fmaf_rn(c.hi, x.hi, -p);
        e = __fmaf_rn(c.hi, x.lo, e);
        e = __fmaf_rn(c.lo, x.hi, e);
        const float s1 = __fadd_rn(s, p);
        const float bb = __fsub_rn(s1, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
        t = __fadd_rn(t, __fadd_rn(err, e));
        s = s1;
    }
    __device__ __forceinline__ dfloat get() const {
        const float hi = __fadd_rn(s, t);
        return dfloat(hi, __fsub_rn(t, __fsub_rn(hi, s)));
    }
};

// FP64 data in double-float arithmetic: split and widen without FP64-rate
// conversions (GB300 runs FP64 at 1/64 of the FP32 rate)
template <>
__device__ __forceinline__ dfloat to_c<dfloat, double>(double x) {
    return df_from_double(x);
}
template <>
__device__ __forceinline__ double from_c<double, dfloat>(dfloat x) {
    return df_to_double(x);
}

// Spatial tile of one CTA: TX x TY x TZ output points, ZS threads per (x, y)
// column (each owning TZ / ZS of its z points).  The double-float 3D tile is
// twice as deep with two threads per column: the x- and y-passes are redone
// on a z halo of 2p slices, which costs 1.5x instead of 2x over the outputs
// (68 instead of 83 multiply-adds per output and time plane at p = 2), with
// the same accumulators per thread.
template <int DIM, bool DF>
struct TileShape;
template <bool DF>
struct TileShape<1, DF> {
    static constexpr int TX = 128, TY = 1, TZ = 1, ZS = 1;
};
template <bool DF>
struct TileShape<2, DF> {
    static constexpr int TX = 32, TY = 16, TZ = 1, ZS = 1;
};
template <>
struct TileShape<3, false> {
    static constexpr int TX = 16, TY = 8, TZ = 4, ZS = 1;
};
template <>
struct TileShape<3, true> {
    static constexpr int TX = 8, TY = 8, TZ = 16, ZS = 4;
};

template <typename T, int P, int DIM>  // T: compute type
struct StencilSmem {
    using TS = TileShape<DIM, std::is_same<T, dfloat>::value>;
    static constexpr int TX = TS::TX, TY = TS::TY, TZ = TS::TZ, ZS = TS::ZS;
    static constexpr int TZL = TZ / ZS;  // z points per thread
    static constexpr int HX = P, HY = (DIM >= 2) ? P : 0, HZ = (DIM >= 3) ? P : 0;
    static constexpr int SX = TX + 2 * HX, SY = TY + 2 * HY, SZ = TZ + 2 * HZ;
    static constexpr int W = 2 * P + 1;
    static constexpr int nS = SZ * SY * SX;
    static constexpr int nA = SZ * SY * TX;
    static constexpr int nAA = SZ * TY * TX;
    static constexpr int nBand = 2 * W * (TX + TY + TZ);
    // the staged plane S and the y-pass results AA, SS are never live at the
    // same time (a barrier separates the z-pass reads from the next staging)
    static constexpr int nR1 = (nS > 2 * nAA) ? nS : 2 * nAA;
    static constexpr size_t bytes = sizeof(T) * (nR1 + 2 * nA + nBand);
    static constexpr int threads = TX * TY * ZS;
    // the deep tile (64 KB): three CTAs per SM (24 warps) where N_t <= 4 lets
    // the accumulators fit 80 registers, else two; the FP64 / FP32 2D tile
    // (512 threads): two CTAs per SM, at most 64 registers
    static constexpr int min_blocks(int ntc) {
        return ZS > 1 ? ((ntc > 0 && ntc <= 4) ? 3 : 2)
                      : (DIM == 2 && !std::is_same<T, dfloat>::value) ? 2 : 1;
    }
};

// NTC > 0: N_t fixed at compile time (exact-length loops, fewer registers
// for the N_t x TZ accumulators); NTC = 0: N_t from tc.nt, loops over NTMAX
template <typename T, typename C, int P, int DIM, int NTC = 0>
__global__ void __launch_bounds__(StencilSmem<C, P, DIM>::threads,
                                  StencilSmem<C, P, DIM>::min_blocks(NTC))
    k_stencil(const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ out, Bands<T> bands,
              Grid g, const __grid_constant__ TimeCoefs<C> tc, int slabs_per_prob, int slab0,
              int slab_end, int sch, int tiles_x, int tiles_y) {
    using SM = StencilSmem<C, P, DIM>;
    constexpr bool DF = std::is_same<C, dfloat>::value;
    constexpr int TX = SM::TX, TY = SM::TY, TZ = SM::TZ, TZL = SM::TZL;
    constexpr int HX = SM::HX, HY = SM::HY, HZ = SM::HZ;
    constexpr int SX = SM::SX, SY = SM::SY, SZ = SM::SZ, W = SM::W;
    constexpr int NTH = SM::threads;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);
    C *AA = S;
    C *SS = AA + SM::nAA;
    C *A = S + SM::nR1;
    C *B = A + SM::nA;
    C *bMx = B + SM::nA;
    C *bKx = bMx + TX * W;
    C *bMy = bKx + TX * W;
    C *bKy = bMy + TY * W;
    C *bMz = bKy + TY * W;
    C *bKz = bMz + TZ * W;

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int x0 = (tile % tiles_x) * TX;
    const int y0 = ((tile / tiles_x) % tiles_y) * TY;
    const int z0 = (tile / (tiles_x * tiles_y)) * TZ;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long nxyz = g.nxyz;
    constexpr int NL = NTC > 0 ? NTC : NTMAX;
    const int nt = NTC > 0 ? NTC : tc.nt;

    // stage the band rows of this tile (zero outside the grid)
    for (int e = tid; e < TX * W; e += NTH) {
        const int gx = x0 + e / W;
        bMx[e] = (gx < nx) ? to_c<C>(bands.M[0][(long long)gx * W + e % W]) : C(0);
        bKx[e] = (gx < nx) ? to_c<C>(bands.K[0][(long long)gx * W + e % W]) : C(0);
    }
    if (DIM >= 2)
        for (int e = tid; e < TY * W; e += NTH) {
            const int gy = y0 + e / W;
            bMy[e] = (gy < ny) ? to_c<C>(bands.M[1][(long long)gy * W + e % W]) : C(0);
            bKy[e] = (gy < ny) ? to_c<C>(bands.K[1][(long long)gy * W + e % W]) : C(0);
        }
    if (DIM >= 3)
        for (int e = tid; e < TZ * W; e += NTH) {
            const int gz = z0 + e / W;
            bMz[e] = (gz < nz) ? to_c<C>(bands.M[2][(long long)gz * W + e % W]) : C(0);
            bKz[e] = (gz < nz) ? to_c<C>(bands.K[2][(long long)gz * W + e % W]) : C(0);
        }

    const int tx = tid % TX, ty = (tid / TX) % TY;
    const int za = (tid / (TX * TY)) * TZL;  // this thread's first z point in the tile
    C mprev[TZL];
#pragma unroll
    for (int a = 0; a < TZL; ++a) mprev[a] = C(0);

    // one slab per CTA (a single trip, known to the compiler) unless double-float
    const int sbeg = slab0 + (int)blockIdx.y * (DF ? sch : 1);
    const int send = DF ? min(sbeg + sch, slab_end) : sbeg + 1;
    for (int slab = sbeg; slab < send; ++slab) {
        Acc<C> acc[TZL][NL];
        const T *uslab = u + (long long)slab * nt * nxyz;
        const bool first = (slab % slabs_per_prob) == 0;
        const bool has_prev = (tc.mode != MODE_MASS) && (!first || tc.halo != nullptr);
        // double-float, not the CTA's first slab: M_x u of the coupling plane is
        // the previous slab's last time plane, kept from that slab's z-pass
        const bool carried = DF && has_prev && !first && slab > sbeg;
        if (carried) {
#pragma unroll
            for (int al = 0; al < TZL; ++al) acc[al][0].add(C(-1), mprev[al]);
        }
        // the coupling plane: the previous slab's last time plane, or for the
        // first slab of a partition the neighbour's plane in the halo buffer
        const T *prev = !first ? uslab - nxyz
                        : tc.halo ? static_cast<const T *>(tc.halo) + (long long)(slab / slabs_per_prob) * nxyz
                                  : nullptr;

        for (int jj = (has_prev && !carried) ? -1 : 0; jj < nt; ++jj) {
            const T *plane = (jj < 0) ? prev : uslab + (long long)jj * nxyz;
            __syncthreads();
            for (int e = tid; e < SZ * SY * SX; e += NTH) {
                const int sx = e % SX, sy = (e / SX) % SY, sz = e / (SX * SY);
                const int gx = x0 + sx - HX, gy = y0 + sy - HY, gz = z0 + sz - HZ;
                C v = C(0);
                if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
                    v = to_c<C>(plane[((long long)gz * ny + gy) * nx + gx]);
                S[e] = v;
            }
            __syncthreads();
            // x-pass: A = M1x u, B = K1x u (the coupling plane needs only M_x u)
            const bool mass_only = jj < 0;
            for (int e = tid; e < SZ * SY * TX; e += NTH) {
                const int ex = e % TX, row = e / TX;  // row = sz*SY + sy
                const C *srow = S + row * SX + ex;
                Acc<C> a, b;
                if (mass_only) {
#pragma unroll
                    for (int o = 0; o < W; ++o) a.add(bMx[ex * W + o], srow[o]);
                } else {
#pragma unroll
                    for (int o = 0; o < W; ++o) {
                        const C sv = srow[o];
                        a.add(bMx[ex * W + o], sv);
                        b.add(bKx[ex * W + o], sv);
                    }
                }
                A[e] = a.get();
                B[e] = b.get();
            }
            __syncthreads();
            const C *pm;
            const C *pk;
            if (DIM >= 2) {
                // y-pass: AA = M1y A, SS = K1y A + M1y B
                for (int e = tid; e < SZ * TY * TX; e += NTH) {
                    const int ex = e % TX, ey = (e / TX) % TY, sz = e / (TX * TY);
                    Acc<C> aa, ss;
                    if (mass_only) {
#pragma unroll
                        for (int o = 0; o < W; ++o)
                            aa.add(bMy[ey * W + o], A[(sz * SY + ey + o) * TX + ex]);
                    } else {
#pragma unroll
                        for (int o = 0; o < W; ++o) {
                            const int idx = (sz * SY + ey + o) * TX + ex;
                            const C av = A[idx], bv = B[idx];
                            const C my = bMy[ey * W + o], ky = bKy[ey * W + o];
                            aa.add(my, av);
                            ss.add(ky, av);
                            ss.add(my, bv);
                        }
                    }
                    AA[e] = aa.get();
                    SS[e] = ss.get();
                }
                __syncthreads();
                pm = AA;
                pk = SS;
            } else {
                pm = A;
                pk = B;
            }
            // z-pass and accumulation into this thread's output points
#pragma unroll
            for (int al = 0; al < TZL; ++al) {
                const int a = za + al;
                C m, k;
                if (DIM >= 3) {
                    Acc<C> am, ak;
#pragma unroll
                    for (int o = 0; o < W; ++o) {
                        const int idx = ((a + o) * TY + ty) * TX + tx;
                        const C mz = bMz[a * W + o], kz = bKz[a * W + o];
                        am.add(mz, pm[idx]);
                        ak.add(kz, pm[idx]);
                        ak.add(mz, pk[idx]);
                    }
                    m = am.get();
                    k = ak.get();
                } else {
                    m = pm[ty * TX + tx];
                    k = pk[ty * TX + tx];
                }
                if (jj < 0) {
                    if constexpr (DF)
                        acc[al][0].add(C(-1), m);
                    else
                        mprev[al] = m;
                } else {
#pragma unroll
                    for (int i = 0; i < NL; ++i)
                        if (i < nt) {
                            acc[al][i].add(tc.CK[i * NTMAX + jj], m);
                            acc[al][i].add(tc.CM[i * NTMAX + jj], k);
                        }
                    if (DF && jj == nt - 1) mprev[al] = m;  // the next slab's coupling plane
                }
            }
        }

        // epilogue (no barrier below: threads outside the grid skip it)
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < nx && gy < ny) {
#pragma unroll
            for (int al = 0; al < TZL; ++al) {
                const int a = al;  // accumulator index; the z point is za + al
                const int gz = z0 + za + al;
                if (gz >= nz) break;
                const long long sp = ((long long)gz * ny + gy) * nx + gx;
                const long long base = (long long)slab * nt * nxyz + sp;
                C r[NL];
#pragma unroll
                for (int i = 0; i < NL; ++i) {
                    if (i >= nt) {
                        r[i] = C(0);
                        continue;
                    }
                    C v = acc[a][i].get();
                    if (tc.mode == MODE_RES) {
                        v = to_c<C>(f[base + (long long)i * nxyz]) - v;
                        if (!DF && i == 0) v += mprev[a];
                    } else if (tc.mode == MODE_APPLY) {
                        if (!DF && i == 0) v -= mprev[a];
                    }
                    r[i] = v;
                }
                if (tc.fuse_y) {
#pragma unroll
                    for (int i = 0; i < NL; ++i) {
                        if (i >= nt) break;
                        C w = C(0);
#pragma unroll
                        for (int j = 0; j < NL; ++j)
                            if (j < nt) w = madd(w, tc.Y[i * NTMAX + j], r[j]);
                        out[base + (long long)i * nxyz] = from_c<T>(w);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < NL; ++i)
                        if (i < nt) out[base + (long long)i * nxyz] = from_c<T>(r[i]);
                }
            }
        }
    }
}

template <typename T, typename C, int P, int DIM, int NTC = 0>
static cudaError_t launch_stencil_t(const T *u, const T *f, T *out, const Bands<T> &bands,
                                    const Grid &g, const TimeCoefs<C> &tc, int slabs_per_prob,
                                    int slab0, int nslabs, cudaStream_t s, int sch_req) {
    using SM = StencilSmem<C, P, DIM>;
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e =
            smem_attr_once((const void *)k_stencil<T, C, P, DIM, NTC>, (int)SM::bytes, attr);
        if (e != cudaSuccess) return e;
    }
    const int tx = (g.nx + SM::TX - 1) / SM::TX;
    const int ty = (g.ny + SM::TY - 1) / SM::TY;
    const int tz = (g.nz + SM::TZ - 1) / SM::TZ;
    if (nslabs <= 0) return cudaSuccess;
    // double-float: up to 8 slabs per CTA while at least 8192 CTAs remain
    // (many waves of the GPU's resident CTAs), or the count asked for;
    // FP64 / FP32: one
    int sch = 1;
    if constexpr (std::is_same<C, dfloat>::value) {
        if (sch_req > 0) {
            sch = sch_req;
        } else {
            const long long tiles = (long long)tx * ty * tz;
            while (sch < 8 && tiles * ((nslabs + 2 * sch - 1) / (2 * sch)) >= 8192) sch *= 2;
        }
    }
    const int gy = (nslabs + sch - 1) / sch;
    if (gy > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)(tx * ty * tz), (unsigned)gy);
    k_stencil<T, C, P, DIM, NTC><<<grid, SM::threads, SM::bytes, s>>>(
        u, f, out, bands, g, tc, slabs_per_prob, slab0, slab0 + nslabs, sch, tx, ty);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// z-marching variant (3D): a CTA owns a 16 x 8 column of (x, y) points of one
// slab and walks its z range slice by slice.  For every slice and time plane
// the slice (plus its x / y halo) is staged, the x-pass and the y-pass run
// once, and each thread keeps the y-pass results of its own point for the
// last 2p + 1 slices in a private ring in shared memory; when a slice
// completes the window of an output slice, the thread runs the z-pass and
// the time combination for that point and writes it.  Compared with the
// tiled kernel, no x- or y-pass work is repeated on a z halo.  Each thread
// reads and writes only its own ring entries, so the ring needs no barrier.
// Used for the double-float residual at p = 3 (48^3, p = 3: 59 -> 47 ms per
// solve); at p = 2 the ring's shared memory lowers the occupancy more than
// the saved halo work gains (114 -> 118 ms), so the tiled kernel stays.
// ---------------------------------------------------------------------------
template <typename C, int P, int NT>
struct ZmSmem {
    static constexpr int TX = 16, TY = 8, W = 2 * P + 1;
    static constexpr int SX = TX + 2 * P, SY = TY + 2 * P;
    static constexpr int threads = TX * TY;
    // S, A, B, x / y bands, ring (NT + 1 planes x W slices x {AA, SS} x threads)
    static constexpr int nfix = SY * SX + 2 * SY * TX + 2 * W * (TX + TY) +
                                (NT + 1) * W * 2 * threads;
    static size_t bytes(int zc) { return sizeof(C) * ((size_t)nfix + 2 * (size_t)zc * W); }
};

template <typename T, typename C, int P, int NT>
__global__ void __launch_bounds__(128)
    k_stencil_zm(const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ out,
                 Bands<T> bands, Grid g, const __grid_constant__ TimeCoefs<C> tc,
                 int slabs_per_prob, int slab0, int tiles_x, int zc_len) {
    using SM = ZmSmem<C, P, NT>;
    constexpr int TX = SM::TX, TY = SM::TY, W = SM::W, SX = SM::SX, SY = SM::SY;
    constexpr int NTH = SM::threads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);
    C *A = S + SY * SX;
    C *B = A + SY * TX;
    C *bMx = B + SY * TX;
    C *bKx = bMx + TX * W;
    C *bMy = bKx + TX * W;
    C *bKy = bMy + TY * W;
    C *ring = bKy + TY * W;                          // [NT + 1][W][2][NTH]
    C *bMz = ring + (NT + 1) * W * 2 * NTH;           // [zc_len][W]
    C *bKz = bMz + zc_len * W;

    const int tid = threadIdx.x;
    const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
    const int slab = slab0 + blockIdx.y;
    const int zb = blockIdx.z * zc_len;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int ze = (zb + zc_len < nz) ? zb + zc_len : nz;
    const long long nxyz = g.nxyz;

    for (int e = tid; e < TX * W; e += NTH) {
        const int gx = x0 + e / W;
        bMx[e] = (gx < nx) ? to_c<C>(bands.M[0][(long long)gx * W + e % W]) : C(0);
        bKx[e] = (gx < nx) ? to_c<C>(bands.K[0][(long long)gx * W + e % W]) : C(0);
    }
    for (int e = tid; e < TY * W; e += NTH) {
        const int gy = y0 + e / W;
        bMy[e] = (gy < ny) ? to_c<C>(bands.M[1][(long long)gy * W + e % W]) : C(0);
        bKy[e] = (gy < ny) ? to_c<C>(bands.K[1][(long long)gy * W + e % W]) : C(0);
    }
    for (int e = tid; e < (ze - zb) * W; e += NTH) {
        const long long gz = zb + e / W;
        bMz[e] = to_c<C>(bands.M[2][gz * W + e % W]);
        bKz[e] = to_c<C>(bands.K[2][gz * W + e % W]);
    }

    const int tx = tid % TX, ty = tid / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    const T *uslab = u + (long long)slab * NT * nxyz;
    const bool first = (slab % slabs_per_prob) == 0;
    const bool has_prev = (tc.mode != MODE_MASS) && (!first || tc.halo != nullptr);
    const T *prev = !first ? uslab - nxyz
                    : tc.halo ? static_cast<const T *>(tc.halo) + (long long)(slab / slabs_per_prob) * nxyz
                              : nullptr;
    const int j0 = has_prev ? -1 : 0;

    for (int zs = zb - P; zs < ze + P; ++zs) {
        const int slot = (zs - zb + P) % W;
        const bool zin = zs >= 0 && zs < nz;
        for (int jj = j0; jj < NT; ++jj) {
            const T *plane = (jj < 0) ? prev : uslab + (long long)jj * nxyz;
            // S is free (the previous x-pass is behind the last barrier)
            for (int e = tid; e < SY * SX; e += NTH) {
                const int sx = e % SX, sy = e / SX;
                const int ggx = x0 + sx - P, ggy = y0 + sy - P;
                C v = C(0);
                if (zin && ggx >= 0 && ggx < nx && ggy >= 0 && ggy < ny)
                    v = to_c<C>(plane[((long long)zs * ny + ggy) * nx + ggx]);
                S[e] = v;
            }
            __syncthreads();  // S staged; the previous y-pass is done with A, B
            const bool mass_only = jj < 0;
            for (int e = tid; e < SY * TX; e += NTH) {
                const int ex = e % TX, row = e / TX;
                const C *srow = S + row * SX + ex;
                Acc<C> a, b;
                if (mass_only) {
#pragma unroll
                    for (int o = 0; o < W; ++o) a.add(bMx[ex * W + o], srow[o]);
                } else {
#pragma unroll
                    for (int o = 0; o < W; ++o) {
                        const C sv = srow[o];
                        a.add(bMx[ex * W + o], sv);
                        b.add(bKx[ex * W + o], sv);
                    }
                }
                A[e] = a.get();
                B[e] = b.get();
            }
            __syncthreads();  // A, B complete
            {
                Acc<C> aa, ss;
                if (mass_only) {
#pragma unroll
                    for (int o = 0; o < W; ++o) aa.add(bMy[ty * W + o], A[(ty + o) * TX + tx]);
                } else {
#pragma unroll
                    for (int o = 0; o < W; ++o) {
                        const int idx = (ty + o) * TX + tx;
                        const C av = A[idx], bv = B[idx];
                        const C my = bMy[ty * W + o], ky = bKy[ty * W + o];
                        aa.add(my, av);
                        ss.add(ky, av);
                        ss.add(my, bv);
                    }
                }
                C *rp = ring + ((size_t)((jj + 1) * W + slot) * 2) * NTH + tid;
                rp[0] = aa.get();
                rp[NTH] = ss.get();
            }
        }
        // output slice zc = zs - P: its window zc - P .. zc + P is in the ring
        const int zc = zs - P;
        if (zc < zb || zc >= ze) continue;
        const int zr = zc - zb;
        Acc<C> acc[NT];
        C mprev = C(0);
        for (int jj = j0; jj < NT; ++jj) {
            Acc<C> am, ak;
#pragma unroll
            for (int o = 0; o < W; ++o) {
                const int sl = (zc - P + o - zb + P) % W;  // slot of slice zc - P + o
                const C *rp = ring + ((size_t)((jj + 1) * W + sl) * 2) * NTH + tid;
                const C mz = bMz[zr * W + o], kz = bKz[zr * W + o];
                am.add(mz, rp[0]);
                if (jj >= 0) {
                    ak.add(kz, rp[0]);
                    ak.add(mz, rp[NTH]);
                }
            }
            const C m = am.get();
            if (jj < 0) {
                mprev = m;
                continue;
            }
            const C k = ak.get();
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                acc[i].add(tc.CK[i * NTMAX + jj], m);
                acc[i].add(tc.CM[i * NTMAX + jj], k);
            }
        }
        if (gx >= nx || gy >= ny) continue;
        const long long base = (long long)slab * NT * nxyz + ((long long)zc * ny + gy) * nx + gx;
        C r[NT];
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            C v = acc[i].get();
            if (tc.mode == MODE_RES) {
                v = to_c<C>(f[base + (long long)i * nxyz]) - v;
                if (i == 0) v += mprev;
            } else if (tc.mode == MODE_APPLY) {
                if (i == 0) v -= mprev;
            }
            r[i] = v;
        }
        if (tc.fuse_y) {
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                C w = C(0);
#pragma unroll
                for (int j = 0; j < NT; ++j) w = madd(w, tc.Y[i * NTMAX + j], r[j]);
                out[base + (long long)i * nxyz] = from_c<T>(w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NT; ++i) out[base + (long long)i * nxyz] = from_c<T>(r[i]);
        }
    }
}

// cudaErrorNotSupported when the shared memory does not fit (the tiled
// kernel is used then)
template <typename T, typename C, int P, int NT>
static cudaError_t launch_stencil_zm_t(const T *u, const T *f, T *out, const Bands<T> &bands,
                                       const Grid &g, const TimeCoefs<C> &tc, int slabs_per_prob,
                                       int slab0, int nslabs, cudaStream_t s) {
    using SM = ZmSmem<C, P, NT>;
    if (nslabs <= 0) return cudaSuccess;
    if (nslabs > 65535) return cudaErrorInvalidValue;
    const int zc = g.nz <= 64 ? g.nz : 32;  // z slices per CTA
    const size_t bytes = SM::bytes(zc);
    if (bytes > 200 * 1024) return cudaErrorNotSupported;
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e =
            smem_attr_once((const void *)k_stencil_zm<T, C, P, NT>, (int)(200 * 1024), attr);
        if (e != cudaSuccess) return e;
    }
    const int tx = (g.nx + SM::TX - 1) / SM::TX;
    const int ty = (g.ny + SM::TY - 1) / SM::TY;
    dim3 grid((unsigned)(tx * ty), (unsigned)nslabs, (unsigned)((g.nz + zc - 1) / zc));
    k_stencil_zm<T, C, P, NT><<<grid, SM::threads, bytes, s>>>(u, f, out, bands, g, tc,
                                                               slabs_per_prob, slab0, tx, zc);
    return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t launch_stencil(const T *u, const T *f, T *out, const Bands<T> &bands, const Grid &g,
                           const TimeCoefs<C> &tc, int slabs_per_prob, int slab0, int nslabs,
                           cudaStream_t s, int sch) {
    if (sch < 0 || sch > 8 || (sch & (sch - 1)) != 0) return cudaErrorInvalidValue;
#define ST_NT(PP, DD, N)                                                                        \
    if (tc.nt == N) {                                                                           \
        if constexpr (DD == 3 && PP >= 3) {                                                     \
            const cudaError_t ez = launch_stencil_zm_t<T, C, PP, N>(                            \
                u, f, out, bands, g, tc, slabs_per_prob, slab0, nslabs, s);                     \
            if (ez != cudaErrorNotSupported) return ez;                                         \
        }                                                                                       \
        return launch_stencil_t<T, C, PP, DD, N>(u, f, out, bands, g, tc, slabs_per_prob, slab0, \
                                                 nslabs, s, sch);                               \
    }
#define ST_CASE(PP, DD)                                                                         \
    if (g.p == PP && g.dim == DD) {                                                             \
        if constexpr (std::is_same<C, dfloat>::value) {                                         \
            ST_NT(PP, DD, 3) ST_NT(PP, DD, 4) ST_NT(PP, DD, 5) ST_NT(PP, DD, 6)                  \
        }                                                                                       \
        return launch_stencil_t<T, C, PP, DD>(u, f, out, bands, g, tc, slabs_per_prob, slab0,   \
                                              nslabs, s, sch);                                  \
    }
    ST_CASE(1, 1)
    ST_CASE(2, 1)
    ST_CASE(3, 1)
    ST_CASE(1, 2)
    ST_CASE(2, 2)
    ST_CASE(3, 2)
    ST_CASE(1, 3)
    ST_CASE(2, 3)
    ST_CASE(3, 3)
#undef ST_CASE
#undef ST_NT
    return cudaErrorInvalidValue;
}

}  // namespace st

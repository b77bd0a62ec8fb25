// Spatial fast-diagonalisation transforms on the 5th-generation tensor cores
// (tcgen05, sm_100 family): one axis of out[..k..] = sum_i W[i][k] in[..i..]
// (W = U for the forward transform U^T, W = U^T for the inverse), the dense
// contraction inside A^{-1} = (X (x) U)(Z (x) I + I (x) Lambda)^{-1}(Y (x) U^T)
// (Eq. 3.1 of arXiv:1802.09277 with fast diagonalisation in space).
//
// FP32 data in HBM; operands rounded to TF32 (cvt.rna) or BF16 while they are
// staged into shared memory; FP32 accumulation in tensor memory.  KIND_TF32X3
// splits each operand x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and
// accumulates hi*hi + hi*lo + lo*hi: three TF32 MMAs per K step for a product
// as accurate as FP32 arithmetic (the lo*lo term is below FP32 rounding).
//
// MODE_X (contracted axis contiguous):  D[k][c] = sum_i Wt[k][i] In[c][i]
//     A = Wt (128 rows = output modes, n_out <= 128), B = 128 input rows
//     c, D in TMEM with lane = k: out[c][k] is written by consecutive lanes.
// MODE_S (contracted axis strided by `inner`): D[c][k] = sum_i In_c[i] Wt[k][i]
//     A = 128 columns c = (outer, inner index), B = Wt (N = n_out padded to
//     16, <= 256), lane = c: out[o][k][ci] is written by consecutive lanes.
//
// One CTA (128 threads) loops over 128-column tiles: all threads stage the
// activation tile, thread 0 issues the MMAs and commits them to an
// mbarrier, all threads wait (bounded) and drain TMEM with tcgen05.ld.
// A wait that runs out is decided for the whole CTA at once (a CTA-wide
// vote, so every thread takes the same barriers): the CTA records the error,
// waits (bounded again) for its MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>
#include <mutex>

#include "st_internal.h"
#include "tc_sm100.cuh"

namespace st {

namespace {

constexpr int TC_THREADS = 256;  // 8 warps: warps w and w + 4 share TMEM lane quarter w % 4
constexpr int TC_COLS = 128;  // columns (GEMM rows of the activation operand) per tile
static_assert(TC_THREADS % TC_COLS == 0, "a thread stages one column of every tile");
constexpr uint64_t TC_DRAIN_NS = 1000000000ull;  // after a timeout: MMAs in flight finish
constexpr int KIND_TF32X3 = 3;  // split TF32 (see above); MMA format TF32

template <int KIND>
struct KindTraits {
    static constexpr int FMT = (KIND == KIND_TF32X3) ? tc::FMT_TF32 : KIND;
    static constexpr int ESZ = (FMT == tc::FMT_TF32) ? 4 : 2;  // bytes per element
    static constexpr int NSPLIT = (KIND == KIND_TF32X3) ? 2 : 1;
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Store 16 bytes of operand data for row r, 16-byte chunk kc of a K-major tile
// with R rows.  TF32: 4 values; BF16: 8 values; split TF32: 4 hi values in
// `tile` and 4 lo values at the same offset in `tile + lo_off`.
template <int KIND>
__device__ __forceinline__ void stage16(unsigned char *tile, int R, int r, int kc, const float *v,
                                        size_t lo_off = 0) {
    uint4 q;
    if (KIND == KIND_TF32X3) {
        uint4 l;
        q.x = to_tf32(v[0]);
        q.y = to_tf32(v[1]);
        q.z = to_tf32(v[2]);
        q.w = to_tf32(v[3]);
        l.x = to_tf32(v[0] - __uint_as_float(q.x));
        l.y = to_tf32(v[1] - __uint_as_float(q.y));
        l.z = to_tf32(v[2] - __uint_as_float(q.z));
        l.w = to_tf32(v[3] - __uint_as_float(q.w));
        const uint32_t off = tc::kmajor_offset(R, r, kc * 16);
        *reinterpret_cast<uint4 *>(tile + off) = q;
        *reinterpret_cast<uint4 *>(tile + lo_off + off) = l;
        return;
    }
    if (KIND == tc::FMT_TF32) {
        q.x = to_tf32(v[0]);
        q.y = to_tf32(v[1]);
        q.z = to_tf32(v[2]);
        q.w = to_tf32(v[3]);
    } else {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 c = __floats2bfloat162_rn(v[4], v[5]);
        __nv_bfloat162 d = __floats2bfloat162_rn(v[6], v[7]);
        q.x = *reinterpret_cast<uint32_t *>(&a);
        q.y = *reinterpret_cast<uint32_t *>(&b);
        q.z = *reinterpret_cast<uint32_t *>(&c);
        q.w = *reinterpret_cast<uint32_t *>(&d);
    }
    *reinterpret_cast<uint4 *>(tile + tc::kmajor_offset(R, r, kc * 16)) = q;
}

}  // namespace

struct TcArgs {
    const float *in;
    float *out;
    const float *wt;   // Wt[k][i] row-major, n_out x n_in (FP32)
    int n_in, n_out;   // contracted / produced axis length
    int k_pad;         // n_in padded to the MMA K step
    int n_pad;         // MODE_S: n_out padded to 16
    int kch;           // 16-byte K chunks staged at a time (even; = all of K when it fits)
    int mh;            // MODE_X: 128-row halves of the output modes (1 or 2)
    int vec4;          // MODE_X: rows start on 16-byte boundaries (n_in % 4 == 0, aligned in)
    long long ncols;   // number of GEMM columns (input rows / (outer, inner) pairs)
    long long inner;   // MODE_S: stride of the contracted axis
    int *err;          // set to 1 if an mbarrier wait ran out
    unsigned long long wait_ns;  // bound of each wait for the MMAs (0: test once)
    int w_tma;         // pipelined kernel: the weight operand arrives by TMA (tensor map)
};

// A strided-axis column c = (outer o, inner index ci): src = in + o n_in inner + ci.
// One division per column (32-bit when the operands fit), not per chunk.
__device__ __forceinline__ const float *col_src(const TcArgs &a, long long c) {
    long long o, ci;
    if (c < 0x7fffffffLL && a.inner < 0x7fffffffLL) {
        const unsigned q = (unsigned)c / (unsigned)a.inner;
        o = q;
        ci = c - (long long)q * a.inner;
    } else {
        o = c / a.inner;
        ci = c - o * a.inner;
    }
    return a.in + o * a.n_in * a.inner + ci;
}

// Stage 16-byte chunks [k0, k0 + kcs) of the weight operand (rows = output
// modes, zero padded) as a K-major tile of wrows rows.
template <int KIND>
__device__ __forceinline__ void stage_w(const TcArgs &a, unsigned char *wtile, int wrows, int k0,
                                        int kcs, size_t lo_off) {
    constexpr int EPC = 16 / KindTraits<KIND>::ESZ;
    // consecutive lanes take consecutive rows: their 16-byte stores are
    // contiguous in the core-matrix layout (no shared-memory bank conflicts)
    for (int t = threadIdx.x; t < wrows * kcs; t += TC_THREADS) {
        const int kc = t / wrows, r = t % wrows;
        float v[8];
#pragma unroll
        for (int j = 0; j < EPC; ++j) {
            const int i = (k0 + kc) * EPC + j;
            v[j] = (r < a.n_out && i < a.n_in) ? a.wt[(long long)r * a.n_in + i] : 0.f;
        }
        stage16<KIND>(wtile, wrows, r, kc, v, lo_off);
    }
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_tc_axis(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    using KT = KindTraits<KIND>;
    constexpr int EPC = 16 / KT::ESZ;  // elements per 16-byte chunk
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KC = a.k_pad / EPC;  // 16-byte chunks per operand row
    const int kch = a.kch;         // chunks staged at a time
    const int nchunk = (KC + kch - 1) / kch;
    const int mh = (MODE == 0) ? a.mh : 1;
    const int wrows = (MODE == 0) ? 128 * mh : a.n_pad;
    // [W hi | W lo] [X hi | X lo] (lo parts only for the split kind), kch chunks each
    const size_t wbytes = (size_t)wrows * kch * 16, xbytes = (size_t)TC_COLS * kch * 16;
    unsigned char *wtile = smem;
    unsigned char *xtile = smem + KT::NSPLIT * wbytes;
    const uint32_t tmem_cols = (MODE == 0) ? (uint32_t)(TC_COLS * mh)
                                           : (a.n_pad <= 32 ? 32u : a.n_pad <= 64 ? 64u
                                              : a.n_pad <= 128 ? 128u : 256u);

    // the whole weight operand fits: staged once for all column tiles
    if (nchunk == 1) stage_w<KIND>(a, wtile, wrows, 0, KC, wbytes);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc(&tmem_base, tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = (MODE == 0) ? tc::make_idesc(KT::FMT, 128, TC_COLS)
                                       : tc::make_idesc(KT::FMT, 128, a.n_pad);
    const long long ntiles = (a.ncols + TC_COLS - 1) / TC_COLS;
    uint32_t phase = 0;
    bool failed = false;

    for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const long long c0 = tile * TC_COLS;
        for (int ch = 0; ch < nchunk && !failed; ++ch) {
            const int k0 = ch * kch;
            const int kcs = (KC - k0 < kch) ? KC - k0 : kch;  // even: KC and kch are
            if (nchunk > 1) stage_w<KIND>(a, wtile, wrows, k0, kcs, wbytes);
            // ---- stage the activation chunk: 128 rows (columns c) x kcs ----
            if (MODE == 0) {
                // lanes: 8 consecutive rows x 4 consecutive 16-byte chunks
                for (int t = tid; t < TC_COLS * kcs; t += TC_THREADS) {
                    const int grp = t / (8 * kcs), rem = t % (8 * kcs);
                    const int kc = rem / 8, r = grp * 8 + rem % 8;
                    const long long c = c0 + r;
                    float v[8];
                    const int i0 = (k0 + kc) * EPC;
                    if (a.vec4 && c < a.ncols && i0 + EPC <= a.n_in) {
                        // whole 16-byte groups of the row: vector loads
#pragma unroll
                        for (int j = 0; j < EPC; j += 4) {
                            const float4 q = *reinterpret_cast<const float4 *>(a.in + c * a.n_in + i0 + j);
                            v[j] = q.x;
                            v[j + 1] = q.y;
                            v[j + 2] = q.z;
                            v[j + 3] = q.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < EPC; ++j) {
                            const int i = i0 + j;
                            v[j] = (c < a.ncols && i < a.n_in) ? a.in[c * a.n_in + i] : 0.f;
                        }
                    }
                    stage16<KIND>(xtile, TC_COLS, r, kc, v, xbytes);
                }
            } else {
                // lanes: consecutive columns (consecutive inner index), same chunk;
                // a thread's column is the same for all its chunks
                const int r = tid % TC_COLS;
                const long long c = c0 + r;
                const float *src = col_src(a, c);
                for (int t = tid; t < TC_COLS * kcs; t += TC_THREADS) {
                    const int kc = t / TC_COLS;
                    float v[8];
#pragma unroll
                    for (int j = 0; j < EPC; ++j) {
                        const int i = (k0 + kc) * EPC + j;
                        v[j] = (c < a.ncols && i < a.n_in) ? src[(long long)i * a.inner] : 0.f;
                    }
                    stage16<KIND>(xtile, TC_COLS, r, kc, v, xbytes);
                }
            }
            tc::fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            // ---- MMAs over the chunk: K in 32-byte steps ----
            if (tid == 0) {
                const uint32_t wa = tc::smem_u32(wtile), xa = tc::smem_u32(xtile);
                const uint32_t lbo_w = (uint32_t)wrows * 16, lbo_x = TC_COLS * 16;
                const int steps = kcs / 2;
                // split kind: (hi, hi), (hi, lo), (lo, hi) per K step
                constexpr int NPROD = (KT::NSPLIT == 2) ? 3 : 1;
                for (int s = 0; s < steps; ++s) {
#pragma unroll
                    for (int q = 0; q < NPROD; ++q) {
                        const uint32_t wo = (q == 2) ? (uint32_t)wbytes : 0u;
                        const uint32_t xo = (q == 1) ? (uint32_t)xbytes : 0u;
                        const uint64_t dx = tc::make_sdesc(xa + xo + 2 * s * lbo_x, lbo_x, 128);
                        const uint32_t acc = (ch > 0 || s > 0 || q > 0) ? 1u : 0u;
                        if (MODE == 0) {
                            // output modes 128h .. 128h + 127: rows 128h.. of the weight
                            // tile (16 core-matrix groups of 128 bytes further), TMEM
                            // columns 128h ..
                            for (int h = 0; h < mh; ++h) {
                                const uint64_t dw = tc::make_sdesc(
                                    wa + wo + 2 * s * lbo_w + (uint32_t)h * 2048u, lbo_w, 128);
                                tc::mma<KT::FMT>(tmem + (uint32_t)(h * TC_COLS), dw, dx, idesc, acc);
                            }
                        } else {
                            const uint64_t dw = tc::make_sdesc(wa + wo + 2 * s * lbo_w, lbo_w, 128);
                            tc::mma<KT::FMT>(tmem, dx, dw, idesc, acc);
                        }
                    }
                }
                tc::commit(&mbar);
            }
            // the MMAs have read the chunk before it is overwritten or the
            // accumulator is read
            const bool ok = tc::mbar_wait_bounded(&mbar, phase, a.wait_ns);
            if (__syncthreads_or(ok ? 0 : 1)) {
                // the MMAs still in flight complete before TMEM is released
                tc::mbar_wait_bounded(&mbar, phase, TC_DRAIN_NS);
                failed = true;
                if (tid == 0) atomicExch(a.err, 1);
            }
            phase ^= 1u;
            tc::fence_after_sync();
        }
        if (!failed) {
            // ---- epilogue: TMEM -> registers -> global ----
            // warp w reads TMEM lanes 32 (w % 4) ..; warps w and w + 4 split the columns
            const int wq = warp & 3, wh = warp >> 2;
            const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
            if (MODE == 0) {
                for (int h = 0; h < mh; ++h) {
                    const int k = 128 * h + 32 * wq + lane;  // output mode of this lane
                    if (128 * h + 32 * wq >= a.n_out) continue;
                    for (int cc = wh * (TC_COLS / 2); cc < (wh + 1) * (TC_COLS / 2); cc += 16) {
                        float v[16];
                        tc::tmem_ld16(tmem + lane_base + (uint32_t)(h * TC_COLS + cc), v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const long long c = c0 + cc + j;
                            if (k < a.n_out && c < a.ncols) a.out[c * a.n_out + k] = v[j];
                        }
                    }
                }
            } else {
                const long long c = c0 + 32 * wq + lane;  // column of this lane
                const long long o = c / a.inner, ci = c % a.inner;
                float *dst = a.out + o * a.n_out * a.inner + ci;
                const int nk = a.n_pad / 16;  // 16-column groups, split between the warp pair
                for (int kk = 16 * ((nk * wh) / 2); kk < 16 * ((nk * (wh + 1)) / 2); kk += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + lane_base + kk, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int k = kk + j;
                        if (k < a.n_out && c < a.ncols) dst[(long long)k * a.inner] = v[j];
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

constexpr size_t TC_SMEM_MAX = 200 * 1024;

// ---------------------------------------------------------------------------
// Pipelined variant: each CTA keeps two tensor-memory accumulators and the
// next column tile in registers, so that the MMAs of tile k, the global loads
// of tile k + 1 and the epilogue of tile k - 1 overlap:
//     wait MMA(k-1) -> convert tile k into shared memory -> issue MMA(k)
//     -> load tile k+1 into registers -> drain accumulator of tile k-1.
// The weight operand is staged once per CTA: a 2D TMA copy of the raw FP32
// W^T (box n_pad x k_pad, zero-filled outside n_out x n_in) into the
// activation area, converted there into the MMA layout.  Covers shapes whose
// whole K fits in shared memory and whose tile fits the register prefetch
// (K <= 80 for TF32 / split TF32, <= 96 for BF16); others use k_tc_axis.
// The contiguous axis runs as MODE_XT: the activation tile (128 input rows)
// is the 128-row operand and W the N = n_pad one, D[c][k] with lane = c, so
// no MMA rows are spent on absent output modes (k_tc_axis's MODE_X makes W
// the 128-row operand); each lane then writes its row out[c][0 .. n_out).
// ---------------------------------------------------------------------------
template <int EPC>
struct PipeTraits {
    static constexpr int PF = (EPC == 4) ? 10 : 6;  // 16-byte chunks per thread in flight
};

// Global -> registers: the 16-byte chunks of column tile c0 this thread
// stages (the same mapping as k_tc_axis's staging loops).
template <int KIND, int MODE>
__device__ __forceinline__ void pipe_load(const TcArgs &a, long long c0, int KC,
                                          float (&pre)[PipeTraits<16 / KindTraits<KIND>::ESZ>::PF]
                                                      [16 / KindTraits<KIND>::ESZ]) {
    constexpr int EPC = 16 / KindTraits<KIND>::ESZ;
    constexpr int PF = PipeTraits<EPC>::PF;
    // MODE_S: a thread's column is the same for all its chunks
    const long long cs = c0 + threadIdx.x % TC_COLS;
    const float *src = (MODE == 1) ? col_src(a, cs) : nullptr;
#pragma unroll
    for (int it = 0; it < PF; ++it) {
        const int t = threadIdx.x + it * TC_THREADS;
        if (t >= TC_COLS * KC) break;
        if (MODE != 1) {
            const int grp = t / (8 * KC), rem = t % (8 * KC);
            const int kc = rem / 8, r = grp * 8 + rem % 8;
            const long long c = c0 + r;
            const int i0 = kc * EPC;
            if (a.vec4 && c < a.ncols && i0 + EPC <= a.n_in) {
#pragma unroll
                for (int j = 0; j < EPC; j += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(a.in + c * a.n_in + i0 + j);
                    pre[it][j] = q.x;
                    pre[it][j + 1] = q.y;
                    pre[it][j + 2] = q.z;
                    pre[it][j + 3] = q.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < EPC; ++j) {
                    const int i = i0 + j;
                    pre[it][j] = (c < a.ncols && i < a.n_in) ? a.in[c * a.n_in + i] : 0.f;
                }
            }
        } else {
            const int kc = t / TC_COLS;
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                const int i = kc * EPC + j;
                pre[it][j] = (cs < a.ncols && i < a.n_in) ? src[(long long)i * a.inner] : 0.f;
            }
        }
    }
}

// Registers -> the activation tile in the MMA layout (TF32 / BF16 / hi + lo).
template <int KIND, int MODE>
__device__ __forceinline__ void pipe_stage(unsigned char *xtile, size_t xbytes, int KC,
                                           const float (&pre)[PipeTraits<16 / KindTraits<KIND>::ESZ>::PF]
                                                             [16 / KindTraits<KIND>::ESZ]) {
    constexpr int EPC = 16 / KindTraits<KIND>::ESZ;
    constexpr int PF = PipeTraits<EPC>::PF;
#pragma unroll
    for (int it = 0; it < PF; ++it) {
        const int t = threadIdx.x + it * TC_THREADS;
        if (t >= TC_COLS * KC) break;
        int kc, r;
        if (MODE != 1) {
            const int grp = t / (8 * KC), rem = t % (8 * KC);
            kc = rem / 8;
            r = grp * 8 + rem % 8;
        } else {
            kc = t / TC_COLS;
            r = t % TC_COLS;
        }
        stage16<KIND>(xtile, TC_COLS, r, kc, pre[it], xbytes);
    }
}

// One column tile's MMAs into the accumulator at `acc` (single thread).
template <int KIND, int MODE>
__device__ __forceinline__ void pipe_mma(const unsigned char *wtile, const unsigned char *xtile,
                                         size_t wbytes, size_t xbytes, int wrows, int KC, int mh,
                                         uint32_t acc, uint32_t idesc) {
    using KT = KindTraits<KIND>;
    const uint32_t wa = tc::smem_u32(wtile), xa = tc::smem_u32(xtile);
    const uint32_t lbo_w = (uint32_t)wrows * 16, lbo_x = TC_COLS * 16;
    constexpr int NPROD = (KT::NSPLIT == 2) ? 3 : 1;  // split: (hi, hi), (hi, lo), (lo, hi)
    for (int st = 0; st < KC / 2; ++st) {
#pragma unroll
        for (int q = 0; q < NPROD; ++q) {
            const uint32_t wo = (q == 2) ? (uint32_t)wbytes : 0u;
            const uint32_t xo = (q == 1) ? (uint32_t)xbytes : 0u;
            const uint64_t dx = tc::make_sdesc(xa + xo + 2 * st * lbo_x, lbo_x, 128);
            const uint32_t accum = (st > 0 || q > 0) ? 1u : 0u;
            if (MODE == 0) {
                for (int h = 0; h < mh; ++h) {
                    const uint64_t dw =
                        tc::make_sdesc(wa + wo + 2 * st * lbo_w + (uint32_t)h * 2048u, lbo_w, 128);
                    tc::mma<KT::FMT>(acc + (uint32_t)(h * TC_COLS), dw, dx, idesc, accum);
                }
            } else {
                const uint64_t dw = tc::make_sdesc(wa + wo + 2 * st * lbo_w, lbo_w, 128);
                tc::mma<KT::FMT>(acc, dx, dw, idesc, accum);
            }
        }
    }
}

// Accumulator -> global for column tile c0 (all 8 warps; warp w reads TMEM
// lanes 32 (w % 4) .., warps w and w + 4 split the columns).
template <int MODE>
__device__ __forceinline__ void pipe_epilogue(const TcArgs &a, long long c0, uint32_t acc, int mh) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wq = warp & 3, wh = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    if (MODE == 0) {
        for (int h = 0; h < mh; ++h) {
            const int k = 128 * h + 32 * wq + lane;
            if (128 * h + 32 * wq >= a.n_out) continue;
            for (int cc = wh * (TC_COLS / 2); cc < (wh + 1) * (TC_COLS / 2); cc += 16) {
                float v[16];
                tc::tmem_ld16(acc + lane_base + (uint32_t)(h * TC_COLS + cc), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const long long c = c0 + cc + j;
                    if (k < a.n_out && c < a.ncols) a.out[c * a.n_out + k] = v[j];
                }
            }
        }
    } else if (MODE == 2) {
        // lane = row c of the output; 16 consecutive modes per TMEM load
        const long long c = c0 + 32 * wq + lane;
        float *dst = a.out + c * a.n_out;
        const bool v4 = a.vec4 && (a.n_out % 4 == 0);
        const int nk = a.n_pad / 16;
        for (int kk = 16 * ((nk * wh) / 2); kk < 16 * ((nk * (wh + 1)) / 2); kk += 16) {
            float v[16];
            tc::tmem_ld16(acc + lane_base + kk, v);
            if (c >= a.ncols) continue;
            if (v4 && kk + 16 <= a.n_out) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4 *>(dst + kk + j) =
                        make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (kk + j < a.n_out) dst[kk + j] = v[j];
            }
        }
    } else {
        const long long c = c0 + 32 * wq + lane;
        const long long o = c / a.inner, ci = c % a.inner;
        float *dst = a.out + o * a.n_out * a.inner + ci;
        const int nk = a.n_pad / 16;
        for (int kk = 16 * ((nk * wh) / 2); kk < 16 * ((nk * (wh + 1)) / 2); kk += 16) {
            float v[16];
            tc::tmem_ld16(acc + lane_base + kk, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = kk + j;
                if (k < a.n_out && c < a.ncols) dst[(long long)k * a.inner] = v[j];
            }
        }
    }
}

__host__ __device__ inline uint32_t tc_acc_cols(int mode, int mh, int n_pad) {
    return mode == 0 ? (uint32_t)(TC_COLS * mh)
                     : (n_pad <= 32 ? 32u : n_pad <= 64 ? 64u : n_pad <= 128 ? 128u : 256u);
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(TC_THREADS)
    k_tc_axis_pipe(const __grid_constant__ TcArgs a, const __grid_constant__ CUtensorMap wmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint64_t mbar_w;
    __shared__ uint32_t tmem_base;
    using KT = KindTraits<KIND>;
    constexpr int EPC = 16 / KT::ESZ;
    constexpr int PF = PipeTraits<EPC>::PF;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int KC = a.k_pad / EPC;
    const int mh = (MODE == 0) ? a.mh : 1;
    const int wrows = (MODE == 0) ? 128 * mh : a.n_pad;
    const size_t wbytes = (size_t)wrows * KC * 16, xbytes = (size_t)TC_COLS * KC * 16;
    // operand area from the next 128-byte boundary (the launch adds 128 bytes):
    // the TMA destination inside it must be 128-byte aligned
    unsigned char *base = smem + ((128u - (tc::smem_u32(smem) & 127u)) & 127u);
    unsigned char *wtile = base;
    unsigned char *xtile = base + KT::NSPLIT * wbytes;  // wbytes is a multiple of 512
    const uint32_t acc_cols = tc_acc_cols(MODE, mh, a.n_pad);
    const long long ntiles = (a.ncols + TC_COLS - 1) / TC_COLS;

    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init(&mbar_w, 1);
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * acc_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    bool failed = false;

    // ---- the weight operand, once per CTA ----
    if (a.w_tma) {
        float *raw = reinterpret_cast<float *>(xtile);  // free until the first tile
        if (tid == 0) {
            tc::mbar_expect_tx(&mbar_w, (uint32_t)(a.n_pad * a.k_pad * 4));
            tc::tma_load_2d(raw, &wmap, 0, 0, &mbar_w);
        }
        const bool ok = tc::mbar_wait_bounded(&mbar_w, 0, TC_DRAIN_NS);
        if (__syncthreads_or(ok ? 0 : 1)) {
            tc::mbar_wait_bounded(&mbar_w, 0, TC_DRAIN_NS);  // the copy lands before exit
            failed = true;
            if (tid == 0) atomicExch(a.err, 1);
        } else {
            for (int t = tid; t < wrows * KC; t += TC_THREADS) {
                const int kc = t / wrows, r = t % wrows;
                float v[EPC];
#pragma unroll
                for (int j = 0; j < EPC; ++j)
                    v[j] = (r < a.n_pad) ? raw[r * a.k_pad + kc * EPC + j] : 0.f;
                stage16<KIND>(wtile, wrows, r, kc, v, wbytes);
            }
        }
        __syncthreads();  // the raw weights are read before the first tile lands there
    } else {
        stage_w<KIND>(a, wtile, wrows, 0, KC, wbytes);
    }
    const uint32_t idesc = (MODE == 0) ? tc::make_idesc(KT::FMT, 128, TC_COLS)
                                       : tc::make_idesc(KT::FMT, 128, a.n_pad);

    float pre[PF][EPC];
    long long tile = blockIdx.x, prev_tile = -1;
    if (!failed && tile < ntiles) pipe_load<KIND, MODE>(a, tile * TC_COLS, KC, pre);
    uint32_t ph[2] = {0u, 0u};
    int k = 0;
    while (!failed && tile < ntiles) {
        const int b = k & 1;
        if (k >= 1) {  // MMA(k-1) done: the activation tile is free, its accumulator ready
            const bool ok = tc::mbar_wait_bounded(&mbar[b ^ 1], ph[b ^ 1], a.wait_ns);
            if (__syncthreads_or(ok ? 0 : 1)) {
                tc::mbar_wait_bounded(&mbar[b ^ 1], ph[b ^ 1], TC_DRAIN_NS);
                failed = true;
                if (tid == 0) atomicExch(a.err, 1);
                break;
            }
            ph[b ^ 1] ^= 1u;
            tc::fence_after_sync();
        }
        pipe_stage<KIND, MODE>(xtile, xbytes, KC, pre);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            pipe_mma<KIND, MODE>(wtile, xtile, wbytes, xbytes, wrows, KC, mh, tmem + b * acc_cols,
                                 idesc);
            tc::commit(&mbar[b]);
        }
        const long long next = tile + gridDim.x;
        if (next < ntiles) pipe_load<KIND, MODE>(a, next * TC_COLS, KC, pre);
        if (k >= 1) pipe_epilogue<MODE>(a, prev_tile * TC_COLS, tmem + (b ^ 1) * acc_cols, mh);
        // this epilogue's tensor-memory reads precede the next MMA into that accumulator
        tc::fence_before_sync();
        prev_tile = tile;
        tile = next;
        ++k;
    }
    if (!failed && k >= 1) {  // the last tile
        const int b = (k - 1) & 1;
        const bool ok = tc::mbar_wait_bounded(&mbar[b], ph[b], a.wait_ns);
        if (__syncthreads_or(ok ? 0 : 1)) {
            tc::mbar_wait_bounded(&mbar[b], ph[b], TC_DRAIN_NS);
            if (tid == 0) atomicExch(a.err, 1);
        } else {
            tc::fence_after_sync();
            pipe_epilogue<MODE>(a, prev_tile * TC_COLS, tmem + b * acc_cols, mh);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * acc_cols);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr if unavailable.
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

template <int KIND, int MODE>
static cudaError_t launch_tc_pipe(TcArgs a, cudaStream_t s, int nsm, int ctas_per_sm) {
    using KT = KindTraits<KIND>;
    constexpr int EPC = 16 / KT::ESZ;
    const int KC = a.k_pad / EPC;
    if (TC_COLS * KC > TC_THREADS * PipeTraits<EPC>::PF) return cudaErrorNotSupported;
    const int mh = (MODE == 0) ? a.mh : 1;
    const int wrows = (MODE == 0) ? 128 * mh : a.n_pad;
    const size_t wbytes = (size_t)wrows * KC * 16, xbytes = (size_t)TC_COLS * KC * 16;
    const size_t smem = KT::NSPLIT * (wbytes + xbytes) + 128;  // + alignment slack
    if (smem > TC_SMEM_MAX) return cudaErrorNotSupported;
    if (wbytes % 512 != 0) return cudaErrorNotSupported;  // keeps the TMA destination aligned
    const uint32_t acc_cols = tc_acc_cols(MODE, mh, a.n_pad);
    if (2 * acc_cols > 512) return cudaErrorNotSupported;
    // the weights by TMA: row pitch a multiple of 16 bytes, the padded box
    // within the activation area it is staged in
    CUtensorMap wmap;
    std::memset(&wmap, 0, sizeof wmap);
    a.w_tma = 0;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (enc && (a.n_in * 4) % 16 == 0 && (reinterpret_cast<uintptr_t>(a.wt) & 15u) == 0 &&
        (size_t)a.n_pad * a.k_pad * 4 <= KT::NSPLIT * xbytes && a.k_pad <= 256 && a.n_pad <= 256) {
        const cuuint64_t gdim[2] = {(cuuint64_t)a.n_in, (cuuint64_t)a.n_out};
        const cuuint64_t gstride[1] = {(cuuint64_t)a.n_in * 4};
        const cuuint32_t box[2] = {(cuuint32_t)a.k_pad, (cuuint32_t)a.n_pad};
        const cuuint32_t estride[2] = {1, 1};
        if (enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(a.wt), gdim,
                gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            a.w_tma = 1;
    }
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e =
            smem_attr_once((const void *)k_tc_axis_pipe<KIND, MODE>, (int)TC_SMEM_MAX, attr);
        if (e != cudaSuccess) return e;
    }
    int per_sm = (int)(512 / (2 * acc_cols));
    const int by_smem = (int)((220 * 1024) / (smem + 1024));
    if (by_smem < per_sm) per_sm = by_smem;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    if (per_sm < 1) return cudaErrorNotSupported;
    const long long ntiles = (a.ncols + TC_COLS - 1) / TC_COLS;
    long long grid = (long long)nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid <= 0) return cudaSuccess;
    k_tc_axis_pipe<KIND, MODE><<<(unsigned)grid, TC_THREADS, smem, s>>>(a, wmap);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// K-streamed pipelined variant, for contractions whose K is too long for the
// register prefetch of k_tc_axis_pipe (the n = 129 axes of a 128-span p = 3
// grid): the weight operand (N = n_pad <= 256 rows, all of K, zero padded)
// stays in shared memory for the CTA's life; each 128-column tile streams its
// activation rows in steps of PK_KB 16-byte K chunks through two
// shared-memory buffers, with the next two steps held in registers, and its
// MMAs chain into one of two TMEM accumulators:
//     wait MMA(s-2) -> stage step s -> MMA(s) -> load step s+2
//     -> (last step of a tile) drain the previous tile's accumulator.
// Strided axis (MODE_S) and the contiguous axis as MODE_XT only (the weight
// is the N operand).  Step s completes on mbarrier s & 1 with parity
// (s >> 1) & 1, tile t on the accumulator barrier t & 1 with parity
// (t >> 1) & 1.
// ---------------------------------------------------------------------------
constexpr int PK_KB = 6;  // 16-byte K chunks per step: three MMA K steps
constexpr size_t PK_SMEM_MAX = 225 * 1024;

template <int KIND>
struct PkTraits {
    static constexpr int EPC = 16 / KindTraits<KIND>::ESZ;
    static constexpr int PF = TC_COLS * PK_KB / TC_THREADS;  // chunks per thread and step
    static constexpr int NPT = PF * EPC;                     // values per thread and step
    static constexpr int W = PK_KB * EPC;                    // K values per step
    static constexpr int RP = W + 4;  // raw row pitch (floats): conflict-free 16-byte reads
    static_assert(TC_COLS * PK_KB % TC_THREADS == 0, "whole chunks per thread");
};

// Global -> registers: K values [kc0 EPC, kc0 EPC + W) of column tile c0.
// MODE_S: a thread loads its column's chunks (lanes: consecutive columns);
// MODE_XT: lanes take consecutive values of a row (rows of n_in values need
// not be 16-byte aligned), and the step is regrouped into chunks through
// shared memory (pk_stage).
template <int KIND, int MODE>
__device__ __forceinline__ void pk_load(const TcArgs &a, long long c0, int kc0,
                                        float (&pre)[PkTraits<KIND>::NPT]) {
    using PT = PkTraits<KIND>;
    constexpr int EPC = PT::EPC;
    if (MODE == 1) {
        const long long c = c0 + threadIdx.x % TC_COLS;
        const float *src = col_src(a, c);
#pragma unroll
        for (int it = 0; it < PT::PF; ++it) {
            const int kc = threadIdx.x / TC_COLS + it * (TC_THREADS / TC_COLS);
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                const int i = (kc0 + kc) * EPC + j;
                pre[it * EPC + j] = (c < a.ncols && i < a.n_in) ? src[(long long)i * a.inner] : 0.f;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < PT::NPT; ++k) {
            const int e = threadIdx.x + k * TC_THREADS;
            const int r = e / PT::W, i = kc0 * EPC + e % PT::W;
            const long long c = c0 + r;
            pre[k] = (c < a.ncols && i < a.n_in) ? a.in[c * a.n_in + i] : 0.f;
        }
    }
}

// Registers -> one step buffer (PK_KB chunks of 128 rows, MMA layout); MODE_XT
// through the raw buffer (one barrier).  Lanes store consecutive rows of a
// chunk (contiguous in the core-matrix layout).
template <int KIND, int MODE>
__device__ __forceinline__ void pk_stage(unsigned char *xbuf, size_t xb, float *raw,
                                         const float (&pre)[PkTraits<KIND>::NPT]) {
    using PT = PkTraits<KIND>;
    constexpr int EPC = PT::EPC;
    if (MODE == 1) {
#pragma unroll
        for (int it = 0; it < PT::PF; ++it) {
            const int kc = threadIdx.x / TC_COLS + it * (TC_THREADS / TC_COLS);
            stage16<KIND>(xbuf, TC_COLS, threadIdx.x % TC_COLS, kc, &pre[it * EPC], xb);
        }
    } else {
#pragma unroll
        for (int k = 0; k < PT::NPT; ++k) {
            const int e = threadIdx.x + k * TC_THREADS;
            raw[(e / PT::W) * PT::RP + e % PT::W] = pre[k];
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < PT::PF; ++it) {
            const int t = threadIdx.x + it * TC_THREADS;
            const int kc = t / TC_COLS, r = t % TC_COLS;
            float v[EPC];
#pragma unroll
            for (int j = 0; j < EPC; j += 4) {
                const float4 q = *reinterpret_cast<const float4 *>(raw + r * PT::RP + kc * EPC + j);
                v[j] = q.x;
                v[j + 1] = q.y;
                v[j + 2] = q.z;
                v[j + 3] = q.w;
            }
            stage16<KIND>(xbuf, TC_COLS, r, kc, v, xb);
        }
    }
}

// One step's MMAs (single thread): K chunks kc0 .. kc0 + PK_KB of the
// resident weight against the step buffer.
template <int KIND>
__device__ __forceinline__ void pk_mma(uint32_t wa, uint32_t xa, size_t wbytes, size_t xb,
                                       int wrows, int kc0, bool first, uint32_t acc,
                                       uint32_t idesc) {
    using KT = KindTraits<KIND>;
    const uint32_t lbo_w = (uint32_t)wrows * 16, lbo_x = TC_COLS * 16;
    constexpr int NPROD = (KT::NSPLIT == 2) ? 3 : 1;  // split: (hi, hi), (hi, lo), (lo, hi)
#pragma unroll
    for (int st = 0; st < PK_KB / 2; ++st) {
#pragma unroll
        for (int q = 0; q < NPROD; ++q) {
            const uint32_t wo = (q == 2) ? (uint32_t)wbytes : 0u;
            const uint32_t xo = (q == 1) ? (uint32_t)xb : 0u;
            const uint64_t dx = tc::make_sdesc(xa + xo + 2 * st * lbo_x, lbo_x, 128);
            const uint64_t dw =
                tc::make_sdesc(wa + wo + (uint32_t)(kc0 + 2 * st) * lbo_w, lbo_w, 128);
            const uint32_t accum = (!first || st > 0 || q > 0) ? 1u : 0u;
            tc::mma<KT::FMT>(acc, dx, dw, idesc, accum);
        }
    }
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_tc_axis_pipek(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar_x[2], mbar_acc[2];
    __shared__ uint32_t tmem_base;
    using KT = KindTraits<KIND>;
    constexpr int EPC = PkTraits<KIND>::EPC, NPT = PkTraits<KIND>::NPT;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int KC = a.k_pad / EPC;  // a multiple of PK_KB
    const int NC = KC / PK_KB;     // steps per tile
    const int wrows = a.n_pad;
    const size_t wbytes = (size_t)wrows * KC * 16, xb = (size_t)TC_COLS * PK_KB * 16;
    unsigned char *base = smem + ((128u - (tc::smem_u32(smem) & 127u)) & 127u);
    unsigned char *wtile = base;
    unsigned char *xbuf0 = base + KT::NSPLIT * wbytes;  // two buffers of NSPLIT * xb
    float *raw = reinterpret_cast<float *>(xbuf0 + 2 * KT::NSPLIT * xb);  // MODE_XT regrouping
    const uint32_t acc_cols = tc_acc_cols(1, 1, a.n_pad);
    const long long ntiles = (a.ncols + TC_COLS - 1) / TC_COLS;
    const long long my_tiles =
        (blockIdx.x < ntiles) ? (ntiles - 1 - (long long)blockIdx.x) / gridDim.x + 1 : 0;
    const long long S = my_tiles * NC;  // steps of this CTA

    if (tid == 0) {
        tc::mbar_init(&mbar_x[0], 1);
        tc::mbar_init(&mbar_x[1], 1);
        tc::mbar_init(&mbar_acc[0], 1);
        tc::mbar_init(&mbar_acc[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * acc_cols);
    stage_w<KIND>(a, wtile, wrows, 0, KC, wbytes);  // made visible by the first step's fence
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::make_idesc(KT::FMT, 128, a.n_pad);
    auto tile_of = [&](long long ti) { return (long long)blockIdx.x + ti * gridDim.x; };

    // after a wait ran out: record it, let the MMAs of step `last` (and so all
    // before it) finish, bounded, before the tensor memory is released
    auto give_up = [&](long long last) {
        if (last >= 0)
            tc::mbar_wait_bounded(&mbar_x[last & 1], (uint32_t)((last >> 1) & 1), TC_DRAIN_NS);
        if (tid == 0) atomicExch(a.err, 1);
    };
    // step s with its data in `cur`; the step s + 2 is loaded into `cur`.  False if
    // a wait ran out (the CTA gives up).
    auto body = [&](long long s, float (&cur)[NPT]) -> bool {
        const int b = (int)(s & 1);
        const long long ti = s / NC;
        const int ch = (int)(s % NC);
        unsigned char *xbuf = xbuf0 + (size_t)b * KT::NSPLIT * xb;
        if (s >= 2) {  // the MMAs of step s - 2 have read this buffer
            const bool ok =
                tc::mbar_wait_bounded(&mbar_x[b], (uint32_t)(((s - 2) >> 1) & 1), a.wait_ns);
            if (__syncthreads_or(ok ? 0 : 1)) {
                give_up(s - 1);
                return false;
            }
            tc::fence_after_sync();
        }
        pk_stage<KIND, MODE>(xbuf, xb, raw, cur);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            pk_mma<KIND>(tc::smem_u32(wtile), tc::smem_u32(xbuf), wbytes, xb, wrows, ch * PK_KB,
                         ch == 0, tmem + (uint32_t)(ti & 1) * acc_cols, idesc);
            tc::commit(&mbar_x[b]);
            if (ch == NC - 1) tc::commit(&mbar_acc[ti & 1]);
        }
        if (s + 2 < S)
            pk_load<KIND, MODE>(a, tile_of((s + 2) / NC) * TC_COLS, (int)((s + 2) % NC) * PK_KB, cur);
        if (ch == NC - 1 && ti >= 1) {  // drain the previous tile while this one's MMAs run
            const int pb = (int)((ti - 1) & 1);
            const bool ok = tc::mbar_wait_bounded(&mbar_acc[pb], (uint32_t)(((ti - 1) >> 1) & 1),
                                                  a.wait_ns);
            if (__syncthreads_or(ok ? 0 : 1)) {
                give_up(s);
                return false;
            }
            tc::fence_after_sync();
            pipe_epilogue<MODE>(a, tile_of(ti - 1) * TC_COLS, tmem + (uint32_t)pb * acc_cols, 1);
            // these tensor-memory reads precede the next MMA into that accumulator
            tc::fence_before_sync();
        }
        return true;
    };

    float pre0[NPT], pre1[NPT];
    if (S > 0) pk_load<KIND, MODE>(a, tile_of(0) * TC_COLS, 0, pre0);
    if (S > 1) pk_load<KIND, MODE>(a, tile_of(1 / NC) * TC_COLS, (1 % NC) * PK_KB, pre1);
    bool failed = false;
    long long s = 0;
    for (; s + 1 < S; s += 2) {
        if (!body(s, pre0) || !body(s + 1, pre1)) {
            failed = true;
            break;
        }
    }
    if (!failed && s < S && !body(s, pre0)) failed = true;
    if (!failed && S > 0) {  // the last tile
        const long long tl = my_tiles - 1;
        const bool ok = tc::mbar_wait_bounded(&mbar_acc[tl & 1], (uint32_t)((tl >> 1) & 1),
                                              a.wait_ns);
        if (__syncthreads_or(ok ? 0 : 1)) {
            give_up(S - 1);
        } else {
            tc::fence_after_sync();
            pipe_epilogue<MODE>(a, tile_of(tl) * TC_COLS, tmem + (uint32_t)(tl & 1) * acc_cols, 1);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * acc_cols);
}

template <int KIND, int MODE>
static cudaError_t launch_tc_pipek(TcArgs a, cudaStream_t s, int nsm, int ctas_per_sm) {
    using KT = KindTraits<KIND>;
    constexpr int EPC = PkTraits<KIND>::EPC;
    if (MODE == 0 || a.n_pad > 256) return cudaErrorNotSupported;
    const int kstep = PK_KB * EPC;  // K per step
    a.k_pad = (a.n_in + kstep - 1) / kstep * kstep;
    const int KC = a.k_pad / EPC;
    const size_t wbytes = (size_t)a.n_pad * KC * 16, xb = (size_t)TC_COLS * PK_KB * 16;
    const size_t rawb = (MODE == 2) ? (size_t)TC_COLS * PkTraits<KIND>::RP * 4 : 0;
    const size_t smem = KT::NSPLIT * (wbytes + 2 * xb) + rawb + 128;  // + alignment slack
    if (smem > PK_SMEM_MAX) return cudaErrorNotSupported;
    const uint32_t acc_cols = tc_acc_cols(1, 1, a.n_pad);
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e =
            smem_attr_once((const void *)k_tc_axis_pipek<KIND, MODE>, (int)PK_SMEM_MAX, attr);
        if (e != cudaSuccess) return e;
    }
    int per_sm = (int)(512 / (2 * acc_cols));
    const int by_smem = (int)((228 * 1024) / (smem + 1024));
    if (by_smem < per_sm) per_sm = by_smem;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    if (per_sm < 1) return cudaErrorNotSupported;
    const long long ntiles = (a.ncols + TC_COLS - 1) / TC_COLS;
    long long grid = (long long)nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid <= 0) return cudaSuccess;
    k_tc_axis_pipek<KIND, MODE><<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KIND, int MODE>
static cudaError_t launch_tc_t(TcArgs a, cudaStream_t s, int nsm, int ctas_per_sm) {
    using KT = KindTraits<KIND>;
    constexpr int EPC = 16 / KT::ESZ;
    const int KC = a.k_pad / EPC;
    const int wrows = (MODE == 0) ? 128 * a.mh : a.n_pad;
    // stage the whole K when it fits (in the shared memory of one CTA, or of
    // one of ctas_per_sm CTAs when that is asked for), else balanced even
    // chunks under that limit
    const size_t per_chunk = (size_t)KT::NSPLIT * (wrows + TC_COLS) * 16;
    size_t limit = TC_SMEM_MAX;
    if (ctas_per_sm > 1) {  // (a share too small for two chunks falls back to one CTA's
                            // limit: the tensor cores keep the transform either way)
        const size_t share = (size_t)(220 * 1024) / ctas_per_sm - 1024;
        if (share < limit && share >= 2 * per_chunk) limit = share;
    }
    int kch = KC;
    if (per_chunk * KC > limit) {
        const int kmax = (int)(limit / per_chunk) & ~1;
        if (kmax < 2) return cudaErrorNotSupported;  // the caller uses CUDA cores
        const int nch = (KC + kmax - 1) / kmax;
        kch = (((KC + nch - 1) / nch) + 1) & ~1;
    }
    a.kch = kch;
    const size_t smem = per_chunk * kch;
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e =
            smem_attr_once((const void *)k_tc_axis<KIND, MODE>, (int)TC_SMEM_MAX, attr);
        if (e != cudaSuccess) return e;
    }
    // CTAs per SM limited so that their TMEM columns fit in 512
    const int tmem_cols = (MODE == 0) ? TC_COLS * a.mh
                                      : (a.n_pad <= 32 ? 32 : a.n_pad <= 64 ? 64
                                         : a.n_pad <= 128 ? 128 : 256);
    int per_sm = 512 / tmem_cols;
    const int by_smem = (int)((220 * 1024) / (smem + 1024));
    if (by_smem < per_sm) per_sm = by_smem;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    const long long ntiles = (a.ncols + TC_COLS - 1) / TC_COLS;
    long long grid = (long long)nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid <= 0) return cudaSuccess;
    k_tc_axis<KIND, MODE><<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// Returns cudaErrorNotSupported when the shape is outside what the kernel
// covers (the caller then uses the CUDA-core transform).
cudaError_t launch_tc_axis(int kind, int mode, const float *in, float *out, const float *wt,
                           int n_in, int n_out, long long ncols, long long inner, int *err,
                           int nsm, cudaStream_t s, int ctas_per_sm,
                           unsigned long long wait_ns) {
    TcArgs a;
    a.wait_ns = wait_ns;
    a.in = in;
    a.out = out;
    a.wt = wt;
    a.n_in = n_in;
    a.n_out = n_out;
    const int kstep = (kind == tc::FMT_BF16) ? 16 : 8;
    a.k_pad = (n_in + kstep - 1) / kstep * kstep;
    a.n_pad = (n_out + 15) / 16 * 16;
    a.ncols = ncols;
    a.inner = inner;
    a.err = err;
    if (ncols <= 0) return cudaSuccess;
    if (mode == 0 && n_out > 256) return cudaErrorNotSupported;
    if (mode == 1 && a.n_pad > 256) return cudaErrorNotSupported;
    a.mh = (mode == 0 && n_out > 128) ? 2 : 1;
    a.kch = 0;
    a.vec4 = (mode == 0 && n_in % 4 == 0 && (reinterpret_cast<uintptr_t>(in) & 15u) == 0 &&
              (reinterpret_cast<uintptr_t>(out) & 15u) == 0) ? 1 : 0;
    a.w_tma = 0;
    // the pipelined kernel where the shape fits it, else the one-tile-at-a-time one
    cudaError_t e;
    // (the contiguous axis as MODE_XT = 2)
    if (kind == KIND_TF32X3)
        e = mode == 0 ? launch_tc_pipe<KIND_TF32X3, 2>(a, s, nsm, ctas_per_sm)
                      : launch_tc_pipe<KIND_TF32X3, 1>(a, s, nsm, ctas_per_sm);
    else if (kind == tc::FMT_TF32)
        e = mode == 0 ? launch_tc_pipe<tc::FMT_TF32, 2>(a, s, nsm, ctas_per_sm)
                      : launch_tc_pipe<tc::FMT_TF32, 1>(a, s, nsm, ctas_per_sm);
    else
        e = mode == 0 ? launch_tc_pipe<tc::FMT_BF16, 2>(a, s, nsm, ctas_per_sm)
                      : launch_tc_pipe<tc::FMT_BF16, 1>(a, s, nsm, ctas_per_sm);
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
    // K too long for the register prefetch: the K-streamed pipeline
    if (kind == KIND_TF32X3)
        e = mode == 0 ? launch_tc_pipek<KIND_TF32X3, 2>(a, s, nsm, ctas_per_sm)
                      : launch_tc_pipek<KIND_TF32X3, 1>(a, s, nsm, ctas_per_sm);
    else if (kind == tc::FMT_TF32)
        e = mode == 0 ? launch_tc_pipek<tc::FMT_TF32, 2>(a, s, nsm, ctas_per_sm)
                      : launch_tc_pipek<tc::FMT_TF32, 1>(a, s, nsm, ctas_per_sm);
    else
        e = mode == 0 ? launch_tc_pipek<tc::FMT_BF16, 2>(a, s, nsm, ctas_per_sm)
                      : launch_tc_pipek<tc::FMT_BF16, 1>(a, s, nsm, ctas_per_sm);
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
    if (kind == KIND_TF32X3)
        return mode == 0 ? launch_tc_t<KIND_TF32X3, 0>(a, s, nsm, ctas_per_sm)
                         : launch_tc_t<KIND_TF32X3, 1>(a, s, nsm, ctas_per_sm);
    if (kind == tc::FMT_TF32)
        return mode == 0 ? launch_tc_t<tc::FMT_TF32, 0>(a, s, nsm, ctas_per_sm)
                         : launch_tc_t<tc::FMT_TF32, 1>(a, s, nsm, ctas_per_sm);
    return mode == 0 ? launch_tc_t<tc::FMT_BF16, 0>(a, s, nsm, ctas_per_sm)
                     : launch_tc_t<tc::FMT_BF16, 1>(a, s, nsm, ctas_per_sm);
}

}  // namespace st

// Thin inline-PTX wrappers for the 5th-generation tensor cores of sm_100 /
// sm_103 (tcgen05), tensor memory (TMEM) and mbarriers.
//
// Operand tiles live in shared memory in the canonical K-major layout
// without swizzle: 8-row x 16-byte "core matrices", row r / byte column b of
// a tile with R rows at
//     (b / 16) * (R * 16) + (r / 8) * 128 + (r % 8) * 16 + (b % 16)
// i.e. stride-dimension byte offset (between 8-row groups) SBO = 128 and
// leading-dimension byte offset (between core matrices along K) LBO = R * 16.
// One MMA instruction consumes 32 bytes of K (8 TF32 or 16 BF16 elements), so
// K-step s starts at tile + 2 s LBO.
#pragma once
#include <cstdint>

namespace st {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of (row r, byte column b) in a K-major no-swizzle tile of R rows.
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int R, int r, int b) {
    return (uint32_t)((b >> 4) * (R * 16) + (r >> 3) * 128 + (r & 7) * 16 + (b & 15));
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor for kind::tf32 / kind::f16: D = F32, A/B format
// (TF32 = 2, BF16 = 1), both operands K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
__host__ __device__ __forceinline__ uint32_t make_idesc(int ab_format, int M, int N) {
    uint32_t d = 0;
    d |= 1u << 4;                          // D format F32
    d |= (uint32_t)(ab_format & 7) << 7;   // A format
    d |= (uint32_t)(ab_format & 7) << 10;  // B format
    d |= (uint32_t)((N >> 3) & 0x3F) << 17;
    d |= (uint32_t)((M >> 4) & 0x1F) << 24;
    return d;
}
constexpr int FMT_BF16 = 1;
constexpr int FMT_TF32 = 2;

// ---- TMEM allocation (one full warp) ----
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(smem_dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols)
                 : "memory");
}

// ---- MMA (single thread) ----
template <int KIND>  // FMT_TF32 or FMT_BF16
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
    if (KIND == FMT_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
    }
}

// Make all prior tcgen05.mma of this thread arrive on the mbarrier when done.
__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

// ---- fences ----
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- mbarrier ----
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return ok != 0;
}
// Non-blocking probe of the phase (mbarrier.test_wait never suspends).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wall-clock bounded wait: returns false if the phase did not complete within
// limit_ns nanoseconds (the caller then records an error and bails out);
// limit_ns = 0 tests the phase once without waiting.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (limit_ns == 0) return mbar_test_wait(mbar, parity);
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_test_wait(mbar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
}

// ---- TMA (tensor memory accelerator) ----
// Arm the mbarrier for one arrival plus `bytes` bytes of asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
// 2D tiled TMA load of the box at element coordinates (x, y) of the tensor map
// (a __grid_constant__ kernel parameter) into shared memory; completion is
// signalled on the mbarrier as transferred bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y,
                                            uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y),
           "r"(smem_u32(mbar))
        : "memory");
}

// ---- TMEM -> registers: 32 lanes x 32 bit, 16 consecutive columns ----
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace st

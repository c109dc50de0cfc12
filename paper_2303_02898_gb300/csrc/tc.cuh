// tc.cuh -- inline-PTX helpers for the fifth-generation tensor cores of
// sm_103a (tcgen05: TMEM accumulators, MMAs issued by one thread, shared
// memory operands described by 64-bit descriptors), for the bulk-copy engine
// (cp.async.bulk) and for mbarriers.
//
// Operand layout used throughout (K-major, no swizzle): a matrix of R rows
// and K columns (K contiguous) is stored as "core matrices" of 8 rows x 16
// bytes, each 128 contiguous bytes (row r at byte 16 (r % 8)).  Core matrices
// adjacent along K are LBO bytes apart, 8-row groups SBO bytes apart:
//   byte(r, k) = (r / 8) SBO + (k / T) LBO + 16 (r % 8) + (k % T) size,
// T = 16 / size elements per 16 bytes.  Here LBO = 128 and SBO = 128 K / T:
// every 8-row group is one contiguous run of K / T core matrices.  One MMA
// reads 32 bytes of K (two core matrices: 16 BF16 or 8 TF32 values), so the
// descriptor of K step s starts 256 s bytes further.
//
// Accumulators (M = 128, cta_group::1): row i of D is TMEM lane i, column j is
// TMEM column (base + j), FP32.  Warp w reads lanes 32 (w % 4) .. + 31.
#pragma once

#include <stdint.h>

namespace mem {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- instruction descriptor (kind::f16 / kind::tf32), dense, FP32 D,
// both operands K-major.  ab: 0 = F16, 1 = BF16, 2 = TF32.
__host__ __device__ constexpr uint32_t idesc(int M, int N, int ab) {
    return (1u << 4) | ((uint32_t)ab << 7) | ((uint32_t)ab << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// ---- shared-memory matrix descriptor, no swizzle (layout type 0),
// version 1 (bits 46-47), base offset 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Shared-memory matrix descriptor for the 128-byte swizzled K-major layout
// that a TMA tensor load with CU_TENSOR_MAP_SWIZZLE_128B writes: rows of 128
// bytes, the 16-byte chunks of row r XOR-permuted by (r mod 8), 8-row atoms of
// 1024 bytes SBO apart (the tile must start on a 1024-byte boundary).  One
// MMA reads 32 bytes of K; K step s starts 32 s bytes further.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46) | (2ull << 61);
}

// Byte offset of element (r, k) in the layout above (size = element bytes).
__host__ __device__ constexpr uint32_t kmajor_off(int r, int k, int K, int size) {
    return (uint32_t)((r >> 3) * (128 * K * size / 16) + (k / (16 / size)) * 128 + (r & 7) * 16 +
                      (k % (16 / size)) * size);
}

// ---- TMEM allocation (one whole warp executes these)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the async proxy
// (tensor cores, bulk copies)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- MMA: D[tmem] (+)= A[smem] . B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
// Arrive on an mbarrier once every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

// ---- TMEM -> registers: 32 lanes x 32 bits, 8 consecutive columns; thread
// t of the warp gets lane (taddr lane + t), columns c .. c + 7.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr)
                 : "memory");
    v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

// ---- mbarriers
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity to complete: false after
// max_polls unsuccessful polls (each poll may suspend the thread briefly).
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t max_polls) {
    for (uint32_t i = 0; i < max_polls; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// ---- bulk copy global -> shared (the TMA engine, no tensor map): bytes a
// multiple of 16, both addresses 16-byte aligned; completion counted on mbar.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

// ---- tiled tensor copy global -> shared through a tensor map (2D box at
// element coordinates (x, y), x innermost; x times the element size must be
// a multiple of 16 bytes); completion counted on mbar.
__device__ __forceinline__ void tma_load_2d(void *dst_smem, const void *tmap, int x, int y, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst_smem)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}

// ---- TF32 rounding (round to nearest, ties away) and the hi/lo split of
// split-precision products: x = hi + lo, both representable in TF32 up to
// the rounding of lo.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace mem

// Inline-PTX helpers of the 5th-generation tensor-core kernels (tcgen05.mma
// with TMEM accumulators, bulk copies completing on mbarriers), shared by the
// dictionary matcher and the patch kNN.
//
// Shared-memory operand layout: canonical K-major, no swizzle: 8-row x 16-byte
// core matrices, core (row group g, k chunk c) at byte (g * KC + c) * 128,
// KC = padded length / 8; descriptor LBO (next core along K) = 128 bytes, SBO
// (next 8-row group) = KC * 128 bytes.
#pragma once
#include <cstdint>

namespace mrf {

constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                  // descriptor version of the 5th-generation tensor core
    return d;                                // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: BF16 x BF16 -> F32, K-major A and B
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// kind::f16 instruction descriptor: F16 x F16 -> F32, K-major A and B
__host__ __device__ constexpr uint32_t mma_idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) in the core-matrix layout with KC k-chunks
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, int KC) {
    return (uint32_t)((((row >> 3) * KC + (k >> 3)) * 128) + ((row & 7) * 16) + ((k & 7) * 2));
}

// bounded wait on an mbarrier phase; returns false if it gave up after
// `limit` polls
__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity, unsigned limit = kSpinLimit) {
    uint32_t done = 0;
    unsigned spins = 0;
    while (!done) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity));
        if (!done && ++spins > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// 16 consecutive 32-bit TMEM columns of the warp's 32 lanes into v.  The copy
// is asynchronous: v is defined only after tmem_wait16, which names v as
// read-written so that no use of v moves above it (and `keep`, a value the
// code between the two computes, so that work stays before the wait).
__device__ __forceinline__ void tmem_ld16(uint32_t (&v)[16], uint32_t taddr) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait16(uint32_t (&v)[16], float& keep) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
                   "+r"(v[14]), "+r"(v[15]), "+f"(keep));
}

}  // namespace mrf

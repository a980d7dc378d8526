// Strided FP32-accurate GEMM on the 5th-generation tensor cores, for the
// learned matcher's training products (forward H W^T, weight gradient
// dZ^T H, input gradient dZ W):
//   C[m][n] (+)= sum_k A(m, k) B(k, n),  A(m, k) = A[m sam + k sak],
//                                         B(k, n) = B[k sbk + n sbn].
// A CTA owns a 128-row tile of C (one TMEM lane per row) and NT columns; the
// reduction runs in chunks of 64: all 128 threads convert the chunk's A rows
// and B columns to BF16 hi/lo parts (v = hi + lo, hi = bf16(v), lo =
// bf16(v - hi)) in the canonical K-major core-matrix layout of shared memory,
// one thread issues the products A_hi B_hi + A_lo B_hi (+ A_hi B_lo when B is
// FP32; the BF16 weight copy is exact in hi alone) into the FP32 accumulators,
// and the block waits on the MMAs' mbarrier before the next chunk reuses the
// tiles.  Products are exact to ~2^-16 relative, as the FP32 SIMT kernel.
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "common.h"
#include "tc5.cuh"

namespace mrf {

constexpr int kGtM = 128;     // rows of C per CTA (TMEM lanes)
constexpr int kGtK = 64;      // reduction chunk (128-byte rows)

__device__ __forceinline__ float gt_val(float v) { return v; }
__device__ __forceinline__ float gt_val(__nv_bfloat16 v) { return __bfloat162float(v); }

// v = hi + lo as two BF16 parts, stored at byte offset `off` of the hi and lo
// tiles (lo tile `part_bytes` after hi)
__device__ __forceinline__ void gt_store(unsigned char* t, int part_bytes, uint32_t off, float v, bool split) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(t + off) = hi;
    if (split) *reinterpret_cast<__nv_bfloat16*>(t + part_bytes + off) = __float2bfloat16_rn(v - __bfloat162float(hi));
}

template <typename TA, typename TB, int NT>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const TA* __restrict__ A, int sam, int sak,
                                                 const TB* __restrict__ B, int sbk, int sbn, float* __restrict__ C,
                                                 int ldc, int accumulate, int* __restrict__ err) {
    constexpr bool SPLIT_B = !std::is_same<TB, __nv_bfloat16>::value;
    constexpr int A_PART = kGtM * kGtK * 2;            // 16 KB per part
    constexpr int B_PART = NT * kGtK * 2;
    constexpr int KC = kGtK / 8;                       // 16-byte cores along a chunk row
    constexpr int NCOLS = NT < 32 ? 32 : NT;           // TMEM allocation (power of two >= 32)
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sA = smraw;                         // hi, lo: [128][64] each
    unsigned char* sB = smraw + 2 * A_PART;            // hi (, lo): [NT][64] each
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGtM, n0 = blockIdx.x * NT;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&s_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = mma_idesc(kGtM, NT);
    uint32_t phase = 0;
    int issued = 0, failed = 0;
    for (int k0 = 0; k0 < K; k0 += kGtK) {
        // A rows m0..m0+127 and B columns n0..n0+NT-1 of this chunk, eight
        // loads in flight per thread
        for (int b = tid; b < kGtM * kGtK; b += 8 * 128) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = b + u * 128, r = e / kGtK, kk = e - r * kGtK;
                v[u] = (e < kGtM * kGtK && m0 + r < M && k0 + kk < K)
                           ? gt_val(A[(size_t)(m0 + r) * sam + (size_t)(k0 + kk) * sak]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = b + u * 128, r = e / kGtK, kk = e - r * kGtK;
                if (e < kGtM * kGtK) gt_store(sA, A_PART, core_off(r, kk, KC), v[u], true);
            }
        }
        for (int b = tid; b < NT * kGtK; b += 8 * 128) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = b + u * 128, c = e / kGtK, kk = e - c * kGtK;
                v[u] = (e < NT * kGtK && n0 + c < N && k0 + kk < K)
                           ? gt_val(B[(size_t)(k0 + kk) * sbk + (size_t)(n0 + c) * sbn]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = b + u * 128, c = e / kGtK, kk = e - c * kGtK;
                if (e < NT * kGtK) gt_store(sB, B_PART, core_off(c, kk, KC), v[u], SPLIT_B);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int ks = 0; ks < kGtK / 16; ++ks) {
#pragma unroll
                for (int pr = 0; pr < (SPLIT_B ? 3 : 2); ++pr) {
                    // (A_hi, B_hi), (A_lo, B_hi), (A_hi, B_lo)
                    const uint32_t ao = pr == 1 ? A_PART : 0, bo = pr == 2 ? B_PART : 0;
                    const uint64_t ad = smem_desc(smem_u32(sA) + ao + ks * 256, 128, KC * 128);
                    const uint64_t bd = smem_desc(smem_u32(sB) + bo + ks * 256, 128, KC * 128);
                    const uint32_t acc = (k0 > 0 || ks > 0 || pr > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            mma_commit(smem_u32(&s_bar));
        }
        ++issued;
        // the tiles are rewritten next chunk: wait for this chunk's products
        // (bounded; the outcome is made block-uniform)
        const int ok = wait_parity(smem_u32(&s_bar), phase) ? 1 : 0;
        phase ^= 1u;
        failed = __syncthreads_or(!ok);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (failed) break;
    }
    if (!failed && issued > 0) {
        // epilogue: warp w holds rows m0 + 32 w + lane
        const int m = m0 + 32 * warp + lane;
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t v[16];
            float keep = 0.f;
            tmem_ld16(v, tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0);
            tmem_wait16(v, keep);
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < N) {
                        float* c = C + (size_t)m * ldc + n;
                        *c = accumulate ? *c + __uint_as_float(v[j]) : __uint_as_float(v[j]);
                    }
                }
            }
        }
    }
    if (failed && tid == 0) {
        atomicExch(err, 1);
        wait_parity(smem_u32(&s_bar), phase ^ 1u);     // the products in flight finish first (bounded)
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

}  // namespace mrf

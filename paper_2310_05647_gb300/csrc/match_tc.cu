// Dictionary matching (Eq. 5) on the 5th-generation tensor cores.
//
// The complex inner products s_nm = <d_m, x_n> = sum_k conj(d_mk) x_nk are a
// real GEMM C = A B^T with
//   A[n]      = (Re x_n0, Im x_n0, Re x_n1, ...)              (fingerprints)
//   B[2m]     = (Re d_m0, Im d_m0, Re d_m1, ...)              -> Re s_nm
//   B[2m + 1] = (-Im d_m0, Re d_m0, -Im d_m1, ...)            -> Im s_nm
// over a reduction length 2L padded to a multiple of 16.  A block owns 128
// fingerprints (one per TMEM lane) and sweeps the dictionary in tiles of 64
// atoms (128 B rows): one elected thread issues tcgen05.mma (BF16 operands in
// shared memory, FP32 accumulators in TMEM, two accumulator buffers so the
// next tile's products overlap the scoring of this one), every warp reads its
// 32 lanes back with tcgen05.ld and keeps, per fingerprint, the best atoms by
// |s|^2 / ||d||^2 (8 for plain BF16 and FP8, 4 for the split form).  The candidates
// are then re-scored in FP32 from the original FP32 data and the best (ties to
// the lowest index) is kept, so BF16 rounding only has to keep the winner
// among the candidates.  No fingerprint x atom score reaches memory.
//
// Shared-memory operand layout: canonical K-major, no swizzle: 8-row x 16-byte
// core matrices, core (row group g, k chunk c) at byte (g * KC + c) * 128,
// KC = padded length / 8; descriptor LBO (next core along K) = 128 bytes, SBO
// (next 8-row group) = KC * 128 bytes.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.h"
#include "match.h"
#include "tc5.cuh"
#include "match_tc.cuh"

namespace mrf {

constexpr int kTcRows = 128;        // fingerprints per block (TMEM lanes)
constexpr int kTcAtoms = 64;        // atoms per tile (128 B rows, N = 128)
constexpr int kTcThreads = 256;       // 8 warps: two per TMEM lane quarter
// B operand of every atom tile, pre-arranged in the shared-memory layout:
// Bg[tile][2 kTcAtoms rows][Lp] (bf16), each atom scaled by the square root of
// its score weight so that the score is the plain |product|^2; padding atoms
// are zero rows.
__global__ void k_tc_prepare_b(const float2* __restrict__ dict, const float* __restrict__ wscore, int m, int len,
                               int Lp, int ntiles, int split, __nv_bfloat16* __restrict__ Bg) {
    const int KC = Lp / 8;
    const size_t per_tile = (size_t)2 * kTcAtoms * Lp;
    const size_t total = per_tile * ntiles;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int tile = (int)(e / per_tile);
        const int rem = (int)(e - (size_t)tile * per_tile);
        const int row = rem / Lp, kk = rem - row * Lp;   // logical (row, k) of the tile
        const int part = kk / (2 * len), k = kk - part * 2 * len;
        int at, imag;
        tile_row(row, &at, &imag);
        const int atom = tile * kTcAtoms + at;
        float v = 0.f;
        if (atom < m && part < split) {
            const float2 d = dict[(size_t)atom * len + (k >> 1)];
            if (!imag) v = (k & 1) ? d.y : d.x;                     // (Re d, Im d)  -> Re s
            else v = (k & 1) ? d.x : -d.y;                          // (-Im d, Re d) -> Im s
            v *= sqrtf(wscore[atom]);                               // |s|^2 w = |<sqrt(w) d, x>|^2
        }
        Bg[(size_t)tile * per_tile + core_off(row, kk, KC) / 2] =
            part < split ? split_part(v, part, false, split) : __float2bfloat16_rn(0.f);
    }
}

// FP8 (e4m3, kind::f8f6f4) operands: 8-bit core matrices are 8 rows x 16
// elements, so the k chunk is 16 elements and KC = padded length / 16.  The
// atoms' rows sqrt(w) d have unit norm (w = 1 / ||d||^2 and the compressed
// atom is no longer than the full one), so one factor 448 (the largest finite
// e4m3) brings every atom to the format's range; a fingerprint row is scaled
// by 448 / max |x|, which leaves its argmax unchanged.
constexpr float kE4m3Max = 448.f;

__host__ __device__ __forceinline__ uint32_t core_off8(int row, int k, int KC) {
    return (uint32_t)((((row >> 3) * KC + (k >> 4)) * 128) + ((row & 7) * 16) + (k & 15));
}

__device__ __forceinline__ unsigned char to_e4m3(float v) {
    return (unsigned char)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

__global__ void k_tc_prepare_b8(const float2* __restrict__ dict, const float* __restrict__ wscore, int m, int len,
                                int Lp, int ntiles, unsigned char* __restrict__ Bg) {
    const int KC = Lp / 16;
    const size_t per_tile = (size_t)2 * kTcAtoms * Lp;
    const size_t total = per_tile * ntiles;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int tile = (int)(e / per_tile);
        const int rem = (int)(e - (size_t)tile * per_tile);
        const int row = rem / Lp, k = rem - row * Lp;
        int at, imag;
        tile_row(row, &at, &imag);
        const int atom = tile * kTcAtoms + at;
        float v = 0.f;
        if (atom < m && k < 2 * len) {
            const float2 d = dict[(size_t)atom * len + (k >> 1)];
            if (!imag) v = (k & 1) ? d.y : d.x;
            else v = (k & 1) ? d.x : -d.y;
            v *= kE4m3Max * sqrtf(wscore[atom]);
        }
        Bg[(size_t)tile * per_tile + core_off8(row, k, KC)] = to_e4m3(v);
    }
}

// Starting threshold of a fingerprint's candidate list from TOPK seed atoms
// (in a loop: the previous call's candidates of the same row): the smallest
// FP32 score among them, less margin ||x||^2.  Any TOPK distinct atoms score
// at most the TOPK-th best, and the tensor-core score of an atom differs from
// its FP32 score by less than the margin (split BF16: |error| <~ 2^-12.6
// ||x||^2 from the operand splitting and the FP32 accumulation, margin
// 2^-10; BF16: <~ 2^-5.5, margin 2^-4), so every atom of the final top TOPK
// scores above the threshold and the list comes out exactly as from an empty
// start; only fewer insertions happen on the way.  -1 (no seeding) for seeds
// that are not TOPK distinct atoms, or an all-zero fingerprint.
template <int TOPK>
__device__ float seed_threshold(const float2* __restrict__ xr, int len, const int* sr,
                                const float2* __restrict__ dict, const float* __restrict__ wscore, int m,
                                float margin) {
    int a[TOPK];
#pragma unroll
    for (int q = 0; q < TOPK; ++q) {
        a[q] = sr[q];
        if (a[q] < 0 || a[q] >= m) return -1.f;
    }
#pragma unroll
    for (int q = 1; q < TOPK; ++q)
#pragma unroll
        for (int r = 0; r < q; ++r)
            if (a[q] == a[r]) return -1.f;
    float2 sq[TOPK];
    atom_products<TOPK>(xr, len, a, dict, m, sq);
    float x2 = 0.f;
    for (int k = 0; k < len; ++k) x2 += cabs2(xr[k]);       // (the row is in L1 by now)
    if (!(x2 > 1e-30f && x2 < 1e30f)) return -1.f;          // zero, tiny, huge or not finite
    float lo = 3.4e38f;
#pragma unroll
    for (int q = 0; q < TOPK; ++q) lo = fminf(lo, cabs2(sq[q]) * wscore[a[q]]);
    return lo - margin * x2;
}

// Warp-specialised sweep over tiles of kTcAtoms atoms.  Warp 8 (loader):
// streams each tile's B operand into a kTcStages-deep shared ring with one
// bulk copy per tile (mbarrier transaction count), as far ahead as the ring
// allows.  Warp 9 (MMA): issues each tile's MMAs into one of two TMEM
// accumulator buffers as soon as its operand has landed and the buffer is
// free.  Warps 0-7 (consumers, two per TMEM lane quarter, one column half
// each): wait for a buffer, copy all of it to registers, hand it back, then
// score.  Every wait is bounded; a wait that gives up sets the error word and
// the block stops once the copies and MMAs it issued have finished.  (The
// loader and MMA loops do not poll the shared error word: a shared-memory read
// per tile costs them several hundred cycles; a role whose partner stopped
// gives up at its own next wait.)
constexpr int kTcStages = 4;
constexpr int kTcConsumers = 8;
constexpr int kTcBlock = kTcThreads + 64;     // consumers, loader, MMA warp

// PREC: 1 = BF16, 3 = split BF16 (three copies along the reduction axis),
// 8 = FP8 e4m3.
template <int LP, int PREC, int TOPK>
__global__ void __launch_bounds__(kTcBlock, 2) k_match_tc(const float2* __restrict__ x, int n, int len,
                                                              const unsigned char* __restrict__ Bg, int ntiles,
                                                              const float* __restrict__ wscore, int m,
                                                              const float2* __restrict__ dict,
                                                              int* __restrict__ best_idx,
                                                              float2* __restrict__ best_ip, int* __restrict__ err,
                                                              const TcSlice* __restrict__ slices, int nslices,
                                                              const int* seed, int* cand_out) {
    constexpr bool F8 = PREC == 8;
    constexpr int SPLIT = PREC == 3 ? 3 : 1;
    constexpr int EB = F8 ? 1 : 2;                   // operand bytes
    constexpr int KC = LP * EB / 16;                 // 16-byte k chunks per row
    constexpr int A_BYTES = kTcRows * LP * EB;
    constexpr int B_BYTES = 2 * kTcAtoms * LP * EB;  // one tile: 2 rows per atom
    constexpr int NCOL = 2 * kTcAtoms;               // accumulator columns per buffer
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sA = smraw;
    unsigned char* sB = smraw + A_BYTES;             // [kTcStages][B_BYTES]
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bfull[kTcStages], s_bempty[kTcStages], s_afull[2], s_aempty[2];
    __shared__ int s_fail, s_loaded, s_mmas;
    __shared__ float s_ms[kTcRows][TOPK];
    __shared__ int s_mi[kTcRows][TOPK];
    __shared__ float s_rs[kTcRows];                  // FP8: row scale 448 / max |x|

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int n0 = blockIdx.x * kTcRows;
    if (nslices > 0) {
        // batched launch: the block's slice is the last one starting at or before it
        int si = 0;
        for (int q = 1; q < nslices; ++q)
            if (slices[q].block0 <= (int)blockIdx.x) si = q;
        x = slices[si].x;
        n = slices[si].n;
        best_idx = slices[si].best_idx;
        best_ip = slices[si].best_ip;
        Bg = slices[si].Bg;
        wscore = slices[si].wscore;
        dict = slices[si].dict;
        n0 = ((int)blockIdx.x - slices[si].block0) * kTcRows;
        if (n0 >= n) return;    // a launch sized for more rows than the slice holds (n written on the device)
        seed = F8 ? nullptr : slices[si].cand;
        cand_out = F8 ? nullptr : slices[si].cand;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        s_loaded = 0;
        s_mmas = 0;
        for (int q = 0; q < kTcStages; ++q) {
            mbar_init(smem_u32(&s_bfull[q]), 1);
            mbar_init(smem_u32(&s_bempty[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&s_afull[q]), 1);
            mbar_init(smem_u32(&s_aempty[q]), kTcConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // A tile.  Each thread loads a batch of 8 complex coefficients (the loads
    // in flight together) before it converts and stores them: a loop with one
    // dependent load per element waits out the memory latency per element.
    const int ncoef = kTcRows * len;                 // complex coefficients of the tile
    auto load_batch = [&](int b0, float2 (&xv)[8]) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = b0 + u * (int)blockDim.x;
            const int row = i / len, kc = i - row * len;
            xv[u] = (i < ncoef && n0 + row < n) ? x[(size_t)(n0 + row) * len + kc] : make_float2(0.f, 0.f);
        }
    };
    if (F8) {
        // FP8: rows scaled by 448 / max |x| (zero rows past n, zero padding past 2 len)
        for (int row = tid; row < kTcRows; row += blockDim.x) {
            float mx = 0.f;
            if (n0 + row < n)
                for (int k = 0; k < len; ++k) {
                    const float2 xv = x[(size_t)(n0 + row) * len + k];
                    mx = fmaxf(mx, fmaxf(fabsf(xv.x), fabsf(xv.y)));
                }
            s_rs[row] = mx > 0.f ? kE4m3Max / mx : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < kTcRows * (LP - 2 * len); e += blockDim.x) {
            const int w = LP - 2 * len, row = e / w;
            sA[core_off8(row, 2 * len + (e - row * w), KC)] = 0;
        }
        for (int b0 = tid; b0 < ncoef; b0 += 8 * (int)blockDim.x) {
            float2 xv[8];
            load_batch(b0, xv);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = b0 + u * (int)blockDim.x;
                if (i >= ncoef) break;
                const int row = i / len, kc = i - row * len;
                sA[core_off8(row, 2 * kc, KC)] = to_e4m3(xv[u].x * s_rs[row]);
                sA[core_off8(row, 2 * kc + 1, KC)] = to_e4m3(xv[u].y * s_rs[row]);
            }
        }
    } else {
        // BF16: the SPLIT copies of the 2 len coefficients (zero rows past n,
        // zero padding past them)
        const int used = SPLIT * 2 * len;
        for (int e = tid; e < kTcRows * (LP - used); e += blockDim.x) {
            const int w = LP - used, row = e / w;
            *reinterpret_cast<__nv_bfloat16*>(sA + core_off(row, used + (e - row * w), KC)) = __float2bfloat16_rn(0.f);
        }
        for (int b0 = tid; b0 < ncoef; b0 += 8 * (int)blockDim.x) {
            float2 xv[8];
            load_batch(b0, xv);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = b0 + u * (int)blockDim.x;
                if (i >= ncoef) break;
                const int row = i / len, kc = i - row * len;
#pragma unroll
                for (int part = 0; part < SPLIT; ++part) {
                    // (Re, Im) are neighbours in one 16-byte chunk: one 4-byte store
                    __nv_bfloat162 pr;
                    pr.x = split_part(xv[u].x, part, true, SPLIT);
                    pr.y = split_part(xv[u].y, part, true, SPLIT);
                    *reinterpret_cast<__nv_bfloat162*>(sA + core_off(row, part * 2 * len + 2 * kc, KC)) = pr;
                }
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    float cs[TOPK];
    int ci[TOPK];
#pragma unroll
    for (int q = 0; q < TOPK; ++q) { cs[q] = -1.f; ci[q] = 0x7fffffff; }

    if (warp == kTcConsumers) {
        // ------------------------------- loader -------------------------------
        if (lane == 0) {
            int loaded = 0;
            for (int tile = 0; tile < ntiles; ++tile) {
                const int st = tile % kTcStages;
                // the stage is free once the MMAs of tile - kTcStages have read it
                if (tile >= kTcStages &&
                    !wait_parity(smem_u32(&s_bempty[st]), (tile / kTcStages - 1) & 1)) {
                    s_fail = 1;
                    break;
                }
                const uint32_t bar = smem_u32(&s_bfull[st]);
                mbar_expect_tx(bar, B_BYTES);
                bulk_g2s(smem_u32(sB + st * B_BYTES), Bg + (size_t)tile * B_BYTES, B_BYTES, bar);
                loaded = tile + 1;
            }
            s_loaded = loaded;
        }
        __syncwarp();
    } else if (warp == kTcConsumers + 1) {
        // --------------------------------- MMA --------------------------------
        if (lane == 0) {
            // kind::f16 BF16 x BF16, or kind::f8f6f4 E4M3 x E4M3 (format code 0)
            const uint32_t idesc = F8 ? mma_idesc_f16(kTcRows, NCOL) : mma_idesc(kTcRows, NCOL);
            int mmas = 0;
            for (int tile = 0; tile < ntiles; ++tile) {
                const int st = tile % kTcStages, buf = tile & 1;
                if (!wait_parity(smem_u32(&s_bfull[st]), (tile / kTcStages) & 1)) { s_fail = 1; break; }
                if (tile >= 2 && !wait_parity(smem_u32(&s_aempty[buf]), ((tile >> 1) - 1) & 1)) {
                    s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t tm = tmem + (uint32_t)(buf * NCOL);
                const uint32_t bbase = smem_u32(sB + st * B_BYTES);
#pragma unroll
                // one MMA consumes 32 bytes of each row: 16 BF16 or 32 FP8 elements
                for (int ks = 0; ks < LP * EB / 32; ++ks) {
                    const uint64_t ad = smem_desc(smem_u32(sA) + ks * 256, 128, KC * 128);
                    const uint64_t bd = smem_desc(bbase + ks * 256, 128, KC * 128);
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    if (F8)
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tm),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    else
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tm),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
                mmas = tile + 1;
                mma_commit(smem_u32(&s_afull[buf]));
                mma_commit(smem_u32(&s_bempty[st]));
            }
            // every issued MMA must finish before the block releases TMEM or
            // its shared memory, also when a wait gave up (bounded again)
            if (mmas > 0) {
                const int last = mmas - 1;
                if (!wait_parity(smem_u32(&s_bempty[last % kTcStages]), (last / kTcStages) & 1)) s_fail = 1;
            }
            s_mmas = mmas;
        }
        __syncwarp();
    } else {
        // ------------------------------ consumers -----------------------------
        const int lq = warp & 3, half = warp >> 2;
        if (!F8 && seed) {
            constexpr float kMargin = PREC == 3 ? 0x1p-10f : 0x1p-4f;
            const int row = n0 + lq * 32 + lane;
            const float thr = row < n ? seed_threshold<TOPK>(x + (size_t)row * len, len, seed + (size_t)row * kTopK,
                                                             dict, wscore, m, kMargin)
                                      : -1.f;
#pragma unroll
            for (int q = 0; q < TOPK; ++q) cs[q] = thr;
        }
        for (int tile = 0; tile < ntiles; ++tile) {
            const int buf = tile & 1;
            // (the warp leaves together: its votes and aligned TMEM loads name every lane)
            if (!__all_sync(0xffffffffu, wait_parity(smem_u32(&s_afull[buf]), (tile >> 1) & 1))) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t taddr = tmem + (uint32_t)(buf * NCOL) + ((uint32_t)(lq * 32) << 16) +
                                   (uint32_t)(half * (NCOL / 2));
            // A lane meets its atoms in increasing index order, so "strictly
            // greater score" ranks a newcomer below equal earlier atoms: the
            // list stays the top TOPK by (score, then lowest index).  The list
            // settles slowly (a newcomer enters with probability ~TOPK / atoms
            // seen, and a seeded threshold starts it near its final level), so
            // a group of 8 atoms is tested against the threshold with one
            // maximum and one vote, and the insertion runs only when some lane
            // of the warp needs it.  The whole accumulator half (4 groups of 8
            // atoms) is copied to registers first, so the buffer goes back to
            // the MMA warp before the scoring.
            const int a0 = tile * kTcAtoms + half * (kTcAtoms / 2);
            auto score = [&](const uint32_t (&v)[16], int ab) {
                // v[0..7]: Re of the group's 8 atoms, v[8..15]: their Im
                float2 sc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    sc[u] = abs2_pair(make_float2(__uint_as_float(v[2 * u]), __uint_as_float(v[2 * u + 1])),
                                      make_float2(__uint_as_float(v[8 + 2 * u]), __uint_as_float(v[9 + 2 * u])));
                const float mx = fmaxf(fmaxf(fmaxf(sc[0].x, sc[0].y), fmaxf(sc[1].x, sc[1].y)),
                                       fmaxf(fmaxf(sc[2].x, sc[2].y), fmaxf(sc[3].x, sc[3].y)));
                if (__any_sync(0xffffffffu, mx > cs[TOPK - 1])) {
#pragma unroll
                    for (int h = 0; h < 8; ++h) {
                        const float s1 = (h & 1) ? sc[h >> 1].y : sc[h >> 1].x;
                        if (s1 > cs[TOPK - 1]) {
                            cs[TOPK - 1] = s1;
                            ci[TOPK - 1] = ab + h;
#pragma unroll
                            for (int r = TOPK - 1; r > 0; --r) {
                                if (cs[r] > cs[r - 1]) {
                                    const float ts = cs[r]; cs[r] = cs[r - 1]; cs[r - 1] = ts;
                                    const int ti = ci[r]; ci[r] = ci[r - 1]; ci[r - 1] = ti;
                                }
                            }
                        }
                    }
                }
            };
            uint32_t va[16], vb[16], vc[16], vd[16];
            tmem_ld16(va, taddr);
            tmem_ld16(vb, taddr + 16u);
            tmem_ld16(vc, taddr + 32u);
            tmem_ld16(vd, taddr + 48u);
            tmem_wait16(va, cs[TOPK - 1]);                  // waits for all four copies
            tmem_wait16(vb, cs[TOPK - 1]);
            tmem_wait16(vc, cs[TOPK - 1]);
            tmem_wait16(vd, cs[TOPK - 1]);
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_aempty[buf]));
            score(va, a0);
            score(vb, a0 + 8);
            score(vc, a0 + 16);
            score(vd, a0 + 24);
            if (*(volatile int*)&s_fail) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // copies that landed for no MMA (a wait gave up): let them finish before
    // the block's shared memory goes (bounded)
    if (warp == kTcConsumers && lane == 0)
        for (int t = s_mmas; t < s_loaded; ++t) wait_parity(smem_u32(&s_bfull[t % kTcStages]), (t / kTcStages) & 1);
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NCOL));
    }
    if (s_fail) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    if (warp >= kTcConsumers) return;
    // merge the two column halves' candidate lists of each fingerprint
    const int lq = warp & 3, half = warp >> 2;
    const int lrow = lq * 32 + lane;
    if (half == 1) {
#pragma unroll
        for (int q = 0; q < TOPK; ++q) { s_ms[lrow][q] = cs[q]; s_mi[lrow][q] = ci[q]; }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kTcThreads));     // consumer warps only
    if (half == 1) return;
#pragma unroll
    for (int q = 0; q < TOPK; ++q) {
        const float sc = s_ms[lrow][q];
        const int a = s_mi[lrow][q];
        if (better_cand(sc, a, cs[TOPK - 1], ci[TOPK - 1])) {
            cs[TOPK - 1] = sc;
            ci[TOPK - 1] = a;
#pragma unroll
            for (int r = TOPK - 1; r > 0; --r) {
                if (better_cand(cs[r], ci[r], cs[r - 1], ci[r - 1])) {
                    const float ts = cs[r]; cs[r] = cs[r - 1]; cs[r - 1] = ts;
                    const int ti = ci[r]; ci[r] = ci[r - 1]; ci[r - 1] = ti;
                }
            }
        }
    }
    // FP32 re-rank of the candidates from the original data
    const int row = n0 + lrow;
    if (row >= n) return;
    if (cand_out)
#pragma unroll
        for (int q = 0; q < TOPK; ++q) cand_out[(size_t)row * kTopK + q] = ci[q];
    float2 sp[TOPK];
    atom_products<TOPK>(x + (size_t)row * len, len, ci, dict, m, sp);
    float bs = -1.f;
    int bi = 0x7fffffff;
    float2 bip = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < TOPK; ++q) {
        const int a = ci[q];
        if (a >= m) continue;
        const float sc = cabs2(sp[q]) * wscore[a];
        if (better_cand(sc, a, bs, bi)) { bs = sc; bi = a; bip = sp[q]; }
    }
    // no finite best score (NaN or infinite entries): index 0, PD 0, like an all-zero x
    const bool found = bi < m && isfinite(bs);
    best_idx[row] = found ? bi : 0;
    best_ip[row] = found ? bip : make_float2(0.f, 0.f);
}

// reduction length: 2 len real coefficients (times 3 for the split form),
// padded to a multiple of 16 (BF16) or 32 (FP8) elements
static int padded_len(int len, int prec) {
    return prec == 8 ? (2 * len + 31) / 32 * 32 : (2 * len * prec + 15) / 16 * 16;
}

size_t tc_operand_bytes(int m, int len, int prec) {
    const int ntiles = (m + kTcAtoms - 1) / kTcAtoms;
    return (size_t)(prec == 8 ? 1 : 2) * ntiles * 2 * kTcAtoms * padded_len(len, prec);
}

static mrf_status tc_launch(MatchWorkspace& ws, const float2* x, int n, int blocks, const TcSlice* slices,
                            int nslices, int len, const float2* dict, int m, int prec, cudaStream_t s,
                            int* cand_io = nullptr);

mrf_status match_tc_candidates(MatchWorkspace& ws, const float2* x, int n, int len, const float2* dict, int m,
                               int prec, cudaStream_t s, int* cand_io) {
    return tc_launch(ws, x, n, (n + kTcRows - 1) / kTcRows, nullptr, 0, len, dict, m, prec, s, cand_io);
}

mrf_status match_tc_batch(MatchWorkspace& ws, const TcSlice* d_slices, int nslices, int total_blocks, int len,
                          int m, int prec, cudaStream_t s) {
    MRF_REQUIRE(d_slices && nslices >= 1, "batched matching: empty slice table");
    MRF_REQUIRE(ws.tc_b && ws.tc_m == m && ws.tc_len == len && ws.tc_split == prec,
                "batched matching: the operands were not prepared");
    return tc_launch(ws, nullptr, 0, total_blocks, d_slices, nslices, len, nullptr, m, prec, s);
}

mrf_status tc_prepare_operand(MatchWorkspace& ws, const float2* dict, int m, int len, int prec, cudaStream_t s) {
    MRF_REQUIRE(prec == 1 || prec == 3 || prec == 8, "tensor-core matching: unknown operand form %d", prec);
    MRF_REQUIRE(padded_len(len, prec) <= 128,
                "tensor-core matching supports a padded reduction length of at most 128 (length %d)", len);
    const int Lp = padded_len(len, prec);
    const int ntiles = (m + kTcAtoms - 1) / kTcAtoms;
    const size_t bbytes = tc_operand_bytes(m, len, prec);
    if (ws.tc_b == nullptr || ws.tc_b_bytes < bbytes || ws.tc_dict != dict || ws.tc_m != m || ws.tc_len != len ||
        ws.tc_split != prec) {
        if (ws.tc_b_bytes < bbytes) {
            MRF_REQUIRE(!ws.borrowed, "tensor-core matching: the dictionary operand does not fit the scratch");
            if (ws.tc_b) cudaFree(ws.tc_b);
            ws.tc_b = nullptr;
            MRF_CUDA(cudaMalloc(&ws.tc_b, bbytes));
            ws.tc_b_bytes = bbytes;
        }
        if (prec == 8) {
            k_tc_prepare_b8<<<1024, 256, 0, s>>>(dict, ws.wscore, m, len, Lp, ntiles,
                                                 reinterpret_cast<unsigned char*>(ws.tc_b));
            MRF_LAUNCHED_AS("k_tc_prepare_b8", s);
        } else {
            k_tc_prepare_b<<<1024, 256, 0, s>>>(dict, ws.wscore, m, len, Lp, ntiles, prec,
                                                reinterpret_cast<__nv_bfloat16*>(ws.tc_b));
            MRF_LAUNCHED_AS("k_tc_prepare_b", s);
        }
        ws.tc_dict = dict;
        ws.tc_m = m;
        ws.tc_len = len;
        ws.tc_split = prec;
    }
    if (!ws.tc_err) {
        MRF_CUDA(cudaMalloc(&ws.tc_err, sizeof(int)));
        MRF_CUDA(cudaMemsetAsync(ws.tc_err, 0, sizeof(int), s));
    }
    return MRF_OK;
}

static mrf_status tc_launch(MatchWorkspace& ws, const float2* x, int n, int blocks, const TcSlice* slices,
                            int nslices, int len, const float2* dict, int m, int prec, cudaStream_t s,
                            int* cand_io) {
    if (!slices) MRF_PROPAGATE(tc_prepare_operand(ws, dict, m, len, prec, s));
    int* cand = (!slices && prec != 8) ? cand_io : nullptr;     // seeds in, candidates out
    const int Lp = padded_len(len, prec);
    const int ntiles = (m + kTcAtoms - 1) / kTcAtoms;
    if (blocks == 0) return MRF_OK;
#define MRF_TC_LAUNCH(LPV, PR)                                                                                   \
    do {                                                                                                         \
        constexpr int TK = PR == 3 ? 4 : kTopK;                                                                  \
        constexpr int EBV = PR == 8 ? 1 : 2;                                                                     \
        const size_t sm = (size_t)kTcRows * LPV * EBV + (size_t)kTcStages * 2 * kTcAtoms * LPV * EBV;            \
        MRF_CUDA(cudaFuncSetAttribute(k_match_tc<LPV, PR, TK>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                      (int)sm));                                                                 \
        k_match_tc<LPV, PR, TK><<<blocks, kTcBlock, sm, s>>>(x, n, len,                                   \
                                                               reinterpret_cast<const unsigned char*>(ws.tc_b),  \
                                                               ntiles, ws.wscore, m, dict, ws.best_idx,          \
                                                               ws.best_ip, ws.tc_err, slices, nslices, cand,     \
                                                               cand);                                            \
    } while (0)
    if (prec == 1) {
        if (Lp == 16) MRF_TC_LAUNCH(16, 1);
        else if (Lp == 32) MRF_TC_LAUNCH(32, 1);
        else if (Lp == 48) MRF_TC_LAUNCH(48, 1);
        else if (Lp == 64) MRF_TC_LAUNCH(64, 1);
        else if (Lp == 96) MRF_TC_LAUNCH(96, 1);
        else MRF_TC_LAUNCH(128, 1);
    } else if (prec == 3) {
        if (Lp == 16) MRF_TC_LAUNCH(16, 3);
        else if (Lp == 32) MRF_TC_LAUNCH(32, 3);
        else if (Lp == 48) MRF_TC_LAUNCH(48, 3);
        else if (Lp == 64) MRF_TC_LAUNCH(64, 3);
        else if (Lp == 80) MRF_TC_LAUNCH(80, 3);
        else if (Lp == 96) MRF_TC_LAUNCH(96, 3);
        else if (Lp == 112) MRF_TC_LAUNCH(112, 3);
        else MRF_TC_LAUNCH(128, 3);
    } else {
        if (Lp == 32) MRF_TC_LAUNCH(32, 8);
        else if (Lp == 64) MRF_TC_LAUNCH(64, 8);
        else if (Lp == 96) MRF_TC_LAUNCH(96, 8);
        else MRF_TC_LAUNCH(128, 8);
    }
#undef MRF_TC_LAUNCH
    MRF_LAUNCHED_AS("k_match_tc", s);
    return MRF_OK;
}

mrf_status match_rerank(MatchWorkspace&, const float2*, int, int, const float2*, cudaStream_t) {
    return MRF_OK;   // the FP32 re-rank is fused into k_match_tc
}

}  // namespace mrf

namespace mrf {

// One thread polls phase 0 of an mbarrier that nothing arrives on: the wait
// gives up after `limit` polls and raises the error word, like every bounded
// wait of the tensor-core kernels.
__global__ void k_wait_selftest(unsigned limit, int* __restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !wait_parity(smem_u32(&bar), 0, limit)) atomicExch(err, 2);
}

}  // namespace mrf

extern "C" mrf_status mrf_wait_selftest(int polls, mrf_stream stream) {
    using namespace mrf;
    MRF_REQUIRE(polls >= 1 && polls <= 65536, "mrf_wait_selftest: polls must be in [1, 65536]");
    cudaStream_t s = as_stream(stream);
    int* err = nullptr;
    MRF_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&err), sizeof(int), s));
    MRF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_wait_selftest<<<1, 32, 0, s>>>((unsigned)polls, err);
    MRF_LAUNCHED_AS("k_wait_selftest", s);
    int h = 0;
    MRF_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaFreeAsync(err, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    if (h == 2) {
        set_error("mrf_wait_selftest: the device wait gave up after %d polls", polls);
        return MRF_ETIMEOUT;
    }
    return MRF_OK;
}

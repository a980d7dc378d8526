// Dictionary matching (Eq. 5) of full-length fingerprints on the
// 5th-generation tensor cores.
//
// Same real GEMM as match_tc.cu (A = fingerprints as (Re, Im) pairs, B = two
// rows per atom giving Re and Im of <d_m, x>, atoms scaled by sqrt of their
// score weight), but the reduction length 2 len (up to 4096 reals, e.g. the
// 2000 of a 1000-frame fingerprint) is far too long to keep a 128-row
// fingerprint tile in shared memory.  Both operands are therefore streamed
// along the reduction axis in chunks of 64 BF16 elements (128 bytes per row):
// a block owns 128 fingerprints (TMEM lanes) and sweeps the dictionary in
// tiles of 128 atoms (256 accumulator columns, N = 256); for every tile it
// runs through all chunks, each a 16 KB fingerprint slab plus a 32 KB atom
// slab landed by bulk copies in a 4-deep ring, accumulating four
// 128 x 256 x 16 MMAs per chunk into one of two TMEM buffers (512 columns),
// so the next tile's products overlap the scoring of this one.  The scoring
// and the FP32 re-rank of the candidates are those of match_tc.cu.
//
// Split BF16 (PREC 3) sums A_hi B_hi + A_hi B_lo + A_lo B_hi: a chunk is 32
// elements and its stage holds both parts of both operands, so the three
// products of a chunk are issued from one stage and each part is fetched
// once per tile (BF16: 64-element chunks of the one part).  Either way a
// stage is a 16 KB fingerprint unit and a 32 KB atom unit.
//
// Global operand layout: chunk units pre-arranged in the canonical K-major
// core-matrix layout (8 rows x 16 bytes per core, KC = CH / 8 cores along a
// chunk of CH elements), so one bulk copy fills each half of a stage:
//   Ag[row block][chunk][part][128 rows][CH]
//   Bg[atom tile][chunk][part][256 rows][CH]   rows in tile_row order
// part = hi (and lo for the split form).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.h"
#include "match.h"
#include "match_tc.cuh"
#include "tc5.cuh"

namespace mrf {

constexpr int kLRows = 128;                      // fingerprints per block
constexpr int kLAtoms = 128;                     // atoms per tile
constexpr int kLCols = 2 * kLAtoms;              // accumulator columns per tile
constexpr int kLStages = 4;
constexpr int kLABytes = 16384;                  // fingerprint unit of a chunk: 128 rows x 128 bytes
constexpr int kLBBytes = 32768;                  // atom unit of a chunk: 256 rows x 128 bytes
// chunk length (elements) and parts per unit of an operand form
__host__ __device__ constexpr int tcl_ch(int prec) { return prec == 3 ? 32 : 64; }
__host__ __device__ constexpr int tcl_parts(int prec) { return prec == 3 ? 2 : 1; }
constexpr int kLConsumers = 8;
constexpr int kLThreads = 32 * kLConsumers + 64; // consumers, loader, MMA warp

// chunks of the reduction (the 2 len reals padded to a multiple of the chunk)
static inline int tcl_chunks(int len, int prec) { return (2 * len + tcl_ch(prec) - 1) / tcl_ch(prec); }

// 8 consecutive reals (one 16-byte core-matrix row) as BF16 hi or lo parts
__device__ __forceinline__ uint4 pack_parts(const float (&v)[8], int part, bool is_a) {
    uint4 o;
    uint32_t* w = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 p;
        p.x = split_part(v[2 * j], part, is_a, 3);
        p.y = split_part(v[2 * j + 1], part, is_a, 3);
        w[j] = *reinterpret_cast<uint32_t*>(&p);
    }
    return o;
}

// fingerprint unit (rb, c, part): part 0 hi = bf16(v), part 1 lo =
// bf16(v - hi); one thread per 8 reals of a row (4 complex loads, one 16-byte
// store)
template <int PREC>
__global__ void k_tcl_prepare_a(const float2* __restrict__ x, int n, int len, int C,
                                __nv_bfloat16* __restrict__ Ag, size_t total8) {
    constexpr int CH = tcl_ch(PREC), NP = tcl_parts(PREC), G8 = CH / 8;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total8; e += (size_t)gridDim.x * blockDim.x) {
        const size_t sub = e / (kLRows * G8);                 // (rb, c, part)
        const int rem = (int)(e - sub * (kLRows * G8));
        const int row = rem / G8, k8 = rem - row * G8;
        const int part = (int)(sub % NP);
        const size_t rc = sub / NP;
        const int rb = (int)(rc / C), c = (int)(rc - (size_t)rb * C);
        const int kk0 = c * CH + 8 * k8;
        const int gr = rb * kLRows + row;
        float v[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = (kk0 >> 1) + j;
            const float2 xv = (gr < n && q < len) ? x[(size_t)gr * len + q] : make_float2(0.f, 0.f);
            v[2 * j] = xv.x;
            v[2 * j + 1] = xv.y;
        }
        *reinterpret_cast<uint4*>(Ag + sub * (kLRows * CH) + core_off(row, 8 * k8, G8) / 2) =
            pack_parts(v, part == 0 ? 0 : 2, true);
    }
}

// atom unit (tile, c, part): rows in tile_row order, scaled by sqrt(score
// weight); one thread per 8 reals of a row
template <int PREC>
__global__ void k_tcl_prepare_b(const float2* __restrict__ dict, const float* __restrict__ wscore, int m, int len,
                                int C, __nv_bfloat16* __restrict__ Bg, size_t total8) {
    constexpr int CH = tcl_ch(PREC), NP = tcl_parts(PREC), G8 = CH / 8;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total8; e += (size_t)gridDim.x * blockDim.x) {
        const size_t sub = e / (kLCols * G8);
        const int rem = (int)(e - sub * (kLCols * G8));
        const int row = rem / G8, k8 = rem - row * G8;
        const int part = (int)(sub % NP);
        const size_t tc = sub / NP;
        const int tile = (int)(tc / C), c = (int)(tc - (size_t)tile * C);
        const int kk0 = c * CH + 8 * k8;
        int at, imag;
        tile_row(row, &at, &imag);
        const int atom = tile * kLAtoms + at;
        const float sw = atom < m ? sqrtf(wscore[atom]) : 0.f;
        float v[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = (kk0 >> 1) + j;
            const float2 d = (atom < m && q < len) ? dict[(size_t)atom * len + q] : make_float2(0.f, 0.f);
            // (Re d, Im d) -> Re s;  (-Im d, Re d) -> Im s
            v[2 * j] = (imag ? -d.y : d.x) * sw;
            v[2 * j + 1] = (imag ? d.x : d.y) * sw;
        }
        *reinterpret_cast<uint4*>(Bg + sub * (kLCols * CH) + core_off(row, 8 * k8, G8) / 2) =
            pack_parts(v, part == 0 ? 0 : 1, false);
    }
}

}  // namespace mrf

namespace mrf {

// Roles as in k_match_tc: warp 8 loads (one bulk copy each of the A and B
// slabs of a chunk into a ring stage), warp 9 issues the MMAs (one elected
// lane), warps 0-7 score (two per TMEM lane quarter, 128 columns = 64 atoms
// each, read in two batches of 64 columns).  Every wait is bounded; a wait
// that gives up sets the error word and the block drains what it issued.
// Block (rb, grp) sweeps atom tiles [grp tpg, (grp + 1) tpg) for row block rb
// (the split of the dictionary into tile groups evens out the waves of blocks
// over the SMs) and writes each row's TOPK candidates and their tensor-core
// scores for that group to cand_idx / cand_sc [n][groups][TOPK]; k_long_rerank
// merges the groups and re-scores in FP32.
template <int PREC, int TOPK>
__global__ void __launch_bounds__(kLThreads, 1)
    k_match_tc_long(int n, const unsigned char* __restrict__ Ag, const unsigned char* __restrict__ Bg, int C,
                    int ntiles, int tpg, int* __restrict__ cand_idx, float* __restrict__ cand_sc,
                    int* __restrict__ err) {
    constexpr int CH = tcl_ch(PREC);
    constexpr int KC = CH / 8;                         // core matrices along a chunk row
    constexpr int PART_A = kLRows * CH * 2;            // bytes of one part of the fingerprint unit
    constexpr int PART_B = kLCols * CH * 2;            // bytes of one part of the atom unit
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sA = smraw;                            // [kLStages][kLABytes]
    unsigned char* sB = smraw + kLStages * kLABytes;      // [kLStages][kLBBytes]
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[kLStages], s_empty[kLStages], s_afull[2], s_aempty[2];
    __shared__ int s_fail, s_loaded, s_mmas;
    __shared__ float s_ms[kLRows][TOPK];
    __shared__ int s_mi[kLRows][TOPK];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rb = blockIdx.x, n0 = rb * kLRows, grp = blockIdx.y, ngroups = gridDim.y;
    const int t0 = grp * tpg, nt = min(ntiles - t0, tpg);      // >= 1 by the launch
    const int NC = C;                         // chunks of one tile's reduction

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * kLCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        s_loaded = 0;
        s_mmas = 0;
        for (int q = 0; q < kLStages; ++q) {
            mbar_init(smem_u32(&s_full[q]), 1);
            mbar_init(smem_u32(&s_empty[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&s_afull[q]), 1);
            mbar_init(smem_u32(&s_aempty[q]), kLConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    const long long total = (long long)nt * NC;         // chunks over the group's sweep

    float cs[TOPK];
    int ci[TOPK];
#pragma unroll
    for (int q = 0; q < TOPK; ++q) { cs[q] = -1.f; ci[q] = 0x7fffffff; }

    if (warp == kLConsumers) {
        // ------------------------------- loader -------------------------------
        if (lane == 0) {
            long long loaded = 0;
            for (long long g = 0; g < total; ++g) {
                const int st = (int)(g % kLStages);
                if (g >= kLStages && !wait_parity(smem_u32(&s_empty[st]), (uint32_t)((g / kLStages - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                const int lt = (int)(g / NC), c = (int)(g - (long long)lt * NC), tile = t0 + lt;
                const uint32_t bar = smem_u32(&s_full[st]);
                mbar_expect_tx(bar, kLABytes + kLBBytes);
                bulk_g2s(smem_u32(sA + st * kLABytes), Ag + ((size_t)rb * C + c) * kLABytes, kLABytes, bar);
                bulk_g2s(smem_u32(sB + st * kLBBytes), Bg + ((size_t)tile * C + c) * kLBBytes, kLBBytes, bar);
                loaded = g + 1;
            }
            s_loaded = (int)loaded;
        }
        __syncwarp();
    } else if (warp == kLConsumers + 1) {
        // --------------------------------- MMA --------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = mma_idesc(kLRows, kLCols);
            long long done = 0;
            bool ok = true;
            for (int tile = 0; tile < nt && ok; ++tile) {
                const int buf = tile & 1;
                if (tile >= 2 && !wait_parity(smem_u32(&s_aempty[buf]), (uint32_t)(((tile >> 1) - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                const uint32_t tm = tmem + (uint32_t)(buf * kLCols);
                for (int c = 0; c < NC; ++c) {
                    const long long g = (long long)tile * NC + c;
                    const int st = (int)(g % kLStages);
                    if (!wait_parity(smem_u32(&s_full[st]), (uint32_t)((g / kLStages) & 1))) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t abase = smem_u32(sA + st * kLABytes), bbase = smem_u32(sB + st * kLBBytes);
                    // one K step is 16 elements = two cores along K (256 bytes);
                    // split: A_hi B_hi + A_hi B_lo + A_lo B_hi per step
#pragma unroll
                    for (int ks = 0; ks < CH / 16; ++ks) {
#pragma unroll
                        for (int pr = 0; pr < (PREC == 3 ? 3 : 1); ++pr) {
                            const uint32_t aoff = pr == 2 ? PART_A : 0, boff = pr == 1 ? PART_B : 0;
                            const uint64_t ad = smem_desc(abase + aoff + ks * 256, 128, KC * 128);
                            const uint64_t bd = smem_desc(bbase + boff + ks * 256, 128, KC * 128);
                            const uint32_t acc = (c > 0 || ks > 0 || pr > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tm),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
                    mma_commit(smem_u32(&s_empty[st]));
                    done = g + 1;
                }
                if (ok) mma_commit(smem_u32(&s_afull[buf]));
            }
            // every issued MMA finishes before the block releases TMEM or its
            // shared memory, also when a wait gave up (bounded again)
            if (done > 0) {
                const long long last = done - 1;
                if (!wait_parity(smem_u32(&s_empty[last % kLStages]), (uint32_t)((last / kLStages) & 1)))
                    s_fail = 1;
            }
            s_mmas = (int)done;
        }
        __syncwarp();
    } else {
        // ------------------------------ consumers -----------------------------
        const int lq = warp & 3, half = warp >> 2;
        for (int tile = 0; tile < nt; ++tile) {
            const int buf = tile & 1;
            // (the warp leaves together: its votes and aligned TMEM loads name every lane)
            if (!__all_sync(0xffffffffu, wait_parity(smem_u32(&s_afull[buf]), (uint32_t)((tile >> 1) & 1)))) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t tbase = tmem + (uint32_t)(buf * kLCols) + ((uint32_t)(lq * 32) << 16) +
                                   (uint32_t)(half * (kLCols / 2));
            auto score = [&](const uint32_t (&v)[16], int ab) {
                // v[0..7]: Re of the group's 8 atoms, v[8..15]: their Im; atoms
                // arrive in increasing index order, so "strictly greater"
                // keeps the list the top TOPK by (score, lowest index)
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
#pragma unroll
            for (int bt = 0; bt < 2; ++bt) {
                uint32_t va[16], vb[16], vc[16], vd[16];
                const uint32_t ta = tbase + (uint32_t)(bt * 64);
                tmem_ld16(va, ta);
                tmem_ld16(vb, ta + 16u);
                tmem_ld16(vc, ta + 32u);
                tmem_ld16(vd, ta + 48u);
                tmem_wait16(va, cs[TOPK - 1]);
                tmem_wait16(vb, cs[TOPK - 1]);
                tmem_wait16(vc, cs[TOPK - 1]);
                tmem_wait16(vd, cs[TOPK - 1]);
                if (bt == 1) {
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&s_aempty[buf]));
                }
                const int a0 = (t0 + tile) * kLAtoms + half * (kLAtoms / 2) + bt * 32;
                score(va, a0);
                score(vb, a0 + 8);
                score(vc, a0 + 16);
                score(vd, a0 + 24);
            }
            if (*(volatile int*)&s_fail) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // copies that landed for no MMA (a wait gave up): let them finish before
    // the block's shared memory goes (bounded)
    if (warp == kLConsumers && lane == 0)
        for (long long g = s_mmas; g < s_loaded; ++g)
            wait_parity(smem_u32(&s_full[g % kLStages]), (uint32_t)((g / kLStages) & 1));
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kLCols));
    }
    if (s_fail) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    if (warp >= kLConsumers) return;
    // merge the two column halves' candidate lists of each fingerprint
    const int lrow = (warp & 3) * 32 + lane;
    const int half = warp >> 2;
    if (half == 1) {
#pragma unroll
        for (int q = 0; q < TOPK; ++q) { s_ms[lrow][q] = cs[q]; s_mi[lrow][q] = ci[q]; }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kLConsumers));     // consumer warps only
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
    const int row = n0 + lrow;
    if (row >= n) return;
    const size_t o = ((size_t)row * ngroups + grp) * TOPK;
#pragma unroll
    for (int q = 0; q < TOPK; ++q) {
        cand_idx[o + q] = ci[q];
        cand_sc[o + q] = cs[q];
    }
}

}  // namespace mrf

namespace mrf {

// One warp per fingerprint: the TOPK best candidates over the groups' lists
// by tensor-core score (ties to the lower index), then their FP32 inner
// products over the full length with the lanes striding the length (each
// load of a dictionary row is one coalesced 256-byte warp access), summed by
// a shuffle tree; the best FP32 score wins (ties to the lower index), and a
// fingerprint whose best score is not finite gets index 0 and PD 0.
template <int TOPK>
__global__ void __launch_bounds__(256) k_long_rerank(const float2* __restrict__ x, int n, int len,
                                                     const float2* __restrict__ dict,
                                                     const float* __restrict__ wscore, int m,
                                                     const int* __restrict__ cand_idx,
                                                     const float* __restrict__ cand_sc, int ngroups,
                                                     int* __restrict__ best_idx, float2* __restrict__ best_ip) {
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float cs[TOPK];
    int ci[TOPK];
#pragma unroll
    for (int q = 0; q < TOPK; ++q) { cs[q] = -1.f; ci[q] = 0x7fffffff; }
    const int ne = ngroups * TOPK;
    for (int e = 0; e < ne; ++e) {
        const float sc = cand_sc[(size_t)row * ne + e];
        const int a = cand_idx[(size_t)row * ne + e];
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
    float2 sp[TOPK];
#pragma unroll
    for (int q = 0; q < TOPK; ++q) sp[q] = make_float2(0.f, 0.f);
    const float2* xr = x + (size_t)row * len;
    for (int k = lane; k < len; k += 32) {
        const float2 xv = xr[k];
#pragma unroll
        for (int q = 0; q < TOPK; ++q)
            if (ci[q] >= 0 && ci[q] < m) sp[q] = cadd(sp[q], cconjmul(dict[(size_t)ci[q] * len + k], xv));
    }
#pragma unroll
    for (int q = 0; q < TOPK; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sp[q].x += __shfl_xor_sync(0xffffffffu, sp[q].x, o);
            sp[q].y += __shfl_xor_sync(0xffffffffu, sp[q].y, o);
        }
    if (lane != 0) return;
    float bs = -1.f;
    int bi = 0x7fffffff;
    float2 bip = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < TOPK; ++q) {
        const int a = ci[q];
        if (a < 0 || a >= m) continue;
        const float sc = cabs2(sp[q]) * wscore[a];
        if (better_cand(sc, a, bs, bi)) { bs = sc; bi = a; bip = sp[q]; }
    }
    const bool found = bi < m && isfinite(bs);
    best_idx[row] = found ? bi : 0;
    best_ip[row] = found ? bip : make_float2(0.f, 0.f);
}

}  // namespace mrf

namespace mrf {

bool tc_long(int len, int prec) {
    // the resident-tile matcher holds a padded reduction of at most 128 elements
    const int lp = prec == 8 ? (2 * len + 31) / 32 * 32 : (2 * len * prec + 15) / 16 * 16;
    return lp > 128;
}

static size_t round1k(size_t b) { return (b + 1023) / 1024 * 1024; }

static size_t tcl_b_bytes(int m, int len, int prec) {
    const int ntiles = (m + kLAtoms - 1) / kLAtoms;
    return round1k((size_t)ntiles * tcl_chunks(len, prec) * kLBBytes);
}

static size_t tcl_a_bytes(int n, int len, int prec) {
    const int nrb = (n + kLRows - 1) / kLRows;
    return round1k((size_t)nrb * tcl_chunks(len, prec) * kLABytes);
}

constexpr int kLMaxGroups = 8;

static size_t tcl_cand_bytes(int n) { return 2 * round1k((size_t)n * kLMaxGroups * kTopK * 4); }

size_t tc_long_scratch_bytes(int n, int m, int len, int prec) {
    return tcl_b_bytes(m, len, prec) + tcl_a_bytes(n, len, prec) + tcl_cand_bytes(n);
}

// tile groups per row block: the fewest groups whose blocks fill the SMs'
// waves within 3 % of the best split (each block holds one SM: 192 KB of
// shared memory and all 512 TMEM columns)
static int tcl_groups(int nrb, int ntiles) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 148;
    double best = 0.0;
    int pick = 1;
    double effs[kLMaxGroups + 1] = {};
    for (int g = 1; g <= std::min(kLMaxGroups, ntiles); ++g) {
        const int tpg = (ntiles + g - 1) / g;
        const int gg = (ntiles + tpg - 1) / tpg;
        const long long units = (long long)nrb * gg;
        const long long waves = (units + sms - 1) / sms;
        effs[g] = (double)nrb * ntiles / ((double)waves * sms * tpg);
        best = std::max(best, effs[g]);
    }
    for (int g = 1; g <= std::min(kLMaxGroups, ntiles); ++g)
        if (effs[g] >= 0.97 * best) { pick = g; break; }
    return pick;
}

mrf_status match_tc_long(MatchWorkspace& ws, const float2* x, int n, int len, const float2* dict, int m, int prec,
                         cudaStream_t s) {
    MRF_REQUIRE(prec == 1 || prec == 3,
                "tensor-core matching of fingerprints longer than the resident tile needs BF16 or split BF16 "
                "(got operand form %d)", prec);
    const int C = tcl_chunks(len, prec);
    const int ntiles = (m + kLAtoms - 1) / kLAtoms;
    const int nrb = (n + kLRows - 1) / kLRows;
    const size_t bb = tcl_b_bytes(m, len, prec), ab = tcl_a_bytes(n, len, prec);
    const size_t need = bb + ab + tcl_cand_bytes(n);
    if (ws.tc_b_bytes < need) {
        MRF_REQUIRE(!ws.borrowed, "tensor-core matching: the operands do not fit the scratch");
        if (ws.tc_b) cudaFree(ws.tc_b);
        ws.tc_b = nullptr;
        ws.tc_dict = nullptr;
        MRF_CUDA(cudaMalloc(&ws.tc_b, need));
        ws.tc_b_bytes = need;
    }
    if (!ws.tc_err) {
        MRF_CUDA(cudaMalloc(&ws.tc_err, sizeof(int)));
        MRF_CUDA(cudaMemsetAsync(ws.tc_err, 0, sizeof(int), s));
    }
    unsigned char* Bg = static_cast<unsigned char*>(ws.tc_b);
    unsigned char* Ag = Bg + bb;
    int* cidx = reinterpret_cast<int*>(Ag + ab);
    float* csc = reinterpret_cast<float*>(Ag + ab + tcl_cand_bytes(n) / 2);
    const int tag = 16 + prec;            // marks the streamed layout in the operand cache
    if (ws.tc_dict != dict || ws.tc_m != m || ws.tc_len != len || ws.tc_split != tag) {
        // 8 reals per thread: units x parts x rows x CH / 8 = units x 16384 / 8
        const size_t tb = (size_t)ntiles * C * (kLBBytes / 16);
        if (prec == 3)
            k_tcl_prepare_b<3><<<2048, 256, 0, s>>>(dict, ws.wscore, m, len, C,
                                                   reinterpret_cast<__nv_bfloat16*>(Bg), tb);
        else
            k_tcl_prepare_b<1><<<2048, 256, 0, s>>>(dict, ws.wscore, m, len, C,
                                                   reinterpret_cast<__nv_bfloat16*>(Bg), tb);
        MRF_LAUNCHED_AS("k_tcl_prepare_b", s);
        ws.tc_dict = dict;
        ws.tc_m = m;
        ws.tc_len = len;
        ws.tc_split = tag;
    }
    const size_t ta = (size_t)nrb * C * (kLABytes / 16);
    if (prec == 3)
        k_tcl_prepare_a<3><<<2048, 256, 0, s>>>(x, n, len, C, reinterpret_cast<__nv_bfloat16*>(Ag), ta);
    else
        k_tcl_prepare_a<1><<<2048, 256, 0, s>>>(x, n, len, C, reinterpret_cast<__nv_bfloat16*>(Ag), ta);
    MRF_LAUNCHED_AS("k_tcl_prepare_a", s);
    const int g = tcl_groups(nrb, ntiles);
    const int tpg = (ntiles + g - 1) / g, ngroups = (ntiles + tpg - 1) / tpg;
    const dim3 grid((unsigned)nrb, (unsigned)ngroups);
    const size_t sm = (size_t)kLStages * (kLABytes + kLBBytes);
    const unsigned rblocks = (unsigned)(((size_t)n * 32 + 255) / 256);
    if (prec == 3) {
        MRF_CUDA(cudaFuncSetAttribute(k_match_tc_long<3, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_match_tc_long<3, 4><<<grid, kLThreads, sm, s>>>(n, Ag, Bg, C, ntiles, tpg, cidx, csc, ws.tc_err);
        MRF_LAUNCHED_AS("k_match_tc_long", s);
        k_long_rerank<4><<<rblocks, 256, 0, s>>>(x, n, len, dict, ws.wscore, m, cidx, csc, ngroups, ws.best_idx,
                                                 ws.best_ip);
    } else {
        MRF_CUDA(cudaFuncSetAttribute(k_match_tc_long<1, kTopK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm));
        k_match_tc_long<1, kTopK><<<grid, kLThreads, sm, s>>>(n, Ag, Bg, C, ntiles, tpg, cidx, csc, ws.tc_err);
        MRF_LAUNCHED_AS("k_match_tc_long", s);
        k_long_rerank<kTopK><<<rblocks, 256, 0, s>>>(x, n, len, dict, ws.wscore, m, cidx, csc, ngroups,
                                                     ws.best_idx, ws.best_ip);
    }
    MRF_LAUNCHED_AS("k_long_rerank", s);
    return MRF_OK;
}

}  // namespace mrf

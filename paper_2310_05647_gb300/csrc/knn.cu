// Exact k nearest patches (the sparse patch graph of Eq. 7; distances between
// patches of the matched (T1, T2) maps, Eq. 7-10).
//
// Patch vectors are 12-bit fixed point integers f in [0, 4096] (one per voxel
// and map), so every squared distance is an exact integer and ties (common:
// matched maps are piecewise constant) break to the lower index on every
// device.  For fd <= 128 the all-pairs distances come from the tensor cores:
//   d_ij = |c_i|^2 + |c_j|^2 - 2 c_i . c_j,   c = f - 2048 in [-2048, 2048]
// with c_j = 32 h_j + l_j, h in [-64, 64], l in [-16, 15], so that
//   c_i . c_j = 32 (c_i . h_j) + (c_i . l_j).
// c, h and l are integers exact in FP16; |c_i . h_j| <= fd 2^17 <= 2^24 and
// |c_i . l_j| <= fd 2^15, so each FP32 accumulator holds an exact integer and
// the distance is assembled exactly in 32-bit integer arithmetic (d < 2^32
// for fd <= 255).  The candidate operand interleaves (h_j, l_j) as the two B
// rows of candidate j, one GEMM with N = 2 x 64 per 64-candidate tile.
//
// A block owns 128 query patches (one per TMEM lane) and one partition of the
// candidates; warp-specialised like the dictionary matcher (a producer warp
// streams 64-candidate operand tiles with bulk copies into a 2-stage ring and
// issues the MMAs into two TMEM accumulator buffers; eight consumer warps,
// two per lane quarter, one candidate half each, keep a sorted list per query).
// k_knn_merge then merges the partitions' lists.
#include <cuda_fp16.h>

#include <algorithm>

#include "common.h"
#include "knn.h"
#include "mrf.h"
#include "tc5.cuh"

namespace mrf {

constexpr int kKnRows = 128;        // queries per block (TMEM lanes)
constexpr int kKnTile = 64;         // candidates per tile (2 B rows each, N = 128)
constexpr int kKnStages = 2;
constexpr int kKnConsumers = 8;
constexpr int kKnThreads = 32 * kKnConsumers;
constexpr int kKnCentre = 2048;
constexpr int kKnMaxTcFd = 128;
constexpr int kKnMaxParts = 16;

__device__ __forceinline__ bool less_dj(unsigned d, int j, unsigned d2, int j2) {
    return d < d2 || (d == d2 && j < j2);
}

// SIMT path (long patch vectors, fd > 128).  k_knn_part: block = 32 query
// patches x one candidate
// partition; 8 threads per query each scan every 8th candidate of each
// 64-candidate tile, 4 candidates at a time with 16-byte shared loads, keep
// their KMAX best and merge them with shuffles into the partition's best knn.
// k_knn_merge: one thread per query merges the partitions' sorted lists.
// Feature rows are padded with zeros to a multiple of 4 (FD4).
template <int KMAX>
__global__ void __launch_bounds__(256) k_knn_part(const int* __restrict__ F, int np, int FD4, int knn,
                                                  int cand_per_part, int* __restrict__ pnbr,
                                                  unsigned* __restrict__ pd2) {
    extern __shared__ int4 shf4[];
    int* shf = reinterpret_cast<int*>(shf4);
    const int ld = FD4 + 4;
    int* Fq = shf;              // [32][ld]
    int* Fc = shf + 32 * ld;    // [64][ld]
    const int ql = threadIdx.x >> 3, sub = threadIdx.x & 7;
    const int q = blockIdx.x * 32 + ql;
    const int part = blockIdx.y;
    const int cb = part * cand_per_part, ce = min(np, cb + cand_per_part);
    const int v4 = FD4 >> 2;
    for (int i = threadIdx.x; i < 32 * v4; i += blockDim.x) {
        const int r = i / v4, c = i - r * v4;
        const int qq = blockIdx.x * 32 + r;
        const int4 v = qq < np ? reinterpret_cast<const int4*>(F + (size_t)qq * FD4)[c] : make_int4(0, 0, 0, 0);
        *reinterpret_cast<int4*>(Fq + r * ld + 4 * c) = v;
    }
    unsigned bd[KMAX];
    int bj[KMAX];
#pragma unroll
    for (int i = 0; i < KMAX; ++i) { bd[i] = 0xffffffffu; bj[i] = 0x7fffffff; }
    for (int c0 = cb; c0 < ce; c0 += 64) {
        __syncthreads();
        for (int i = threadIdx.x; i < 64 * v4; i += blockDim.x) {
            const int r = i / v4, c = i - r * v4;
            const int4 v = c0 + r < ce ? reinterpret_cast<const int4*>(F + (size_t)(c0 + r) * FD4)[c]
                                       : make_int4(0, 0, 0, 0);
            *reinterpret_cast<int4*>(Fc + r * ld + 4 * c) = v;
        }
        __syncthreads();
        if (q < np) {
#pragma unroll
            for (int grp = 0; grp < 2; ++grp) {
                unsigned d[4] = {0u, 0u, 0u, 0u};
                const int* a = Fq + ql * ld;
                for (int t = 0; t < FD4; t += 4) {
                    const int4 av = *reinterpret_cast<const int4*>(a + t);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int4 bv = *reinterpret_cast<const int4*>(Fc + (sub + 8 * (4 * grp + u)) * ld + t);
                        const int e0 = av.x - bv.x, e1 = av.y - bv.y, e2 = av.z - bv.z, e3 = av.w - bv.w;
                        d[u] += (unsigned)(e0 * e0) + (unsigned)(e1 * e1) + (unsigned)(e2 * e2) +
                                (unsigned)(e3 * e3);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = c0 + sub + 8 * (4 * grp + u);
                    if (j >= ce || j == q) continue;
                    if (less_dj(d[u], j, bd[KMAX - 1], bj[KMAX - 1])) {
                        bd[KMAX - 1] = d[u];
                        bj[KMAX - 1] = j;
#pragma unroll
                        for (int i = KMAX - 1; i > 0; --i) {
                            if (less_dj(bd[i], bj[i], bd[i - 1], bj[i - 1])) {
                                const unsigned td = bd[i]; bd[i] = bd[i - 1]; bd[i - 1] = td;
                                const int tj = bj[i]; bj[i] = bj[i - 1]; bj[i - 1] = tj;
                            }
                        }
                    }
                }
            }
        }
    }
    // merge the 8 sorted lists of this query into the partition's best knn
    for (int r = 0; r < knn; ++r) {
        unsigned d = bd[0];
        int j = bj[0];
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            const unsigned d2 = __shfl_xor_sync(0xffffffffu, d, o);
            const int j2 = __shfl_xor_sync(0xffffffffu, j, o);
            if (less_dj(d2, j2, d, j)) { d = d2; j = j2; }
        }
        if (bj[0] == j) {
#pragma unroll
            for (int i = 0; i < KMAX - 1; ++i) { bd[i] = bd[i + 1]; bj[i] = bj[i + 1]; }
            bd[KMAX - 1] = 0xffffffffu;
            bj[KMAX - 1] = 0x7fffffff;
        }
        if (sub == 0 && q < np) {
            pnbr[((size_t)part * np + q) * knn + r] = j;
            pd2[((size_t)part * np + q) * knn + r] = d;
        }
    }
}

// The partitions' sorted lists of one query merged by one warp: every lane
// holds up to kMergePer of the parts x knn candidates, and each of the knn
// rounds takes the warp-wide (distance, index) minimum and retires it.
constexpr int kMergePer = 8;   // parts * knn <= 8 * 32

__global__ void k_knn_merge_warp(const int* __restrict__ pnbr, const unsigned* __restrict__ pd2, int parts,
                                 int np, int knn, int* __restrict__ nbr, unsigned* __restrict__ d2out) {
    const int q = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (q >= np) return;                      // whole warps leave together
    unsigned cd[kMergePer];
    int cj[kMergePer];
    const int total = parts * knn;
#pragma unroll
    for (int u = 0; u < kMergePer; ++u) {
        const int c = lane + 32 * u;
        if (c < total) {
            const int p = c / knn, r = c - p * knn;
            const size_t o = ((size_t)p * np + q) * knn + r;
            cd[u] = pd2[o];
            cj[u] = pnbr[o];
        } else {
            cd[u] = 0xffffffffu;
            cj[u] = 0x7fffffff;
        }
    }
    for (int r = 0; r < knn; ++r) {
        unsigned bd = 0xffffffffu;
        int bj = 0x7fffffff, bu = -1;
#pragma unroll
        for (int u = 0; u < kMergePer; ++u)
            if (less_dj(cd[u], cj[u], bd, bj)) { bd = cd[u]; bj = cj[u]; bu = u; }
        unsigned wd = bd;
        int wj = bj;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned d2 = __shfl_xor_sync(0xffffffffu, wd, o);
            const int j2 = __shfl_xor_sync(0xffffffffu, wj, o);
            if (less_dj(d2, j2, wd, wj)) { wd = d2; wj = j2; }
        }
        // the lane holding the winner retires it (indices are distinct)
        if (bu >= 0 && bj == wj && bd == wd) {
#pragma unroll
            for (int u = 0; u < kMergePer; ++u)
                if (u == bu) { cd[u] = 0xffffffffu; cj[u] = 0x7fffffff; }
        }
        if (lane == 0) {
            nbr[(size_t)q * knn + r] = wj;
            d2out[(size_t)q * knn + r] = wd;
        }
    }
}

__global__ void k_knn_merge(const int* __restrict__ pnbr, const unsigned* __restrict__ pd2, int parts, int np,
                            int knn, int* __restrict__ nbr, unsigned* __restrict__ d2out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    int pos[16];
    for (int p = 0; p < parts; ++p) pos[p] = 0;
    for (int r = 0; r < knn; ++r) {
        int bp = -1;
        unsigned bd = 0xffffffffu;
        int bjj = 0x7fffffff;
        for (int p = 0; p < parts; ++p) {
            if (pos[p] >= knn) continue;
            const size_t o = ((size_t)p * np + q) * knn + pos[p];
            if (less_dj(pd2[o], pnbr[o], bd, bjj)) { bd = pd2[o]; bjj = pnbr[o]; bp = p; }
        }
        nbr[(size_t)q * knn + r] = bjj;
        d2out[(size_t)q * knn + r] = bd;
        if (bp >= 0) pos[bp]++;
    }
}


// Candidate operand: tile t holds candidates 64 t .. 64 t + 63; B row 2 c is
// h of candidate c, row 2 c + 1 its l (zero past fd and past np), in the
// core-matrix layout; nrm[j] = |c_j|^2; with seed, bound[j] (below).  One
// warp per candidate.
__global__ void k_knn_prepare(const int* __restrict__ F, int np, int fd, int ld, int LP, int ntiles,
                              __half* __restrict__ Bg, int* __restrict__ nrm, int* __restrict__ err,
                              const int* __restrict__ seed, int knn, unsigned* __restrict__ bound) {
    const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= ntiles * kKnTile) return;
    const int tile = j / kKnTile, c = j - tile * kKnTile;
    const int KC = LP / 8;
    __half* bt = Bg + (size_t)tile * 2 * kKnTile * LP;
    int s = 0;
    bool bad = false;
    int fv[kKnMaxTcFd / 32];            // the row's entries k = lane + 32 i (LP <= 128)
#pragma unroll
    for (int i = 0; i < kKnMaxTcFd / 32; ++i) {
        const int k = lane + 32 * i;
        fv[i] = kKnCentre;
        if (k >= LP) continue;
        int v = 0;
        if (j < np && k < fd) {
            int f = F[(size_t)j * ld + k];
            if (f < 0 || f > 2 * kKnCentre) { bad = true; f = kKnCentre; }
            fv[i] = f;
            v = f - kKnCentre;
        }
        const int h = (v + 16) >> 5;        // floor((v + 16) / 32)
        const int l = v - 32 * h;
        bt[core_off(2 * c, k, KC) / 2] = __int2half_rn(h);
        bt[core_off(2 * c + 1, k, KC) / 2] = __int2half_rn(l);
        s += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(err, 1);
    if (lane == 0 && j < np) nrm[j] = s;
    if (!seed || j >= np) return;
    // bound[j]: an upper bound of row j's knn-th smallest distance from a
    // seed list (the previous graph): the largest exact distance from F_j to
    // the seed rows when these are knn distinct rows other than j (any knn
    // such rows are candidates, so the knn nearest lie within it), else
    // UINT_MAX (no bound).  Lane t < knn holds seed t; the seeds' rows are
    // read four at a time, their loads in flight together.  |F_jk - F_ik|
    // <= 4096 and fd <= 128 keep the sums exact in 32 bits.
    const int sj = lane < knn ? seed[(size_t)j * knn + lane] : -1;
    bool ok = lane >= knn || (sj >= 0 && sj < np && sj != j);
    for (int t = 0; t < knn; ++t) {
        const int o = __shfl_sync(0xffffffffu, sj, t);
        if (lane < knn && t != lane && o == sj) ok = false;
    }
    ok = __all_sync(0xffffffffu, ok);
    unsigned bmax = 0u;
    if (ok) {
        for (int t0 = 0; t0 < knn; t0 += 4) {
            unsigned dd[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u;
                const int r = __shfl_sync(0xffffffffu, sj, t & 31);
                unsigned d = 0u;
                if (t < knn) {
#pragma unroll
                    for (int i = 0; i < kKnMaxTcFd / 32; ++i) {
                        const int k = lane + 32 * i;
                        if (k < fd) {
                            const int df = fv[i] - F[(size_t)r * ld + k];
                            d += (unsigned)(df * df);
                        }
                    }
                }
                dd[u] = d;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) bmax = max(bmax, __reduce_add_sync(0xffffffffu, dd[u]));
        }
    }
    if (lane == 0) bound[j] = ok ? bmax : 0xffffffffu;
}

template <int KN>
__global__ void __launch_bounds__(kKnThreads + 32) k_knn_tc(const int* __restrict__ F, int np, int fd, int ld,
                                                            int LP, const __half* __restrict__ Bg,
                                                            const int* __restrict__ nrm, int per, int knn,
                                                            int* __restrict__ pnbr, unsigned* __restrict__ pd2,
                                                            int* __restrict__ err,
                                                            const unsigned* __restrict__ bound) {
    const int KC = LP / 8;
    const int A_BYTES = kKnRows * LP * 2;
    const int B_BYTES = 2 * kKnTile * LP * 2;
    constexpr int NCOL = 2 * kKnTile;   // accumulator columns per buffer
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sA = smraw;
    unsigned char* sB = smraw + A_BYTES;   // [kKnStages][B_BYTES]; reused for the final merge
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bfull[kKnStages], s_bempty[kKnStages], s_afull[2], s_aempty[2];
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * kKnRows;
    const int part = blockIdx.y;
    const int cb = part * per, ce = min(np, cb + per);
    const int ntiles = (ce - cb + kKnTile - 1) / kKnTile;
    const int t0 = cb / kKnTile;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        for (int q = 0; q < kKnStages; ++q) {
            mbar_init(smem_u32(&s_bfull[q]), 1);
            mbar_init(smem_u32(&s_bempty[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&s_afull[q]), 1);
            mbar_init(smem_u32(&s_aempty[q]), kKnConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // A tile: centred query vectors (zero past fd and past np); each thread
    // loads 8 entries before it converts and stores them, so the loads are in
    // flight together instead of one dependent load per entry
    for (int b0 = tid; b0 < kKnRows * LP; b0 += 8 * (int)blockDim.x) {
        int vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = b0 + u * (int)blockDim.x;
            const int row = e / LP, k = e - row * LP;
            const int q = q0 + row;
            vv[u] = (e < kKnRows * LP && q < np && k < fd) ? F[(size_t)q * ld + k] - kKnCentre : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = b0 + u * (int)blockDim.x;
            if (e >= kKnRows * LP) break;
            const int row = e / LP, k = e - row * LP;
            *reinterpret_cast<__half*>(sA + core_off(row, k, KC)) = __int2half_rn(vv[u]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    unsigned bd[KN];
    int bj[KN];
#pragma unroll
    for (int q = 0; q < KN; ++q) { bd[q] = 0xffffffffu; bj[q] = 0x7fffffff; }

    if (warp == kKnConsumers) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) {
            const uint32_t idesc = mma_idesc_f16(kKnRows, NCOL);
            int loaded = 0, mmas = 0;   // tiles whose copy / whose MMAs were issued
            auto load = [&](int tile) {
                const int st = tile % kKnStages;
                const uint32_t bar = smem_u32(&s_bfull[st]);
                mbar_expect_tx(bar, B_BYTES);
                loaded = tile + 1;
                bulk_g2s(smem_u32(sB + st * B_BYTES), Bg + (size_t)(t0 + tile) * (B_BYTES / 2), B_BYTES, bar);
            };
            for (int t = 0; t < kKnStages && t < ntiles; ++t) load(t);
            // (no read of the shared error word per tile: it costs the producer
            // several hundred cycles; a role whose partner stopped gives up at
            // its own next bounded wait)
            for (int tile = 0; tile < ntiles; ++tile) {
                const int st = tile % kKnStages, buf = tile & 1;
                if (!wait_parity(smem_u32(&s_bfull[st]), (tile / kKnStages) & 1)) { s_fail = 1; break; }
                if (tile >= 2 && !wait_parity(smem_u32(&s_aempty[buf]), ((tile >> 1) - 1) & 1)) {
                    s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t tm = tmem + (uint32_t)(buf * NCOL);
                const uint32_t bbase = smem_u32(sB + st * B_BYTES);
                for (int ks = 0; ks < LP / 16; ++ks) {
                    const uint64_t ad = smem_desc(smem_u32(sA) + ks * 256, 128, KC * 128);
                    const uint64_t bdsc = smem_desc(bbase + ks * 256, 128, KC * 128);
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tm),
                        "l"(ad), "l"(bdsc), "r"(idesc), "r"(acc));
                }
                mmas = tile + 1;
                mma_commit(smem_u32(&s_afull[buf]));
                mma_commit(smem_u32(&s_bempty[st]));
                // refill the stage of the previous tile once its MMA has read it
                const int prev = tile - 1;
                if (prev >= 0 && prev + kKnStages < ntiles) {
                    const int ps = prev % kKnStages;
                    if (!wait_parity(smem_u32(&s_bempty[ps]), (prev / kKnStages) & 1)) { s_fail = 1; break; }
                    load(prev + kKnStages);
                }
            }
            // every issued MMA and copy must finish before the block reuses shared
            // memory or releases TMEM, also when a wait gave up (bounded again)
            if (mmas > 0) {
                const int last = mmas - 1;
                if (!wait_parity(smem_u32(&s_bempty[last % kKnStages]), (last / kKnStages) & 1)) s_fail = 1;
            }
            if (s_fail)
                for (int t = mmas; t < loaded; ++t)
                    wait_parity(smem_u32(&s_bfull[t % kKnStages]), (t / kKnStages) & 1);
        }
        __syncwarp();
    } else {
        // ------------------------------ consumers -----------------------------
        const int lq = warp & 3, half = warp >> 2;
        const int qrow = q0 + lq * 32 + lane;
        const unsigned nq = qrow < np ? (unsigned)nrm[qrow] : 0u;
        // candidates farther than the query's bound cannot be among its knn
        // nearest (UINT_MAX: no bound)
        const unsigned tq = bound && qrow < np ? bound[qrow] : 0xffffffffu;
        for (int tile = 0; tile < ntiles; ++tile) {
            const int buf = tile & 1;
            const int jb = cb + tile * kKnTile + half * (kKnTile / 2);
            const unsigned nbl = jb + lane < ce ? (unsigned)__ldg(nrm + jb + lane) : 0u;
            // (the warp leaves together: its votes and aligned TMEM loads name every lane)
            if (!__all_sync(0xffffffffu, wait_parity(smem_u32(&s_afull[buf]), (tile >> 1) & 1))) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t taddr = tmem + (uint32_t)(buf * NCOL) + ((uint32_t)(lq * 32) << 16) +
                                   (uint32_t)(half * (NCOL / 2));
            // A lane meets its candidates in increasing index order, so a strict
            // "less" keeps equal earlier candidates ahead: the list is the best
            // KN by (distance, then lowest index).  The accumulator is read in
            // four groups of 8 candidates (a small loop body for the
            // instruction cache); the buffer goes back to the producer after
            // the last group.
#pragma unroll 1
            for (int grp = 0; grp < 4; ++grp) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr + 16u * (uint32_t)grp));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                // one vote per two candidates; the pair's insertions stay
                // predicated per lane and in index order
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    unsigned d[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q = 8 * grp + u + h;
                        const int j = jb + q;
                        const int ch = __float2int_rn(__uint_as_float(v[2 * (u + h)]));
                        const int cl = __float2int_rn(__uint_as_float(v[2 * (u + h) + 1]));
                        const unsigned nb = __shfl_sync(0xffffffffu, nbl, q);
                        d[h] = nq + nb - 2u * (unsigned)(32 * ch + cl);
                        if (j >= ce || j == qrow || d[h] > tq) d[h] = 0xffffffffu;
                    }
                    if (__any_sync(0xffffffffu, d[0] < bd[KN - 1] || d[1] < bd[KN - 1])) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (d[h] < bd[KN - 1]) { bd[KN - 1] = d[h]; bj[KN - 1] = jb + 8 * grp + u + h; }
#pragma unroll
                            for (int r = KN - 1; r > 0; --r) {
                                if (bd[r] < bd[r - 1]) {
                                    const unsigned td = bd[r]; bd[r] = bd[r - 1]; bd[r - 1] = td;
                                    const int tj = bj[r]; bj[r] = bj[r - 1]; bj[r - 1] = tj;
                                }
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_aempty[buf]));
            if (__any_sync(0xffffffffu, s_fail)) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NCOL));
    }
    if (s_fail) {
        if (tid == 0) atomicExch(err, 2);
        return;
    }
    if (warp >= kKnConsumers) return;
    // merge the two candidate halves' lists of each query (the ring is idle now)
    const int lq = warp & 3, half = warp >> 2;
    const int lrow = lq * 32 + lane;
    unsigned* s_md = reinterpret_cast<unsigned*>(sB);
    int* s_mj = reinterpret_cast<int*>(sB + sizeof(unsigned) * kKnRows * KN);
    if (half == 1) {
#pragma unroll
        for (int q = 0; q < KN; ++q) { s_md[lrow * KN + q] = bd[q]; s_mj[lrow * KN + q] = bj[q]; }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kKnThreads));   // consumer warps only
    if (half == 1) return;
#pragma unroll
    for (int q = 0; q < KN; ++q) {
        const unsigned d = s_md[lrow * KN + q];
        const int j = s_mj[lrow * KN + q];
        if (less_dj(d, j, bd[KN - 1], bj[KN - 1])) {
            bd[KN - 1] = d;
            bj[KN - 1] = j;
#pragma unroll
            for (int r = KN - 1; r > 0; --r) {
                if (less_dj(bd[r], bj[r], bd[r - 1], bj[r - 1])) {
                    const unsigned td = bd[r]; bd[r] = bd[r - 1]; bd[r - 1] = td;
                    const int tj = bj[r]; bj[r] = bj[r - 1]; bj[r - 1] = tj;
                }
            }
        }
    }
    const int qrow = q0 + lrow;
    if (qrow >= np) return;
#pragma unroll
    for (int r = 0; r < KN; ++r) {
        if (r < knn) {
            pnbr[((size_t)part * np + qrow) * knn + r] = bj[r];
            pd2[((size_t)part * np + qrow) * knn + r] = bd[r];
        }
    }
}

static int tc_lp(int fd) { return (fd + 15) / 16 * 16; }
static int tc_kn(int knn) { return knn <= 8 ? 8 : knn <= 10 ? 10 : knn <= 16 ? 16 : 32; }

KnnWorkspace::~KnnWorkspace() { release(); }

void KnnWorkspace::release() {
    cudaFree(bop); cudaFree(nrm); cudaFree(bound); cudaFree(pnbr); cudaFree(pd2); cudaFree(err);
    bop = nullptr; nrm = nullptr; bound = nullptr; pnbr = nullptr; pd2 = nullptr; err = nullptr;
    bop_bytes = 0; part_entries = 0; np_cap = 0;
}

mrf_status KnnWorkspace::reserve(int np, int fd, int knn) {
    if (!err) {
        MRF_CUDA(cudaMalloc(&err, sizeof(int)));
        MRF_CUDA(cudaMemset(err, 0, sizeof(int)));
    }
    const size_t entries = (size_t)kKnMaxParts * np * knn;
    if (part_entries < entries) {
        cudaFree(pnbr); cudaFree(pd2);
        pnbr = nullptr; pd2 = nullptr; part_entries = 0;
        MRF_CUDA(cudaMalloc(&pnbr, sizeof(int) * entries));
        MRF_CUDA(cudaMalloc(&pd2, sizeof(unsigned) * entries));
        part_entries = entries;
    }
    if (fd <= kKnMaxTcFd) {
        const size_t bytes = sizeof(__half) * (size_t)((np + kKnTile - 1) / kKnTile) * 2 * kKnTile * tc_lp(fd);
        if (bop_bytes < bytes) {
            cudaFree(bop);
            bop = nullptr; bop_bytes = 0;
            MRF_CUDA(cudaMalloc(&bop, bytes));
            bop_bytes = bytes;
        }
        if (np_cap < np) {
            cudaFree(nrm);
            cudaFree(bound);
            nrm = nullptr; bound = nullptr; np_cap = 0;
            MRF_CUDA(cudaMalloc(&nrm, sizeof(int) * (size_t)np));
            MRF_CUDA(cudaMalloc(&bound, sizeof(unsigned) * (size_t)np));
            np_cap = np;
        }
    }
    return MRF_OK;
}

mrf_status knn_run(KnnWorkspace& ws, const int* F, int np, int fd, int ld, int knn, int* nbr, unsigned* d2,
                   cudaStream_t s, const int* seed) {
    MRF_REQUIRE(F && nbr && d2, "patch kNN: NULL pointer");
    MRF_REQUIRE(knn >= 1 && knn <= 32, "patch kNN: knn = %d outside [1, 32]", knn);
    MRF_REQUIRE(np > knn, "patch kNN: needs more than knn = %d vectors (got %d)", knn, np);
    MRF_REQUIRE(fd >= 1 && fd <= 255, "patch kNN: vector length %d outside [1, 255]", fd);
    MRF_REQUIRE(ld >= fd && ld % 4 == 0, "patch kNN: row stride %d must be >= %d and a multiple of 4", ld, fd);
    MRF_PROPAGATE(ws.reserve(np, fd, knn));
    int parts = 1;
    if (fd <= kKnMaxTcFd) {
        const int LP = tc_lp(fd);
        const int ntiles = (np + kKnTile - 1) / kKnTile;
        const size_t thr = (size_t)ntiles * kKnTile * 32;
        k_knn_prepare<<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(F, np, fd, ld, LP, ntiles,
                                                                     static_cast<__half*>(ws.bop), ws.nrm, ws.err,
                                                                     seed, knn, ws.bound);
        MRF_LAUNCHED_AS("k_knn_prepare", s);
        // about two blocks per SM: 128 queries x one candidate partition each
        const int qb = (np + kKnRows - 1) / kKnRows;
        parts = std::max(1, std::min(kKnMaxParts, (2 * 152 + qb - 1) / qb));
        int per = (np + parts - 1) / parts;
        per = (per + kKnTile - 1) / kKnTile * kKnTile;
        parts = (np + per - 1) / per;
        const int kn = tc_kn(knn);
        const size_t ring = std::max<size_t>((size_t)kKnStages * 2 * kKnTile * LP * 2, (size_t)kKnRows * kn * 8);
        const size_t sm = (size_t)kKnRows * LP * 2 + ring;
        dim3 grid(qb, parts);
#define MRF_KNN_LAUNCH(KNV)                                                                                  \
    do {                                                                                                     \
        MRF_CUDA(cudaFuncSetAttribute(k_knn_tc<KNV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); \
        k_knn_tc<KNV><<<grid, kKnThreads + 32, sm, s>>>(F, np, fd, ld, LP,                                  \
                                                        static_cast<const __half*>(ws.bop), ws.nrm, per,    \
                                                        knn, ws.pnbr, ws.pd2, ws.err,                       \
                                                        seed ? ws.bound : nullptr);                         \
    } while (0)
        if (kn == 8) MRF_KNN_LAUNCH(8);
        else if (kn == 10) MRF_KNN_LAUNCH(10);
        else if (kn == 16) MRF_KNN_LAUNCH(16);
        else MRF_KNN_LAUNCH(32);
#undef MRF_KNN_LAUNCH
        MRF_LAUNCHED_AS("k_knn_tc", s);
    } else {
        const size_t sm = sizeof(int) * (size_t)(32 + 64) * (ld + 4);
        const int qb = (np + 31) / 32;
        parts = std::max(1, std::min(kKnMaxParts, (4 * 152 + qb - 1) / qb));
        int per = (np + parts - 1) / parts;
        per = (per + 63) / 64 * 64;
        parts = (np + per - 1) / per;
        dim3 grid(qb, parts);
        if (knn <= 16) {
            MRF_CUDA(cudaFuncSetAttribute(k_knn_part<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_knn_part<16><<<grid, 256, sm, s>>>(F, np, ld, knn, per, ws.pnbr, ws.pd2);
        } else {
            MRF_CUDA(cudaFuncSetAttribute(k_knn_part<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_knn_part<32><<<grid, 256, sm, s>>>(F, np, ld, knn, per, ws.pnbr, ws.pd2);
        }
        MRF_LAUNCHED_AS("k_knn_part", s);
    }
    if (parts * knn <= 32 * kMergePer)
        k_knn_merge_warp<<<(unsigned)(((size_t)np * 32 + 255) / 256), 256, 0, s>>>(ws.pnbr, ws.pd2, parts, np, knn,
                                                                                   nbr, d2);
    else
        k_knn_merge<<<(np + 127) / 128, 128, 0, s>>>(ws.pnbr, ws.pd2, parts, np, knn, nbr, d2);
    MRF_LAUNCHED_AS("k_knn_merge", s);
    return MRF_OK;
}

}  // namespace mrf

using namespace mrf;

static mrf_status patch_knn(const int* F, int np, int fd, int ld, int knn, const int* seed, int* nbr, unsigned* d2,
                            mrf_stream stream) {
    cudaStream_t s = as_stream(stream);
    KnnWorkspace ws;
    MRF_PROPAGATE(knn_run(ws, F, np, fd, ld, knn, nbr, d2, s, seed));
    int h = 0;
    MRF_CUDA(cudaMemcpyAsync(&h, ws.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    MRF_REQUIRE(h != 1, "mrf_patch_knn: a feature lies outside [0, 4096]");
    if (h) {
        set_error("mrf_patch_knn: a tensor-core wait timed out");
        return MRF_ETIMEOUT;
    }
    return MRF_OK;
}

extern "C" mrf_status mrf_patch_knn(const int* F, int np, int fd, int ld, int knn, int* nbr, unsigned* d2,
                                    mrf_stream stream) {
    return patch_knn(F, np, fd, ld, knn, nullptr, nbr, d2, stream);
}

extern "C" mrf_status mrf_patch_knn_seeded(const int* F, int np, int fd, int ld, int knn, const int* seed, int* nbr,
                                           unsigned* d2, mrf_stream stream) {
    MRF_REQUIRE(seed != nullptr, "mrf_patch_knn_seeded: NULL seed");
    return patch_knn(F, np, fd, ld, knn, seed, nbr, d2, stream);
}

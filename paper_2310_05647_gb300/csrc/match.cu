// Dictionary matching Phi_D (Eq. 5): for every fingerprint x_i
//   k_i = argmax_m |<d_m, x_i>| / ||d_m||   (||d_m||^2 with the literal flag)
//   rho_i = max(Re<d_k, x_i> / ||d_k||^2, 0),  eta_i = LUT[k_i]
// with <a, b> = sum conj(a) b and ties resolved to the lowest index.
//
// The plain form (MRF_MATCH_FP32) is a SIMT FP32 GEMM tile (64 fingerprints x
// 64 atoms, 4 x 4 complex micro-tiles per thread) whose epilogue keeps, per
// fingerprint, the running best (score, index, inner product) over all atom
// tiles; no fingerprint x atom score is ever written to memory.  The BF16
// tensor-core form lives in match_tc.cu.

#include "common.h"
#include "match.h"

namespace mrf {

constexpr int BM = 64, BN = 64, BK = 8;

__device__ __forceinline__ bool better(float s, int i, float bs, int bi) {
    return s > bs || (s == bs && i < bi);
}

__global__ void __launch_bounds__(256) k_match_fp32(const float2* __restrict__ x, int n, int len,
                                                    const float2* __restrict__ dict,
                                                    const float* __restrict__ wscore, int m,
                                                    int* __restrict__ best_idx, float2* __restrict__ best_ip) {
    __shared__ float2 xs[BK][BM + 1];
    __shared__ float2 ds[BK][BN + 1];
    __shared__ float ws[BN];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int v0 = blockIdx.x * BM;
    float bsc[4];
    int bid[4];
    float2 bip[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { bsc[i] = -1.f; bid[i] = 0x7fffffff; bip[i] = make_float2(0.f, 0.f); }
    for (int a0 = 0; a0 < m; a0 += BN) {
        float2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
        __syncthreads();   // every warp is done with the previous tile's weights
        if (threadIdx.x < BN) ws[threadIdx.x] = (a0 + threadIdx.x < m) ? wscore[a0 + threadIdx.x] : 0.f;
        for (int k0 = 0; k0 < len; k0 += BK) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int e = threadIdx.x + q * 256;
                const int r = e >> 3, kk = e & 7;
                const int k = k0 + kk;
                const int v = v0 + r, a = a0 + r;
                xs[kk][r] = (v < n && k < len) ? x[(size_t)v * len + k] : make_float2(0.f, 0.f);
                ds[kk][r] = (a < m && k < len) ? dict[(size_t)a * len + k] : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float2 xv[4], dv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) xv[i] = xs[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) dv[j] = ds[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        // conj(d) * x
                        acc[i][j].x = fmaf(dv[j].x, xv[i].x, fmaf(dv[j].y, xv[i].y, acc[i][j].x));
                        acc[i][j].y = fmaf(dv[j].x, xv[i].y, fmaf(-dv[j].y, xv[i].x, acc[i][j].y));
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = a0 + tx + 16 * j;
            if (a < m) {
                const float w = ws[tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float sc = cabs2(acc[i][j]) * w;
                    if (better(sc, a, bsc[i], bid[i])) { bsc[i] = sc; bid[i] = a; bip[i] = acc[i][j]; }
                }
            }
        }
    }
    // reduce over the 16 threads (tx) that share the same fingerprints
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, bsc[i], o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bid[i], o);
            const float px = __shfl_xor_sync(0xffffffffu, bip[i].x, o);
            const float py = __shfl_xor_sync(0xffffffffu, bip[i].y, o);
            if (better(s2, i2, bsc[i], bid[i])) { bsc[i] = s2; bid[i] = i2; bip[i] = make_float2(px, py); }
        }
        const int v = v0 + ty + 16 * i;
        // no finite best score (NaN or infinite entries): index 0, PD 0, like an all-zero x
        const bool found = bid[i] < m && isfinite(bsc[i]);
        if (tx == 0 && v < n) {
            best_idx[v] = found ? bid[i] : 0;
            best_ip[v] = found ? bip[i] : make_float2(0.f, 0.f);
        }
    }
}

// per-atom weights of the score: 1/||d||^2 (argmax of |s|^2/||d||^2 is the
// argmax of |s|/||d||) or 1/||d||^4 for the literal |s|/||d||^2.  One warp
// per atom: the lanes read consecutive entries and sum their (non-negative)
// terms in FP32, len / 32 of them each; the 32 lane sums are combined in FP64
// by a fixed shuffle tree (FP64 work per element is slow on this GPU).
__global__ void k_match_weights(const float2* __restrict__ dict, const float* __restrict__ norm2_in, int m, int len,
                                int literal, float* __restrict__ norm2, float* __restrict__ wscore) {
    const int a = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (a >= m) return;                                   // whole warps
    float n2;
    if (norm2_in) {
        n2 = norm2_in[a];
    } else {
        float f = 0.f;
        for (int k = lane; k < len; k += 32) f += cabs2(dict[(size_t)a * len + k]);
        double s = (double)f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        n2 = (float)s;
    }
    if (lane == 0) {
        norm2[a] = n2;
        const float inv = n2 > 0.f ? 1.0f / n2 : 0.f;
        wscore[a] = literal ? inv * inv : inv;
    }
}

__global__ void k_match_finish(const int* __restrict__ best_idx, const float2* __restrict__ best_ip, int n,
                               const float* __restrict__ norm2, const float* __restrict__ lut,
                               int* __restrict__ idx, float* __restrict__ pd, float* __restrict__ t1t2,
                               float pd_scale) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int k = best_idx[v];
    const float n2 = norm2[k];
    if (idx) idx[v] = k;
    if (pd) pd[v] = n2 > 0.f ? fmaxf(best_ip[v].x / n2, 0.f) * pd_scale : 0.f;
    if (t1t2) {
        t1t2[2 * v] = lut[2 * k];
        t1t2[2 * v + 1] = lut[2 * k + 1];
    }
}

MatchWorkspace::~MatchWorkspace() { release(); }

void MatchWorkspace::carve(char* base, int n, int m, size_t tc_bytes) {
    auto take = [&](size_t b) { char* p = base; base += (b + 255) / 256 * 256; return p; };
    best_idx = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
    best_ip = reinterpret_cast<float2*>(take(sizeof(float2) * (size_t)n));
    cand = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n * kTopK));
    norm2 = reinterpret_cast<float*>(take(sizeof(float) * (size_t)m));
    wscore = reinterpret_cast<float*>(take(sizeof(float) * (size_t)m));
    if (tc_bytes) {
        tc_err = reinterpret_cast<int*>(take(sizeof(int)));
        tc_b = take(tc_bytes);
        tc_b_bytes = tc_bytes;
    }
    cap_n = n;
    cap_m = m;
    borrowed = true;
}

void MatchWorkspace::detach() {
    best_idx = nullptr; best_ip = nullptr; norm2 = nullptr; wscore = nullptr; cand = nullptr;
    tc_b = nullptr; tc_err = nullptr; tc_b_bytes = 0; tc_dict = nullptr; tc_m = tc_len = 0;
    cap_n = cap_m = 0;
    borrowed = false;
}

void MatchWorkspace::release() {
    if (borrowed) { detach(); return; }
    cudaFree(best_idx); cudaFree(best_ip); cudaFree(norm2); cudaFree(wscore);
    cudaFree(cand); cudaFree(tc_b); cudaFree(tc_err);
    best_idx = nullptr; best_ip = nullptr; norm2 = nullptr; wscore = nullptr; cand = nullptr;
    tc_b = nullptr; tc_err = nullptr; tc_b_bytes = 0; tc_dict = nullptr;
    cap_n = cap_m = 0;
}

mrf_status MatchWorkspace::reserve(int n, int m) {
    if (n > cap_n) {
        cudaFree(best_idx); cudaFree(best_ip); cudaFree(cand);
        best_idx = nullptr; best_ip = nullptr; cand = nullptr;
        MRF_CUDA(cudaMalloc(&best_idx, sizeof(int) * (size_t)n));
        MRF_CUDA(cudaMalloc(&best_ip, sizeof(float2) * (size_t)n));
        MRF_CUDA(cudaMalloc(&cand, sizeof(int) * (size_t)n * kTopK));
        cap_n = n;
    }
    if (m > cap_m) {
        cudaFree(norm2); cudaFree(wscore);
        norm2 = nullptr; wscore = nullptr;
        MRF_CUDA(cudaMalloc(&norm2, sizeof(float) * (size_t)m));
        MRF_CUDA(cudaMalloc(&wscore, sizeof(float) * (size_t)m));
        cap_m = m;
    }
    return MRF_OK;
}

mrf_status match_prepare(MatchWorkspace& ws, const float2* dict, const float* norm2_in, int m, int len,
                         int literal, cudaStream_t s) {
    k_match_weights<<<(unsigned)(((size_t)m * 32 + 255) / 256), 256, 0, s>>>(dict, norm2_in, m, len, literal,
                                                                             ws.norm2, ws.wscore);
    MRF_LAUNCHED_AS("k_match_weights", s);
    ws.tc_dict = nullptr;   // the tensor-core operand carries the weights: rebuild it
    return MRF_OK;
}

mrf_status match_run(MatchWorkspace& ws, const float2* x, int n, int len, const float2* dict, int m,
                     int precision, const float* lut, int* idx, float* pd, float* t1t2, float pd_scale,
                     cudaStream_t s, int* cand_io) {
    if (tc_form(precision) && tc_long(len, tc_form(precision))) {
        MRF_PROPAGATE(match_tc_long(ws, x, n, len, dict, m, tc_form(precision), s));
    } else if (tc_form(precision)) {
        MRF_PROPAGATE(match_tc_candidates(ws, x, n, len, dict, m, tc_form(precision), s, cand_io));
        MRF_PROPAGATE(match_rerank(ws, x, n, len, dict, s));
    } else {
        k_match_fp32<<<(n + BM - 1) / BM, 256, 0, s>>>(x, n, len, dict, ws.wscore, m, ws.best_idx, ws.best_ip);
        MRF_LAUNCHED_AS("k_match_fp32", s);
    }
    return match_finish(ws, n, lut, idx, pd, t1t2, pd_scale, s);
}

mrf_status match_finish(MatchWorkspace& ws, int n, const float* lut, int* idx, float* pd, float* t1t2,
                        float pd_scale, cudaStream_t s) {
    k_match_finish<<<(n + 255) / 256, 256, 0, s>>>(ws.best_idx, ws.best_ip, n, ws.norm2, lut, idx, pd, t1t2,
                                                   pd_scale);
    MRF_LAUNCHED_AS("k_match_finish", s);
    return MRF_OK;
}

}  // namespace mrf

using namespace mrf;

static mrf_status match_call(const mrf_c64* x, int n, int len, const mrf_c64* dict, const float* atom_norm2,
                             const float* lut, int m, int precision, int* cand, int* idx, float* pd, float* t1t2,
                             mrf_stream stream) {
    MRF_REQUIRE(x && dict && lut, "mrf_match: NULL x, dict or lut");
    MRF_REQUIRE(n >= 0 && len >= 1 && len <= 2048, "mrf_match: bad n or len (%d, %d)", n, len);
    MRF_REQUIRE(m >= 1 && m <= (1 << 24), "mrf_match: bad m (%d)", m);
    const int prec = precision & 0xff;
    const int literal = (precision & MRF_MATCH_LITERAL_NORM2) ? 1 : 0;
    MRF_REQUIRE(prec == MRF_MATCH_FP32 || prec == MRF_MATCH_BF16 || prec == MRF_MATCH_BF16X3 ||
                    prec == MRF_MATCH_FP8,
                "mrf_match: unknown precision %d", prec);
    MRF_REQUIRE(!(literal && prec != MRF_MATCH_FP32), "mrf_match: the literal norm flag needs FP32");
    if (n == 0) return MRF_OK;
    cudaStream_t s = as_stream(stream);
    // stream-ordered scratch: released on the stream after the kernels
    MatchWorkspace ws;
    MRF_REQUIRE(!(prec == MRF_MATCH_FP8 && tc_long(len, 8)),
                "mrf_match: FP8 matching supports lengths up to 64 (got %d)", len);
    MRF_REQUIRE(!(cand && tc_long(len, tc_form(prec))),
                "mrf_match_seeded: lengths beyond the resident tile are not seeded (got %d)", len);
    const size_t tcb = prec == MRF_MATCH_FP32 ? 0
                       : tc_long(len, tc_form(prec)) ? tc_long_scratch_bytes(n, m, len, tc_form(prec))
                                                     : tc_operand_bytes(m, len, tc_form(prec));
    const size_t bytes = sizeof(int) * (size_t)n + sizeof(float2) * (size_t)n + sizeof(int) * (size_t)n * kTopK +
                         2 * sizeof(float) * (size_t)m + tcb + 8 * 256;
    char* base = nullptr;
    MRF_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, s));
    ws.carve(base, n, m, tcb);
    if (tcb) MRF_CUDA(cudaMemsetAsync(ws.tc_err, 0, sizeof(int), s));
    mrf_status st = match_prepare(ws, reinterpret_cast<const float2*>(dict), atom_norm2, m, len, literal, s);
    if (st == MRF_OK)
        st = match_run(ws, reinterpret_cast<const float2*>(x), n, len, reinterpret_cast<const float2*>(dict), m,
                       prec, lut, idx, pd, t1t2, 1.0f, s, cand);
    if (st == MRF_OK && tcb) {
        // a bounded device wait that gave up is reported, not hidden
        int h = 0;
        if (cudaMemcpyAsync(&h, ws.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess && h) {
            set_error("mrf_match: a tensor-core wait timed out");
            st = MRF_ETIMEOUT;
        }
    }
    ws.detach();
    MRF_CUDA(cudaFreeAsync(base, s));
    return st;
}

extern "C" mrf_status mrf_match(const mrf_c64* x, int n, int len, const mrf_c64* dict, const float* atom_norm2,
                                const float* lut, int m, int precision, int* idx, float* pd, float* t1t2,
                                mrf_stream stream) {
    return match_call(x, n, len, dict, atom_norm2, lut, m, precision, nullptr, idx, pd, t1t2, stream);
}

extern "C" mrf_status mrf_match_seeded(const mrf_c64* x, int n, int len, const mrf_c64* dict,
                                       const float* atom_norm2, const float* lut, int m, int precision, int* cand,
                                       int* idx, float* pd, float* t1t2, mrf_stream stream) {
    const int prec = precision & 0xff;
    MRF_REQUIRE(prec == MRF_MATCH_BF16 || prec == MRF_MATCH_BF16X3,
                "mrf_match_seeded: precision must be MRF_MATCH_BF16 or MRF_MATCH_BF16X3 (got %d)", prec);
    MRF_REQUIRE(cand || n == 0, "mrf_match_seeded: NULL cand");
    return match_call(x, n, len, dict, atom_norm2, lut, m, precision, cand, idx, pd, t1t2, stream);
}

namespace mrf {

// ---------------------------------------------------------------------------
// Matching without device allocation.
//
// Some callers cannot allocate device memory at the moment they match: a
// scanner-side reconstruction service that reserves all of the GPU's memory
// for its own pool at start-up (a cudaMalloc then fails or steals from that
// pool), or a latency-bound serving loop that must not pay for cudaMalloc /
// cudaFree (which can block the host and synchronise the device).  This
// variant keeps the per-call scratch of the FP32 matcher in a fixed
// file-scope device array instead: up to kNoAllocMaxN fingerprints and
// kNoAllocMaxM atoms (about 3.6 MB, held by every GPU that loads the
// library until the process exits).
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxN = 1 << 18;   // 512 x 512 voxels
constexpr int kNoAllocMaxM = 1 << 16;   // atoms
constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kNoAllocBytes = round_up(sizeof(int) * kNoAllocMaxN) + round_up(sizeof(float2) * kNoAllocMaxN) +
                                 2 * round_up(sizeof(float) * kNoAllocMaxM);

static __device__ __align__(256) unsigned char g_match_scratch[kNoAllocBytes];

// Device address of g_match_scratch on the current device, looked up on every
// call: the lookup allocates nothing, and a cached address would go stale if
// the device's primary context were destroyed (cudaDeviceReset) and the module
// loaded again at another address.  The first lookup on a device loads the
// library's module there, so that first call should come before any stream
// capture.
static char* scratch_for_current_device(mrf_status* st) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_match_scratch);
    if (e != cudaSuccess || !p) {
        set_error("mrf_match_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        *st = MRF_ECUDA;
        return nullptr;
    }
    return static_cast<char*>(p);
}

}  // namespace mrf

extern "C" mrf_status mrf_match_noalloc(const mrf_c64* x, int n, int len, const mrf_c64* dict,
                                        const float* atom_norm2, const float* lut, int m, int precision,
                                        int* idx, float* pd, float* t1t2, mrf_stream stream) {
    using namespace mrf;
    MRF_REQUIRE(x && dict && lut, "mrf_match_noalloc: NULL x, dict or lut");
    MRF_REQUIRE(n >= 0 && len >= 1 && len <= 2048, "mrf_match_noalloc: bad n or len (%d, %d)", n, len);
    MRF_REQUIRE(n <= kNoAllocMaxN, "mrf_match_noalloc: n = %d exceeds the fixed scratch (at most %d fingerprints)",
                n, kNoAllocMaxN);
    MRF_REQUIRE(m >= 1 && m <= kNoAllocMaxM,
                "mrf_match_noalloc: m = %d outside [1, %d] (the fixed scratch holds at most %d atoms)", m,
                kNoAllocMaxM, kNoAllocMaxM);
    const int prec = precision & 0xff;
    const int literal = (precision & MRF_MATCH_LITERAL_NORM2) ? 1 : 0;
    MRF_REQUIRE(prec == MRF_MATCH_FP32, "mrf_match_noalloc: only MRF_MATCH_FP32 (got %d)", prec);
    if (n == 0) return MRF_OK;
    mrf_status st = MRF_OK;
    char* base = scratch_for_current_device(&st);
    if (!base) return st;
    // every scratch word this call reads is written by this call first, so
    // nothing needs clearing between calls
    MatchWorkspace ws;
    ws.best_idx = reinterpret_cast<int*>(base);
    base += round_up(sizeof(int) * kNoAllocMaxN);
    ws.best_ip = reinterpret_cast<float2*>(base);
    base += round_up(sizeof(float2) * kNoAllocMaxN);
    ws.norm2 = reinterpret_cast<float*>(base);
    base += round_up(sizeof(float) * kNoAllocMaxM);
    ws.wscore = reinterpret_cast<float*>(base);
    ws.cap_n = n;
    ws.cap_m = m;
    ws.borrowed = true;
    cudaStream_t s = as_stream(stream);
    st = match_prepare(ws, reinterpret_cast<const float2*>(dict), atom_norm2, m, len, literal, s);
    if (st == MRF_OK)
        st = match_run(ws, reinterpret_cast<const float2*>(x), n, len, reinterpret_cast<const float2*>(dict), m,
                       MRF_MATCH_FP32, lut, idx, pd, t1t2, 1.0f, s);
    ws.detach();
    return st;
}

// Learned signal-to-parameter matcher: a 20-256-256-256-3 multilayer
// perceptron with GELU hidden units that maps a fingerprint's subspace
// coefficients (divided by their norm) to normalised log T1, log T2 and PD
// per unit input norm, standing in for dictionary matching (Eq. 5) in the
// loop; the paper's related work (Section I) cites this replacement.
//
// Everything is hand-written: training-set synthesis from EPG signals,
// forward and backward passes (the three products of every layer on the
// tensor cores -- split BF16 operands, FP32 accumulation, gemm_tc.cuh -- or a
// strided SIMT GEMM, plus bias/GELU, loss, GELU-derivative and bias-sum
// kernels), Adam, and inference (tcgen05, or a fused SIMT kernel).  Weights
// are used in BF16 (a copy of the FP32 master weights refreshed by every Adam
// step), biases and all activations and accumulations are FP32.
//
// Parameter layout (packed, host and device): per layer W [out][in]
// row-major, then b [out].  Loss 1 / (2B) sum (y - t)^2.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
#include "gemm_tc.cuh"
#include "mlp.h"
#include "tc5.cuh"

namespace mrf {

constexpr int kLayers = 4;
constexpr int kSizes[kLayers + 1] = {kMlpIn, kMlpHidden, kMlpHidden, kMlpHidden, kMlpOut};

struct Layout {
    size_t w[kLayers], b[kLayers], total;
};

static Layout layout() {
    Layout L{};
    size_t at = 0;
    for (int l = 0; l < kLayers; ++l) {
        L.w[l] = at;
        at += (size_t)kSizes[l + 1] * kSizes[l];
        L.b[l] = at;
        at += kSizes[l + 1];
    }
    L.total = at;
    return L;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
    return cdf + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// C[m][n] (+)= sum_k A[m sam + k sak] B[k sbk + n sbn]: 64 x 64 tiles, k steps of
// 16, each of 256 threads a 4 x 4 block of C; strides give the transposes.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const TA* __restrict__ A, int sam, int sak,
                                              const TB* __restrict__ B, int sbk, int sbn, float* __restrict__ C,
                                              int ldc, int accumulate) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int r = e / 16, c = e - r * 16;
            As[c][r] = (m0 + r < M && k0 + c < K) ? to_f(A[(size_t)(m0 + r) * sam + (size_t)(k0 + c) * sak]) : 0.f;
            const int rb = e / 64, cb = e - rb * 64;
            Bs[rb][cb] = (k0 + rb < K && n0 + cb < N) ? to_f(B[(size_t)(k0 + rb) * sbk + (size_t)(n0 + cb) * sbn])
                                                      : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float* c = C + (size_t)m * ldc + n;
                *c = accumulate ? *c + acc[i][j] : acc[i][j];
            }
        }
}

template <typename TA, typename TB, int NT>
static mrf_status gemm_tc_launch(int M, int N, int K, const TA* A, int sam, int sak, const TB* B, int sbk, int sbn,
                                 float* C, int ldc, bool accumulate, int* err, cudaStream_t s) {
    constexpr bool split_b = !std::is_same<TB, __nv_bfloat16>::value;
    const size_t sm = (size_t)2 * kGtM * kGtK * 2 + (size_t)(split_b ? 2 : 1) * NT * kGtK * 2;
    MRF_CUDA(cudaFuncSetAttribute(k_gemm_tc<TA, TB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const dim3 grid((unsigned)((N + NT - 1) / NT), (unsigned)((M + kGtM - 1) / kGtM));
    k_gemm_tc<TA, TB, NT><<<grid, 128, sm, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, accumulate ? 1 : 0, err);
    MRF_LAUNCHED_AS("k_mlp_gemm_tc", s);
    return MRF_OK;
}

// tc: the tensor-core kernel (split BF16, FP32-accurate products; a device
// wait that gives up raises *err), else the SIMT kernel
template <typename TA, typename TB>
static mrf_status gemm(int M, int N, int K, const TA* A, int sam, int sak, const TB* B, int sbk, int sbn, float* C,
                       int ldc, bool accumulate, cudaStream_t s, bool tc = false, int* err = nullptr) {
    if (tc) {
        if (N <= 16) return gemm_tc_launch<TA, TB, 16>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, accumulate, err, s);
        if (N <= 32) return gemm_tc_launch<TA, TB, 32>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, accumulate, err, s);
        return gemm_tc_launch<TA, TB, 128>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, accumulate, err, s);
    }
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, accumulate ? 1 : 0);
    MRF_LAUNCHED_AS("k_mlp_gemm", s);
    return MRF_OK;
}

// Z += b (per column); A = GELU(Z) for hidden layers
__global__ void k_bias_act(float* __restrict__ Z, const float* __restrict__ b, int rows, int cols, int hidden,
                           float* __restrict__ A) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= (size_t)rows * cols) return;
    const float z = Z[e] + b[e % cols];
    Z[e] = z;
    if (hidden) A[e] = gelu(z);
}

// dY = (Y - T) / B and L = sum (Y - T)^2 / (2 B), one block, fixed-order sum
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ Y, const float* __restrict__ T, int n,
                                              float invB, float* __restrict__ dY, float* __restrict__ loss) {
    __shared__ double red[256];
    double s = 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const float d = Y[e] - T[e];
        dY[e] = d * invB;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = (float)(red[0] * 0.5 * invB);
}

// dZ = dA GELU'(Z), elementwise (dZ may be dA)
__global__ void k_gelu_bwd(const float* dA, const float* __restrict__ Z, size_t n, float* dZ) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e < n) dZ[e] = dA[e] * gelu_grad(Z[e]);
}

// db[o] = sum over rows of dZ[row][o] (row order fixed)
__global__ void k_bias_grad(const float* __restrict__ dZ, int rows, int cols, float* __restrict__ db) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dZ[(size_t)r * cols + o];
    db[o] = s;
}

__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, size_t n, __nv_bfloat16* __restrict__ wb) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// Wt[l][k][o] = W[l][o][k] (BF16, the inference kernel's coalesced layout)
__global__ void k_transpose_w(const __nv_bfloat16* __restrict__ W, int out, int in, __nv_bfloat16* __restrict__ Wt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= out * in) return;
    const int o = e / in, k = e - o * in;
    Wt[(size_t)k * out + o] = W[e];
}

// Fused inference: a block owns 32 fingerprints; activations stay in shared
// memory, each of the 256 threads computes one hidden unit for all 32 (its
// weights read coalesced from the transposed BF16 copy), the 3 outputs are
// 96 (fingerprint, output) dot products.
constexpr int kInfRows = 32;
constexpr int kInfLd = kMlpHidden + 4;

struct InferParams {
    const __nv_bfloat16* wt[kLayers];
    const float* b[kLayers];
};

__global__ void __launch_bounds__(kMlpHidden) k_mlp_infer(InferParams P, const float* __restrict__ x, int n,
                                                          float* __restrict__ y) {
    extern __shared__ float4 sm4[];
    float* act = reinterpret_cast<float*>(sm4);            // [2][kInfRows][kInfLd]
    const int r0 = blockIdx.x * kInfRows;
    const int t = threadIdx.x;
    for (int e = t; e < kInfRows * kMlpIn; e += blockDim.x) {
        const int r = e / kMlpIn, k = e - r * kMlpIn;
        act[r * kInfLd + k] = r0 + r < n ? x[(size_t)(r0 + r) * kMlpIn + k] : 0.f;
    }
    __syncthreads();
    int cur = 0;
    for (int l = 0; l < kLayers - 1; ++l) {
        const int in = l == 0 ? kMlpIn : kMlpHidden;
        const float* a = act + cur * kInfRows * kInfLd;
        float* o = act + (cur ^ 1) * kInfRows * kInfLd;
        float acc[kInfRows];
        const float bt = P.b[l][t];
#pragma unroll
        for (int r = 0; r < kInfRows; ++r) acc[r] = bt;
        const __nv_bfloat16* wt = P.wt[l];
        for (int k = 0; k < in; k += 4) {
            const float w0 = __bfloat162float(wt[(size_t)(k + 0) * kMlpHidden + t]);
            const float w1 = __bfloat162float(wt[(size_t)(k + 1) * kMlpHidden + t]);
            const float w2 = __bfloat162float(wt[(size_t)(k + 2) * kMlpHidden + t]);
            const float w3 = __bfloat162float(wt[(size_t)(k + 3) * kMlpHidden + t]);
#pragma unroll
            for (int r = 0; r < kInfRows; ++r) {
                const float4 av = *reinterpret_cast<const float4*>(a + r * kInfLd + k);
                acc[r] = fmaf(av.x, w0, fmaf(av.y, w1, fmaf(av.z, w2, fmaf(av.w, w3, acc[r]))));
            }
        }
#pragma unroll
        for (int r = 0; r < kInfRows; ++r) o[r * kInfLd + t] = gelu(acc[r]);
        __syncthreads();
        cur ^= 1;
    }
    if (t < kInfRows * kMlpOut) {
        const int r = t / kMlpOut, j = t - r * kMlpOut;
        const float* a = act + cur * kInfRows * kInfLd + r * kInfLd;
        const __nv_bfloat16* wt = P.wt[kLayers - 1];
        float s = P.b[kLayers - 1][j];
        for (int k = 0; k < kMlpHidden; ++k) s = fmaf(a[k], __bfloat162float(wt[(size_t)k * kMlpOut + j]), s);
        if (r0 + r < n) y[(size_t)(r0 + r) * kMlpOut + j] = s;
    }
}

// Tensor-core inference (tcgen05, BF16 operands, FP32 accumulators in TMEM).
// A block owns 128 fingerprints per tile (one per TMEM lane) and loops over
// tiles.  The layer input sits in shared memory as the MMA's A operand
// ([128][K] BF16, canonical K-major core matrices); each layer's weights
// [N][K] arrive with one bulk copy (pre-arranged in the same layout), the
// 128 x N product lands in TMEM (N = 256, or 16 for the 3 padded outputs),
// and 16 warps (four per lane quarter, one column quarter each) add the
// bias (staged in shared memory), apply GELU and write the next layer's input
// back as BF16.  The next
// layer's weights are requested as soon as the current products are done,
// so the copy overlaps the epilogue.  Every wait is bounded.
constexpr int kTcMlpRows = 128;
constexpr int kTcMlpWarps = 16;
constexpr int kL0K = 32;                   // the 20 inputs padded to two MMA k-steps
constexpr int kOutN = 16;                  // the 3 outputs padded to the smallest N
constexpr int kWBytes = kMlpHidden * kMlpHidden * 2;        // largest weight operand
constexpr int kABytes = kTcMlpRows * kMlpHidden * 2;

struct TcInferParams {
    const unsigned char* w[kLayers];       // pre-arranged BF16 operands
    int wbytes[kLayers];
    const float* b[kLayers];
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(32 * kTcMlpWarps) k_mlp_infer_tc(TcInferParams P, const float* __restrict__ x,
                                                                   int n, float* __restrict__ y,
                                                                   int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sA = smraw;                 // layer input [128][K]
    unsigned char* sW = smraw + kABytes;       // layer weights [N][K]
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_wbar, s_mbar;
    __shared__ int s_fail;
    __shared__ float s_bias[kLayers - 1][kMlpHidden + 4];   // hidden biases, then the outputs' at [2][256..]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lq = warp & 3, quarter = warp >> 2;
    for (int e = tid; e < (kLayers - 1) * kMlpHidden; e += blockDim.x)
        s_bias[e / kMlpHidden][e % kMlpHidden] = P.b[e / kMlpHidden][e % kMlpHidden];
    if (tid < kMlpOut) s_bias[kLayers - 2][kMlpHidden + tid] = P.b[kLayers - 1][tid];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kMlpHidden));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        mbar_init(smem_u32(&s_wbar), 1);
        mbar_init(smem_u32(&s_mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    uint32_t wphase = 0, mphase = 0;
    int pending_w = 0;                         // weight copies issued and not yet waited for
    int pending_m = 0;                         // products committed and not yet seen complete
    const int ntiles = (n + kTcMlpRows - 1) / kTcMlpRows;
    auto load_w = [&](int l) {
        const uint32_t bar = smem_u32(&s_wbar);
        mbar_expect_tx(bar, (uint32_t)P.wbytes[l]);
        bulk_g2s(smem_u32(sW), P.w[l], (uint32_t)P.wbytes[l], bar);
    };
    if (tid == 0 && blockIdx.x < ntiles) { load_w(0); pending_w = 1; }
    for (int tile = blockIdx.x; tile < ntiles && !s_fail; tile += gridDim.x) {
        const int r0 = tile * kTcMlpRows;
        // layer-0 input: 20 features per row, padded to 32, rows past n zero
        for (int e = tid; e < kTcMlpRows * kL0K / 2; e += blockDim.x) {
            const int row = e / (kL0K / 2), k = 2 * (e - row * (kL0K / 2));
            float a = 0.f, b = 0.f;
            if (r0 + row < n && k < kMlpIn) {
                a = x[(size_t)(r0 + row) * kMlpIn + k];
                b = x[(size_t)(r0 + row) * kMlpIn + k + 1];
            }
            *reinterpret_cast<uint32_t*>(sA + core_off(row, k, kL0K / 8)) = pack_bf16x2(a, b);
        }
        for (int l = 0; l < kLayers; ++l) {
            const int K = l == 0 ? kL0K : kMlpHidden;
            const int N = l == kLayers - 1 ? kOutN : kMlpHidden;
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) {
                if (!wait_parity(smem_u32(&s_wbar), wphase)) s_fail = 1;
                wphase ^= 1;
                pending_w = 0;
                if (!s_fail) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t idesc = mma_idesc(kTcMlpRows, N);
                    for (int ks = 0; ks < K / 16; ++ks) {
                        const uint64_t ad = smem_desc(smem_u32(sA) + ks * 256, 128, (K / 8) * 128);
                        const uint64_t bd = smem_desc(smem_u32(sW) + ks * 256, 128, (K / 8) * 128);
                        const uint32_t acc = ks > 0 ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                    mma_commit(smem_u32(&s_mbar));
                    if (!wait_parity(smem_u32(&s_mbar), mphase)) { s_fail = 1; pending_m = 1; }
                    // the weights and the layer input are free: request the next weights
                    const int nl = l + 1 < kLayers ? l + 1 : 0;
                    const bool more = l + 1 < kLayers || tile + (int)gridDim.x < ntiles;
                    if (!s_fail && more) { load_w(nl); pending_w = 1; }
                }
                mphase ^= 1;
            }
            __syncthreads();
            if (s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int row = lq * 32 + lane;
            const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16);
            if (l < kLayers - 1) {
                // bias + GELU of this warp's 64 columns, written back as the next input
#pragma unroll 1
                for (int c0 = quarter * 64; c0 < quarter * 64 + 64; c0 += 32) {
                    uint32_t v[32];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                        : "r"(tl + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    const float* bias = s_bias[l] + c0;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        uint4 q;
                        q.x = pack_bf16x2(gelu(__uint_as_float(v[8 * g + 0]) + bias[8 * g + 0]),
                                          gelu(__uint_as_float(v[8 * g + 1]) + bias[8 * g + 1]));
                        q.y = pack_bf16x2(gelu(__uint_as_float(v[8 * g + 2]) + bias[8 * g + 2]),
                                          gelu(__uint_as_float(v[8 * g + 3]) + bias[8 * g + 3]));
                        q.z = pack_bf16x2(gelu(__uint_as_float(v[8 * g + 4]) + bias[8 * g + 4]),
                                          gelu(__uint_as_float(v[8 * g + 5]) + bias[8 * g + 5]));
                        q.w = pack_bf16x2(gelu(__uint_as_float(v[8 * g + 6]) + bias[8 * g + 6]),
                                          gelu(__uint_as_float(v[8 * g + 7]) + bias[8 * g + 7]));
                        *reinterpret_cast<uint4*>(sA + core_off(row, c0 + 8 * g, kMlpHidden / 8)) = q;
                    }
                }
            } else if (quarter == 0) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(tl));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (r0 + row < n)
#pragma unroll
                    for (int j = 0; j < kMlpOut; ++j)
                        y[(size_t)(r0 + row) * kMlpOut + j] = __uint_as_float(v[j]) + s_bias[kLayers - 2][kMlpHidden + j];
            }
        }
    }
    // after a failed wait: a copy or products still in flight must end before exit
    if (tid == 0 && pending_w) wait_parity(smem_u32(&s_wbar), wphase);
    if (tid == 0 && pending_m) wait_parity(smem_u32(&s_mbar), mphase ^ 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpHidden));
    if (s_fail && tid == 0) atomicExch(err, 2);
}

// weight operand of layer l in the shared-memory layout: row = output unit
// (N rows, zero past the layer's outputs), k = input (zero past its inputs)
__global__ void k_mlp_prepare_tc(const __nv_bfloat16* __restrict__ W, int out, int in, int N, int K,
                                 __nv_bfloat16* __restrict__ dst) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * K) return;
    const int r = e / K, k = e - r * K;
    const __nv_bfloat16 v = (r < out && k < in) ? W[(size_t)r * in + k] : __float2bfloat16_rn(0.f);
    dst[core_off(r, k, K / 8) / 2] = v;
}

// Training set: one warp per fingerprint.  alpha = rho sig Phi + sigma noise
// with sigma^2 = ||rho sig Phi||^2 / K 10^(-snr / 10); x = alpha / ||alpha||
// as (Re, Im); y = (u1, u2, rho / ||alpha|| / pd_scale) with u the log T maps
// of [Tmin, Tmax] onto [-1, 1].
struct Ranges {
    float t1min, t1max, t2min, t2max, pd_scale;
};

__global__ void k_training_set(const float2* __restrict__ sig, const float* __restrict__ t1t2,
                               const float* __restrict__ rho, const float* __restrict__ snr_db,
                               const float2* __restrict__ noise, int n, int T, const float2* __restrict__ phi, int K,
                               Ranges rg, float* __restrict__ x, float* __restrict__ y) {
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    float re[16], im[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { re[k] = 0.f; im[k] = 0.f; }
    const float2* d = sig + (size_t)i * T;
    for (int t = lane; t < T; t += 32) {
        const float2 v = d[t];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < K) {
                const float2 p = phi[(size_t)t * K + k];
                re[k] += v.x * p.x - v.y * p.y;
                im[k] += v.x * p.y + v.y * p.x;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re[k] += __shfl_xor_sync(0xffffffffu, re[k], o);
            im[k] += __shfl_xor_sync(0xffffffffu, im[k], o);
        }
    }
    if (lane != 0) return;
    const float r = rho[i];
    float s2 = 0.f;
    for (int k = 0; k < K; ++k) {
        re[k] *= r;
        im[k] *= r;
        s2 += re[k] * re[k] + im[k] * im[k];
    }
    const float sigma = sqrtf(s2 / K) * powf(10.f, -snr_db[i] / 20.f);
    float n2 = 0.f;
    for (int k = 0; k < K; ++k) {
        re[k] += sigma * noise[(size_t)i * K + k].x;
        im[k] += sigma * noise[(size_t)i * K + k].y;
        n2 += re[k] * re[k] + im[k] * im[k];
    }
    const float nrm = sqrtf(n2), inv = nrm > 0.f ? 1.f / nrm : 0.f;
    for (int k = 0; k < K; ++k) {
        x[(size_t)i * 2 * K + 2 * k] = re[k] * inv;
        x[(size_t)i * 2 * K + 2 * k + 1] = im[k] * inv;
    }
    const float l1 = logf(rg.t1min), l1r = logf(rg.t1max) - l1, l2 = logf(rg.t2min), l2r = logf(rg.t2max) - l2;
    y[(size_t)i * 3 + 0] = 2.f * (logf(t1t2[2 * i]) - l1) / l1r - 1.f;
    y[(size_t)i * 3 + 1] = 2.f * (logf(t1t2[2 * i + 1]) - l2) / l2r - 1.f;
    y[(size_t)i * 3 + 2] = r * inv / rg.pd_scale;
}

__global__ void k_mlp_features(const float2* __restrict__ alpha, int n, float* __restrict__ x,
                               float* __restrict__ norm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 a[kMlpIn / 2];
    float n2 = 0.f;
#pragma unroll
    for (int k = 0; k < kMlpIn / 2; ++k) {
        a[k] = alpha[(size_t)i * (kMlpIn / 2) + k];
        n2 += a[k].x * a[k].x + a[k].y * a[k].y;
    }
    const float nrm = sqrtf(n2), inv = nrm > 0.f ? 1.f / nrm : 0.f;
#pragma unroll
    for (int k = 0; k < kMlpIn / 2; ++k) {
        x[(size_t)i * kMlpIn + 2 * k] = a[k].x * inv;
        x[(size_t)i * kMlpIn + 2 * k + 1] = a[k].y * inv;
    }
    norm[i] = nrm;
}

}  // namespace mrf

struct mrf_mlp_s {
    mrf::Layout L{};
    float* w = nullptr;             // [P] FP32 master weights and biases
    __nv_bfloat16* wb = nullptr;    // [P] BF16 copy (weights used in the products)
    __nv_bfloat16* wt = nullptr;    // [P] transposed BF16 weights for inference
    float *g = nullptr, *m = nullptr, *v = nullptr;
    int max_batch = 0;
    float* ws = nullptr;            // activations and their gradients for max_batch rows
    float* z[mrf::kLayers] = {};
    float* a[mrf::kLayers] = {};
    float *d0 = nullptr, *d1 = nullptr;
    long long step = 0;
    bool wt_fresh = false;
    unsigned char* wtc = nullptr;   // tensor-core weight operands, layer by layer
    bool tensor_cores = true;       // inference and training products on tcgen05 (false: SIMT kernels)
    int* err = nullptr;             // set when a bounded device wait gave up
    float decode[5] = {};
};

namespace mrf {

// operand sizes (bytes) of the tensor-core inference per layer
static int tc_rows(int l) { return l == kLayers - 1 ? kOutN : kMlpHidden; }
static int tc_k(int l) { return l == 0 ? kL0K : kMlpHidden; }
static size_t tc_offset(int l) {
    size_t at = 0;
    for (int i = 0; i < l; ++i) at += (size_t)tc_rows(i) * tc_k(i) * 2;
    return at;
}

static mrf_status refresh_transposed(mrf_mlp_s* N, cudaStream_t s) {
    if (N->wt_fresh) return MRF_OK;
    for (int l = 0; l < kLayers; ++l) {
        const int out = kSizes[l + 1], in = kSizes[l];
        k_transpose_w<<<(out * in + 255) / 256, 256, 0, s>>>(N->wb + N->L.w[l], out, in, N->wt + N->L.w[l]);
        MRF_LAUNCHED_AS("k_transpose_w", s);
        const int R = tc_rows(l), K = tc_k(l);
        k_mlp_prepare_tc<<<(R * K + 255) / 256, 256, 0, s>>>(
            N->wb + N->L.w[l], out, in, R, K, reinterpret_cast<__nv_bfloat16*>(N->wtc + tc_offset(l)));
        MRF_LAUNCHED_AS("k_mlp_prepare_tc", s);
    }
    N->wt_fresh = true;
    return MRF_OK;
}

static mrf_status mlp_infer_tc(mrf_mlp_s* N, const float* x, int n, float* y, cudaStream_t s) {
    TcInferParams P;
    for (int l = 0; l < kLayers; ++l) {
        P.w[l] = N->wtc + tc_offset(l);
        P.wbytes[l] = tc_rows(l) * tc_k(l) * 2;
        P.b[l] = N->w + N->L.b[l];
    }
    const size_t sm = (size_t)kABytes + kWBytes;
    MRF_CUDA(cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int tiles = (n + kTcMlpRows - 1) / kTcMlpRows;
    int dev = 0, sms = 152;
    MRF_CUDA(cudaGetDevice(&dev));
    MRF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    k_mlp_infer_tc<<<std::min(tiles, sms), 32 * kTcMlpWarps, sm, s>>>(P, x, n, y, N->err);
    MRF_LAUNCHED_AS("k_mlp_infer_tc", s);
    return MRF_OK;
}

mrf_status mlp_infer(mrf_mlp_s* N, const float* x, int n, float* y, cudaStream_t s) {
    MRF_REQUIRE(N && x && y && n >= 0, "mlp_infer: bad arguments");
    if (n == 0) return MRF_OK;
    MRF_PROPAGATE(refresh_transposed(N, s));
    if (N->tensor_cores) return mlp_infer_tc(N, x, n, y, s);
    InferParams P;
    for (int l = 0; l < kLayers; ++l) {
        P.wt[l] = N->wt + N->L.w[l];
        P.b[l] = N->w + N->L.b[l];
    }
    const size_t sm = sizeof(float) * 2 * kInfRows * kInfLd;
    MRF_CUDA(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_mlp_infer<<<(n + kInfRows - 1) / kInfRows, kMlpHidden, sm, s>>>(P, x, n, y);
    MRF_LAUNCHED_AS("k_mlp_infer", s);
    return MRF_OK;
}

mrf_status mlp_features(const float2* alpha, int n, float* x, float* norm, cudaStream_t s) {
    if (n == 0) return MRF_OK;
    k_mlp_features<<<(n + 255) / 256, 256, 0, s>>>(alpha, n, x, norm);
    MRF_LAUNCHED_AS("k_mlp_features", s);
    return MRF_OK;
}

const float* mlp_decode(const mrf_mlp_s* N) { return N->decode; }

static unsigned nblk(size_t n) { return (unsigned)((n + 255) / 256); }

// forward pass of B rows, then the loss and the gradient into N->g
static mrf_status forward_backward(mrf_mlp_s* N, const float* x, const float* t, int B, float* loss,
                                   cudaStream_t s) {
    const float* h = x;
    for (int l = 0; l < kLayers; ++l) {
        const int in = kSizes[l], out = kSizes[l + 1];
        // Z = H W^T: B(k, n) = W[n][k]
        MRF_PROPAGATE(gemm(B, out, in, h, in, 1, N->wb + N->L.w[l], 1, in, N->z[l], out, false, s, N->tensor_cores,
                           N->err));
        k_bias_act<<<nblk((size_t)B * out), 256, 0, s>>>(N->z[l], N->w + N->L.b[l], B, out, l < kLayers - 1,
                                                          N->a[l]);
        MRF_LAUNCHED_AS("k_mlp_bias_act", s);
        h = N->a[l];
    }
    float* dz = N->d0;
    k_loss<<<1, 256, 0, s>>>(N->z[kLayers - 1], t, B * kMlpOut, 1.f / B, dz, loss);
    MRF_LAUNCHED_AS("k_mlp_loss", s);
    for (int l = kLayers - 1; l >= 0; --l) {
        const int in = kSizes[l], out = kSizes[l + 1];
        const float* hin = l > 0 ? N->a[l - 1] : x;
        // dW = dZ^T H: A(m, k) = dZ[k][m], B(k, n) = H[k][n]
        MRF_PROPAGATE(gemm(out, in, B, dz, 1, out, hin, in, 1, N->g + N->L.w[l], in, false, s, N->tensor_cores,
                           N->err));
        k_bias_grad<<<(out + 255) / 256, 256, 0, s>>>(dz, B, out, N->g + N->L.b[l]);
        MRF_LAUNCHED_AS("k_mlp_bias_grad", s);
        if (l > 0) {
            float* dh = dz == N->d0 ? N->d1 : N->d0;
            // dH = dZ W: B(k, n) = W[k][n]
            MRF_PROPAGATE(gemm(B, in, out, dz, out, 1, N->wb + N->L.w[l], in, 1, dh, in, false, s, N->tensor_cores,
                               N->err));
            k_gelu_bwd<<<nblk((size_t)B * in), 256, 0, s>>>(dh, N->z[l - 1], (size_t)B * in, dh);
            MRF_LAUNCHED_AS("k_mlp_gelu_bwd", s);
            dz = dh;
        }
    }
    return MRF_OK;
}

}  // namespace mrf

using namespace mrf;

extern "C" mrf_status mrf_mlp_create(mrf_mlp* out, const float* params, int nparams, const float* decode,
                                     int max_batch) {
    MRF_REQUIRE(out && params && decode, "mrf_mlp_create: NULL argument");
    const Layout L = layout();
    MRF_REQUIRE((size_t)nparams == L.total, "mrf_mlp_create: expected %zu parameters (got %d)", L.total, nparams);
    MRF_REQUIRE(max_batch >= 1 && max_batch <= (1 << 20), "mrf_mlp_create: max_batch must be in [1, 2^20]");
    MRF_REQUIRE(decode[0] > 0.f && decode[1] > decode[0] && decode[2] > 0.f && decode[3] > decode[2] &&
                    decode[4] > 0.f,
                "mrf_mlp_create: decode needs 0 < t1min < t1max, 0 < t2min < t2max, pd_scale > 0");
    *out = nullptr;
    auto* N = new mrf_mlp_s();
    N->L = L;
    N->max_batch = max_batch;
    for (int i = 0; i < 5; ++i) N->decode[i] = decode[i];
    const size_t P = L.total;
    size_t per_row = 0;
    for (int l = 0; l < kLayers; ++l) per_row += 2 * (size_t)kSizes[l + 1];
    per_row += 2 * (size_t)kMlpHidden;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    A(reinterpret_cast<void**>(&N->w), sizeof(float) * P);
    A(reinterpret_cast<void**>(&N->wb), sizeof(__nv_bfloat16) * P);
    A(reinterpret_cast<void**>(&N->wt), sizeof(__nv_bfloat16) * P);
    A(reinterpret_cast<void**>(&N->g), sizeof(float) * P);
    A(reinterpret_cast<void**>(&N->m), sizeof(float) * P);
    A(reinterpret_cast<void**>(&N->v), sizeof(float) * P);
    A(reinterpret_cast<void**>(&N->ws), sizeof(float) * per_row * max_batch);
    A(reinterpret_cast<void**>(&N->wtc), tc_offset(kLayers));
    A(reinterpret_cast<void**>(&N->err), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(N->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(N->w, params, sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(N->m, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(N->v, 0, sizeof(float) * P);
    if (e == cudaSuccess) {
        k_to_bf16<<<(unsigned)((P + 255) / 256), 256>>>(N->w, P, N->wb);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        set_error("mrf_mlp_create: %s", cudaGetErrorString(e));
        cudaFree(N->w); cudaFree(N->wb); cudaFree(N->wt); cudaFree(N->g); cudaFree(N->m); cudaFree(N->v);
        cudaFree(N->ws); cudaFree(N->wtc); cudaFree(N->err);
        delete N;
        return MRF_ECUDA;
    }
    float* p = N->ws;
    for (int l = 0; l < kLayers; ++l) {
        N->z[l] = p;
        p += (size_t)kSizes[l + 1] * max_batch;
        N->a[l] = p;
        p += (size_t)kSizes[l + 1] * max_batch;
    }
    N->d0 = p;
    p += (size_t)kMlpHidden * max_batch;
    N->d1 = p;
    *out = N;
    return MRF_OK;
}

extern "C" mrf_status mrf_mlp_destroy(mrf_mlp N) {
    if (!N) return MRF_OK;
    cudaFree(N->w); cudaFree(N->wb); cudaFree(N->wt); cudaFree(N->g); cudaFree(N->m); cudaFree(N->v);
    cudaFree(N->ws); cudaFree(N->wtc); cudaFree(N->err);
    delete N;
    return MRF_OK;
}

extern "C" mrf_status mrf_mlp_get_params(mrf_mlp N, float* params, float* params_bf16) {
    MRF_REQUIRE(N && params, "mrf_mlp_get_params: NULL argument");
    const size_t P = N->L.total;
    MRF_CUDA(cudaDeviceSynchronize());
    MRF_CUDA(cudaMemcpy(params, N->w, sizeof(float) * P, cudaMemcpyDeviceToHost));
    if (params_bf16) {
        std::vector<__nv_bfloat16> h(P);
        MRF_CUDA(cudaMemcpy(h.data(), N->wb, sizeof(__nv_bfloat16) * P, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < P; ++i) params_bf16[i] = __bfloat162float(h[i]);
    }
    return MRF_OK;
}

extern "C" mrf_status mrf_mlp_grad(mrf_mlp N, const float* x, const float* t, int B, float* grad, float* loss,
                                   mrf_stream stream) {
    MRF_REQUIRE(N && x && t && grad, "mrf_mlp_grad: NULL argument");
    MRF_REQUIRE(B >= 1 && B <= N->max_batch, "mrf_mlp_grad: batch %d outside [1, %d]", B, N->max_batch);
    cudaStream_t s = as_stream(stream);
    MRF_PROPAGATE(forward_backward(N, x, t, B, loss, s));
    MRF_CUDA(cudaMemcpyAsync(grad, N->g, sizeof(float) * N->L.total, cudaMemcpyDeviceToDevice, s));
    return MRF_OK;
}

extern "C" mrf_status mrf_mlp_train_step(mrf_mlp N, const float* x, const float* t, int B, float lr, float* loss,
                                         mrf_stream stream) {
    MRF_REQUIRE(N && x && t, "mrf_mlp_train_step: NULL argument");
    MRF_REQUIRE(B >= 1 && B <= N->max_batch, "mrf_mlp_train_step: batch %d outside [1, %d]", B, N->max_batch);
    MRF_REQUIRE(lr > 0.f, "mrf_mlp_train_step: lr must be > 0");
    cudaStream_t s = as_stream(stream);
    MRF_PROPAGATE(forward_backward(N, x, t, B, loss, s));
    ++N->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)N->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)N->step)));
    const size_t P = N->L.total;
    k_adam<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(N->w, N->wb, N->g, N->m, N->v, P, lr, b1, b2, 1e-8f, c1, c2);
    MRF_LAUNCHED_AS("k_mlp_adam", s);
    N->wt_fresh = false;
    return MRF_OK;
}

extern "C" mrf_status mrf_mlp_infer(mrf_mlp N, const float* x, int n, float* y, mrf_stream stream) {
    return mlp_infer(N, x, n, y, as_stream(stream));
}

extern "C" mrf_status mrf_mlp_set_engine(mrf_mlp N, int tensor_cores) {
    MRF_REQUIRE(N, "mrf_mlp_set_engine: NULL network");
    N->tensor_cores = tensor_cores != 0;
    return MRF_OK;
}

extern "C" mrf_status mrf_mlp_check(mrf_mlp N, mrf_stream stream) {
    MRF_REQUIRE(N, "mrf_mlp_check: NULL network");
    int h = 0;
    cudaStream_t s = as_stream(stream);
    MRF_CUDA(cudaMemcpyAsync(&h, N->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    if (h) {
        set_error("mrf_mlp: a tensor-core wait timed out");
        return MRF_ETIMEOUT;
    }
    return MRF_OK;
}

extern "C" mrf_status mrf_mlp_training_set(const mrf_c64* sig, const float* t1t2, const float* rho,
                                           const float* snr_db, const mrf_c64* noise, int n, int T,
                                           const mrf_c64* phi, int K, const float* ranges, float* x, float* y,
                                           mrf_stream stream) {
    MRF_REQUIRE(sig && t1t2 && rho && snr_db && noise && phi && ranges && x && y,
                "mrf_mlp_training_set: NULL argument");
    MRF_REQUIRE(n >= 0 && T >= 1 && K >= 1 && K <= 16, "mrf_mlp_training_set: bad sizes");
    if (n == 0) return MRF_OK;
    Ranges rg{ranges[0], ranges[1], ranges[2], ranges[3], ranges[4]};
    cudaStream_t s = as_stream(stream);
    const size_t thr = (size_t)n * 32;
    k_training_set<<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float2*>(sig), t1t2, rho, snr_db, reinterpret_cast<const float2*>(noise), n, T,
        reinterpret_cast<const float2*>(phi), K, rg, x, y);
    MRF_LAUNCHED_AS("k_training_set", s);
    return MRF_OK;
}

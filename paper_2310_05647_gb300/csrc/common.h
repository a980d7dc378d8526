// Shared host/device helpers of the MS-LLR CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>

#include "mrf.h"

namespace mrf {

// Thread-local error message, read back through mrf_last_error().
void set_error(const char* fmt, ...);

// Launch accounting and the optional per-kernel CUDA-event profiler: every
// launch site reports itself after the launch; with profiling on, an event is
// recorded on the launching stream and the interval since the previous event
// on that stream is charged to the kernel.
void note_launch(const char* name, cudaStream_t s);
// kernels launched so far (every launch site's report), and a CUDA graph
// replay's kernels added to that count
long long launches_so_far();
void note_replayed_launches(long long n);
// the per-kernel profiler is recording (launches must then go one by one)
bool profiling_enabled();

inline cudaStream_t as_stream(mrf_stream s) { return reinterpret_cast<cudaStream_t>(s); }

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

}  // namespace mrf

#define MRF_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            mrf::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call,            \
                           cudaGetErrorString(e_));                                      \
            return e_ == cudaErrorMemoryAllocation ? MRF_ENOMEM : MRF_ECUDA;             \
        }                                                                                \
    } while (0)

#define MRF_REQUIRE(cond, ...)                                                           \
    do {                                                                                 \
        if (!(cond)) {                                                                   \
            mrf::set_error(__VA_ARGS__);                                                 \
            return MRF_EINVAL;                                                           \
        }                                                                                \
    } while (0)

#define MRF_LAUNCHED_AS(name, stream)                                                    \
    do {                                                                                 \
        MRF_CUDA(cudaGetLastError());                                                    \
        mrf::note_launch(name, stream);                                                  \
    } while (0)

#define MRF_PROPAGATE(expr)                                                              \
    do {                                                                                 \
        mrf_status s_ = (expr);                                                          \
        if (s_ != MRF_OK) return s_;                                                     \
    } while (0)

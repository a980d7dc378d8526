// Learned signal-to-parameter matcher (internal interface for the loop).
#pragma once
#include "common.h"

struct mrf_mlp_s;

namespace mrf {

constexpr int kMlpIn = 20;        // K = 10 complex coefficients as (Re, Im)
constexpr int kMlpHidden = 256;
constexpr int kMlpOut = 3;        // normalised log T1, log T2, PD per unit input norm

// x [n][20] and ||alpha|| [n] of fingerprints alpha [n][10]
mrf_status mlp_features(const float2* alpha, int n, float* x, float* norm, cudaStream_t s);
// y [n][3] = network(x)
mrf_status mlp_infer(mrf_mlp_s* net, const float* x, int n, float* y, cudaStream_t s);
// decode constants (t1min, t1max, t2min, t2max, pd_scale)
const float* mlp_decode(const mrf_mlp_s* net);

}  // namespace mrf

// BF16 tensor-core matching (candidate search + FP32 re-rank).
#include "common.h"
#include "match.h"

namespace mrf {
mrf_status match_bf16_candidates(MatchWorkspace&, const float2*, int, int, const float2*, int, cudaStream_t) {
    set_error("BF16 matching is not built yet");
    return MRF_EUNSUPPORTED;
}
mrf_status match_rerank(MatchWorkspace&, const float2*, int, int, const float2*, cudaStream_t) {
    set_error("BF16 matching is not built yet");
    return MRF_EUNSUPPORTED;
}
}  // namespace mrf

// Algorithm 1 (MS-LLR) loop -- placeholder until the loop kernels land.
#include "common.h"

extern "C" mrf_status mrf_recon_create(mrf_recon* out, mrf_plan, const mrf_recon_params*, const mrf_c64*, int,
                                       const mrf_c64*, const float*, const float*, int, const mrf_c64*,
                                       mrf_stream) {
    if (out) *out = nullptr;
    mrf::set_error("mrf_recon_create: not built yet");
    return MRF_EUNSUPPORTED;
}
extern "C" mrf_status mrf_recon_iter(mrf_recon, int, double*, mrf_stream) { return MRF_EUNSUPPORTED; }
extern "C" mrf_status mrf_recon_maps(mrf_recon, float*, float*, float*, int*, mrf_stream) { return MRF_EUNSUPPORTED; }
extern "C" mrf_status mrf_recon_alpha(mrf_recon, mrf_c64*, mrf_stream) { return MRF_EUNSUPPORTED; }
extern "C" mrf_status mrf_recon_info(mrf_recon, double*, double*, double*, double*, mrf_stream) { return MRF_EUNSUPPORTED; }
extern "C" mrf_status mrf_recon_destroy(mrf_recon) { return MRF_OK; }
extern "C" mrf_status mrf_dict_subspace(const mrf_c64*, int, int, int, mrf_c64*, mrf_c64*, float*, mrf_stream) {
    mrf::set_error("mrf_dict_subspace: not built yet");
    return MRF_EUNSUPPORTED;
}

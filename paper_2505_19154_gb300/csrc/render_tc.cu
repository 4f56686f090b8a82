// tcgen05 tensor-core render kernels (feature blend as W(P x B) . F(B x D)).
#include "fhgs_internal.cuh"

namespace fhgs {

int tc_supported(int D, int d_split) {
    (void)D;
    (void)d_split;
    return 0;
}

void launch_render_fwd_tc(long long, const CamSet &, const Params &, ProjView, const fhgs_bins &,
                          const __nv_bfloat16 *, int, int, float *, float *, float *, int32_t *, unsigned *,
                          cudaStream_t) {}

void launch_render_bwd_tc(long long, const CamSet &, const Params &, ProjView, const fhgs_bins &,
                          const __nv_bfloat16 *, int, int, const float *, const int32_t *, const float *,
                          const float *, float *, float *, unsigned *, cudaStream_t) {}

}  // namespace fhgs

// k_force_lc_f32.cu -- Linked Cells force kernels, pair arithmetic in float.
#include "k_force_dispatch.cuh"

namespace ljgb {
cudaError_t force_lc_f32(Ctx& c, const lj_config& cfg, bool ev) { return force_lc_t<float>(c, cfg, ev); }
}  // namespace ljgb

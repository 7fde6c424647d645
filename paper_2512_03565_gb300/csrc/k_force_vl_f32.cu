// k_force_vl_f32.cu -- Verlet-list force kernels, pair arithmetic in float.
#include "k_force_dispatch.cuh"

namespace ljgb {
cudaError_t force_vl_f32(Ctx& c, const lj_config& cfg, bool ev) { return force_vl_t<float>(c, cfg, ev); }
}  // namespace ljgb

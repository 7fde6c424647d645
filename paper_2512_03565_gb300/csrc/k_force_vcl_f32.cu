// k_force_vcl_f32.cu -- Verlet-cluster-list force kernels, pair arithmetic in float.
#include "k_force_vcl.cuh"

namespace ljgb {
cudaError_t force_vcl_f32(Ctx& c, const lj_config& cfg, bool ev) { return force_vcl_t<float>(c, cfg, ev); }
}  // namespace ljgb

// k_force_vl_f64.cu -- Verlet-list force kernels, pair arithmetic in double.
#include "k_force_dispatch.cuh"

namespace ljgb {
cudaError_t force_vl_f64(Ctx& c, const lj_config& cfg, bool ev) { return force_vl_t<double>(c, cfg, ev); }
}  // namespace ljgb

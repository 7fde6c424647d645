// k_force_vcl_f64.cu -- Verlet-cluster-list force kernels, pair arithmetic in double.
#include "k_force_vcl.cuh"

namespace ljgb {
cudaError_t force_vcl_f64(Ctx& c, const lj_config& cfg, bool ev) { return force_vcl_t<double>(c, cfg, ev); }
}  // namespace ljgb

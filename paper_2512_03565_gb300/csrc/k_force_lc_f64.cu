// k_force_lc_f64.cu -- Linked Cells force kernels, pair arithmetic in double.
#include "k_force_dispatch.cuh"

namespace ljgb {
cudaError_t force_lc_f64(Ctx& c, const lj_config& cfg, bool ev) { return force_lc_t<double>(c, cfg, ev); }
}  // namespace ljgb

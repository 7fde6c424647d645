// tune.cu -- run-time selection of the configuration (Sec. 2.3.2 full search,
// extended to the interaction order as in Sec. 4; Sec. 6's data-driven
// tuning as a learned ranking).
//
// Full search: every valid configuration runs a warm-up evaluation and then
// `samples` timed force evaluations (CUDA events on the context's stream);
// the evidence is reduced by the mean and the fastest configuration wins.
// The cost of a configuration is that of one MD step's force work: Linked
// Cells rebin at every step, so each timed evaluation includes the binning;
// Verlet lists add the list build amortised over the rebuild period.
//
// Learned: the MLP (k_mlp.cu) predicts the log time of its configurations
// from the 16 features; the best predicted valid configuration is taken, or
// the fastest of the top `samples` predictions after timing them.  Systems
// whose standardised features lie beyond kMaxFeatureZ fall back to full search.
#include <cmath>
#include <limits>
#include <numeric>

#include "ljgb_internal.cuh"

namespace ljgb {
cudaError_t mlp_forward_dev(const float* d_params, int C, const float* d_X, int64_t M, float* d_Y, cudaStream_t s);
}

using namespace ljgb;

namespace {

// A standardised feature beyond this many training standard deviations puts
// the system outside the learned tuner's training data.
constexpr double kMaxFeatureZ = 8.0;

lj_status tfail(Ctx& c, lj_status s, const std::string& m) {
  c.err = m;
  return s;
}

// Mean time (ms) of `samples` force evaluations of cfg; VL adds the list
// build time over the rebuild period.
lj_status time_config(lj_ctx* h, const lj_config& cfg, int samples, double& ms) {
  Ctx& c = h->c;
  lj_status st = lj_compute_forces(h, cfg, nullptr, nullptr);  // warm-up, builds lists
  if (st != LJ_OK) return st;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return tfail(c, LJ_ERR_CUDA, "cudaEventCreate");
  double total = 0.0;
  for (int s = 0; s < samples && st == LJ_OK; ++s) {
    if (cfg.container == LJ_LC || cfg.container == LJ_LCS) c.moved = true;  // a step's rebin is part of the cost
    cudaEventRecord(e0, c.stream);
    st = lj_compute_forces(h, cfg, nullptr, nullptr);
    cudaEventRecord(e1, c.stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = tfail(c, LJ_ERR_CUDA, "cudaEventSynchronize");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    total += t;
  }
  double build = 0.0;
  if (st == LJ_OK && cfg.container != LJ_LC && cfg.container != LJ_LCS) {
    c.moved_since_build = true;
    c.vl_valid = false;  // force one rebuild to time it
    c.vcl_valid = false;
    cudaEventRecord(e0, c.stream);
    st = lj_compute_forces(h, cfg, nullptr, nullptr);
    cudaEventRecord(e1, c.stream);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    const double one = samples > 0 ? total / samples : 0.0;
    build = std::max(0.0, (double)t - one) / std::max(1, c.rebuild_every);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LJ_OK) return st;
  ms = (samples > 0 ? total / samples : 0.0) + build;
  return LJ_OK;
}

}  // namespace

extern "C" {

int32_t lj_tune_select(const double* timings, int32_t n_cfg, int32_t samples, const int32_t* valid, int32_t reduce) {
  if (!timings || n_cfg < 1 || samples < 1) return -1;
  int32_t best = -1;
  double best_v = std::numeric_limits<double>::infinity();
  for (int32_t k = 0; k < n_cfg; ++k) {
    if (valid && !valid[k]) continue;
    double acc = reduce == 1 ? std::numeric_limits<double>::infinity() : 0.0;
    int cnt = 0;
    for (int32_t s = 0; s < samples; ++s) {
      const double t = timings[(int64_t)k * samples + s];
      if (std::isnan(t)) continue;
      acc = reduce == 1 ? std::min(acc, t) : acc + t;
      ++cnt;
    }
    if (cnt == 0) continue;
    const double v = reduce == 1 ? acc : acc / cnt;
    if (v < best_v) {
      best_v = v;
      best = k;
    }
  }
  return best;
}

lj_status lj_tuner_set_model(lj_ctx* h, const float* params, int32_t C, const float* feat_mean,
                             const float* feat_std, const lj_config* cfgs) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (!params || C < 1 || !feat_mean || !feat_std || !cfgs) return tfail(c, LJ_ERR_ARG, "bad tuner model");
  const int64_t P = 64 * 16 + 64 + 64 * 64 + 64 + (int64_t)C * 64 + C;
  c.mlp_params.assign(params, params + P);
  c.mlp_mean.assign(feat_mean, feat_mean + 16);
  c.mlp_std.assign(feat_std, feat_std + 16);
  c.mlp_cfgs.assign(cfgs, cfgs + C);
  c.mlp_C = C;
  return LJ_OK;
}

lj_status lj_tune(lj_ctx* h, int32_t kind, int32_t samples, lj_config* chosen, double* times_ms) {
  if (!h || !chosen) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (!c.have_particles) return tfail(c, LJ_ERR_STATE, "no particles loaded");
  if (samples < 0) return tfail(c, LJ_ERR_ARG, "samples must be >= 0");
  std::vector<lj_config> all(lj_config_list(nullptr, 0));
  lj_config_list(all.data(), (int32_t)all.size());
  if (times_ms)
    for (size_t k = 0; k < all.size(); ++k) times_ms[k] = std::numeric_limits<double>::quiet_NaN();
  auto index_of = [&](const lj_config& g) -> int {
    for (size_t k = 0; k < all.size(); ++k)
      if (all[k].container == g.container && all[k].order == g.order && all[k].param == g.param &&
          all[k].newton3 == g.newton3)
        return (int)k;
    return -1;
  };
  // configurations usable on this machine (both cell grids need >= 3 cells per axis)
  auto usable = [&](const lj_config& g) {
    return lj_config_valid(g) && (g.container == LJ_LC    ? c.nc_lc >= 3
                                  : g.container == LJ_LCS ? c.nc_lcs >= 5
                                  : g.container == LJ_VL  ? c.nc_vl >= 3
                                                          : true);
  };
  std::vector<lj_config> cand;
  if (kind == 1 && c.mlp_C > 0) {
    double f[16];
    lj_status st = lj_features(h, f);
    if (st != LJ_OK) return st;
    float xin[16];
    bool in_range = true;
    for (int k = 0; k < 16; ++k) {
      xin[k] = (float)((f[k] - c.mlp_mean[k]) / (c.mlp_std[k] > 0 ? c.mlp_std[k] : 1.0f));
      if (!(std::fabs(xin[k]) <= kMaxFeatureZ)) in_range = false;
    }
    if (!in_range) {
      // the system lies outside the training data: full search instead
      return lj_tune(h, 0, samples > 0 ? samples : 1, chosen, times_ms);
    }
    float *dp = nullptr, *dx = nullptr, *dy = nullptr;
    std::vector<float> y(c.mlp_C);
    cudaError_t e = cudaMalloc(&dp, c.mlp_params.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dx, 16 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dy, c.mlp_C * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dp, c.mlp_params.data(), c.mlp_params.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, xin, sizeof(xin), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = mlp_forward_dev(dp, c.mlp_C, dx, 1, dy, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y.data(), dy, c.mlp_C * sizeof(float), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    cudaFree(dp);
    cudaFree(dx);
    cudaFree(dy);
    if (e != cudaSuccess) return tfail(c, LJ_ERR_CUDA, cudaGetErrorString(e));
    std::vector<int> idx;
    for (int k = 0; k < c.mlp_C; ++k)
      if (usable(c.mlp_cfgs[k]) && std::isfinite(y[k])) idx.push_back(k);
    if (idx.empty()) return tfail(c, LJ_ERR_STATE, "no usable configuration predicted");
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return y[a] < y[b]; });
    if (samples == 0) {
      *chosen = c.mlp_cfgs[idx[0]];
      return LJ_OK;
    }
    for (int k = 0; k < (int)idx.size() && k < samples; ++k) cand.push_back(c.mlp_cfgs[idx[k]]);
    samples = 3;
  } else {
    for (const lj_config& g : all)
      if (usable(g)) cand.push_back(g);
    if (samples == 0) samples = 1;
  }
  std::vector<double> t(cand.size(), std::numeric_limits<double>::quiet_NaN());
  for (size_t k = 0; k < cand.size(); ++k) {
    double ms = 0.0;
    lj_status st = time_config(h, cand[k], samples, ms);
    if (st != LJ_OK) return st;
    t[k] = ms;
    const int gi = index_of(cand[k]);
    if (times_ms && gi >= 0) times_ms[gi] = ms;
  }
  const int32_t best = lj_tune_select(t.data(), (int32_t)t.size(), 1, nullptr, 0);
  if (best < 0) return tfail(c, LJ_ERR_STATE, "no configuration could be timed");
  *chosen = cand[best];
  return LJ_OK;
}

}  // extern "C"

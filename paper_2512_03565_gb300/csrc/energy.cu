// energy.cu -- energy consumption as the tuning metric (Sec. 2.3.3: the
// tuner may choose the configuration by the energy measured over its
// evaluations instead of their time; Sec. 5.2 observes that the two metrics
// can select different interaction orders).
//
// The energy source is the GPU's total-energy counter (millijoules since the
// driver loaded), read through NVML, which is loaded at run time so that the
// library neither links against it nor needs it unless this path is used.
// Only read-only NVML calls are made.  The counter advances in steps (every
// 100 ms on GB300; lj_energy_period measures it), so a configuration runs a
// batch of force evaluations several periods long, with the list rebuilds at
// the tuner's period (Verlet lists) or a rebin per evaluation (linked cells)
// as in the full-search cost of tune.cu.  The energy per evaluation is the
// average power between two counter updates inside the batch times the
// evaluation's CUDA-event time.
#include <dlfcn.h>
#include <nvml.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <limits>
#include <thread>
#include <utility>
#include <vector>

#include "ljgb_internal.cuh"

using namespace ljgb;

namespace {

struct Nvml {
  bool ok = false;
  nvmlReturn_t (*init)() = nullptr;
  nvmlReturn_t (*by_pci)(const char*, nvmlDevice_t*) = nullptr;
  nvmlReturn_t (*energy)(nvmlDevice_t, unsigned long long*) = nullptr;
};

Nvml load_nvml() {
  Nvml n;
  void* so = dlopen("libnvidia-ml.so.1", RTLD_NOW | RTLD_LOCAL);
  if (!so) so = dlopen("libnvidia-ml.so", RTLD_NOW | RTLD_LOCAL);
  if (!so) return n;
  n.init = reinterpret_cast<nvmlReturn_t (*)()>(dlsym(so, "nvmlInit_v2"));
  n.by_pci = reinterpret_cast<nvmlReturn_t (*)(const char*, nvmlDevice_t*)>(
      dlsym(so, "nvmlDeviceGetHandleByPciBusId_v2"));
  n.energy = reinterpret_cast<nvmlReturn_t (*)(nvmlDevice_t, unsigned long long*)>(
      dlsym(so, "nvmlDeviceGetTotalEnergyConsumption"));
  n.ok = n.init && n.by_pci && n.energy && n.init() == NVML_SUCCESS;
  return n;
}

const Nvml& nvml() {
  static const Nvml n = load_nvml();
  return n;
}

// NVML handle of a CUDA device (the current one for device < 0), matched by
// PCI bus id so that CUDA_VISIBLE_DEVICES renumbering does not matter.
lj_status device_handle(int32_t device, nvmlDevice_t* h) {
  const Nvml& n = nvml();
  if (!n.ok) return LJ_ERR_STATE;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return LJ_ERR_CUDA;
  char bus[32] = {0};
  if (cudaDeviceGetPCIBusId(bus, (int)sizeof(bus), dev) != cudaSuccess) return LJ_ERR_CUDA;
  return n.by_pci(bus, h) == NVML_SUCCESS ? LJ_OK : LJ_ERR_STATE;
}

lj_status read_mj(nvmlDevice_t h, double* mj) {
  unsigned long long v = 0;
  if (nvml().energy(h, &v) != NVML_SUCCESS) return LJ_ERR_STATE;
  *mj = (double)v;
  return LJ_OK;
}

lj_status efail(Ctx& c, lj_status s, const std::string& m) {
  c.err = m;
  return s;
}

}  // namespace

extern "C" {

lj_status lj_energy_read(int32_t device, double* mj) {
  if (!mj) return LJ_ERR_ARG;
  nvmlDevice_t h;
  lj_status st = device_handle(device, &h);
  if (st != LJ_OK) return st;
  return read_mj(h, mj);
}

lj_status lj_energy_period(int32_t device, double probe_ms, double* period_ms) {
  if (!period_ms || !(probe_ms > 0)) return LJ_ERR_ARG;
  nvmlDevice_t h;
  lj_status st = device_handle(device, &h);
  if (st != LJ_OK) return st;
  // Polls until kWanted updates have been seen or probe_ms has passed.  The
  // first update only marks a phase (the poll starts at an arbitrary point of
  // the counter's period), so k updates give k - 1 whole intervals.
  constexpr size_t kWanted = 5;
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  double last = 0.0, v = 0.0;
  if ((st = read_mj(h, &last)) != LJ_OK) return st;
  std::vector<double> ticks;
  while (ticks.size() < kWanted &&
         std::chrono::duration<double, std::milli>(clk::now() - t0).count() < probe_ms) {
    if ((st = read_mj(h, &v)) != LJ_OK) return st;
    if (v != last) {
      ticks.push_back(std::chrono::duration<double, std::milli>(clk::now() - t0).count());
      last = v;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  if (ticks.size() < 2) {
    *period_ms = std::numeric_limits<double>::quiet_NaN();
    return LJ_OK;
  }
  std::vector<double> d;
  for (size_t k = 1; k < ticks.size(); ++k) d.push_back(ticks[k] - ticks[k - 1]);
  std::sort(d.begin(), d.end());
  *period_ms = d[d.size() / 2];
  return LJ_OK;
}

lj_status lj_tune_energy(lj_ctx* ctx, double min_ms, lj_config* chosen, double* time_ms, double* energy_mj) {
  if (!ctx || !chosen || !(min_ms > 0)) return LJ_ERR_ARG;
  Ctx& c = ctx->c;
  if (!c.have_particles) return efail(c, LJ_ERR_STATE, "no particles loaded");
  nvmlDevice_t h;
  lj_status st = device_handle(-1, &h);
  if (st != LJ_OK) return efail(c, st, "the GPU energy counter (NVML) cannot be read");
  std::vector<lj_config> all(lj_config_list(nullptr, 0));
  lj_config_list(all.data(), (int32_t)all.size());
  const double nan = std::numeric_limits<double>::quiet_NaN();
  for (size_t k = 0; k < all.size(); ++k) {
    if (time_ms) time_ms[k] = nan;
    if (energy_mj) energy_mj[k] = nan;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return efail(c, LJ_ERR_CUDA, "cudaEventCreate");
  using clk = std::chrono::steady_clock;
  const auto origin = clk::now();
  auto now_ms = [&]() { return std::chrono::duration<double, std::milli>(clk::now() - origin).count(); };
  int best = -1;
  double best_mj = std::numeric_limits<double>::infinity();
  for (size_t k = 0; k < all.size() && st == LJ_OK; ++k) {
    const lj_config& g = all[k];
    if (!lj_config_valid(g) || (g.container == LJ_LC    ? c.nc_lc < 3
                                : g.container == LJ_LCS ? c.nc_lcs < 5
                                                        : g.container == LJ_VL && c.nc_vl < 3))
      continue;
    // warm-up (builds the lists or bins), then one timed evaluation sizes the batch
    if ((st = lj_compute_forces(ctx, g, nullptr, nullptr)) != LJ_OK) break;
    cudaEventRecord(e0, c.stream);
    if ((st = lj_compute_forces(ctx, g, nullptr, nullptr)) != LJ_OK) break;
    cudaEventRecord(e1, c.stream);
    cudaEventSynchronize(e1);
    float t1 = 0.f;
    cudaEventElapsedTime(&t1, e0, e1);
    const int per = std::max(1, c.rebuild_every);
    const int64_t evals = std::max<int64_t>(per, (int64_t)std::ceil(min_ms / std::max(1e-3, (double)t1)));
    // A host thread records every update of the energy counter (time, value)
    // while the batch runs; the average power comes from two updates inside
    // the busy window (after its first 15 %), so the idle time around the
    // batch and the counter's 100 ms steps at its ends do not enter.
    std::vector<std::pair<double, double>> ticks;
    std::atomic<bool> stop{false};
    std::thread poller([&]() {
      double last = -1.0, v = 0.0;
      while (!stop.load(std::memory_order_relaxed)) {
        if (read_mj(h, &v) == LJ_OK && v != last) {
          if (last >= 0.0) ticks.emplace_back(now_ms(), v);
          last = v;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
      }
    });
    cudaStreamSynchronize(c.stream);
    const double w0 = now_ms();
    cudaEventRecord(e0, c.stream);
    for (int64_t s = 0; s < evals && st == LJ_OK; ++s) {
      const bool cells = g.container == LJ_LC || g.container == LJ_LCS;
      if (cells) c.moved = true;  // a step's rebin is part of the cost
      if (!cells && s % per == 0 && s > 0) {
        c.moved_since_build = true;
        c.vl_valid = false;  // the list build of the rebuild period
        c.vcl_valid = false;
      }
      st = lj_compute_forces(ctx, g, nullptr, nullptr);
    }
    cudaEventRecord(e1, c.stream);
    cudaEventSynchronize(e1);
    const double w1 = now_ms();
    stop.store(true);
    poller.join();
    if (st != LJ_OK) break;
    float tw = 0.f;
    cudaEventElapsedTime(&tw, e0, e1);
    const double ms = (double)tw / (double)evals;
    const double lo = w0 + 0.15 * (w1 - w0);
    int a = -1, b = -1;
    for (int q = 0; q < (int)ticks.size(); ++q) {
      if (ticks[q].first < lo || ticks[q].first > w1) continue;
      if (a < 0) a = q;
      b = q;
    }
    double mj = nan;
    if (a >= 0 && b > a) {
      const double watts = (ticks[b].second - ticks[a].second) / (ticks[b].first - ticks[a].first);  // mJ/ms
      mj = watts * ms;
    }
    if (time_ms) time_ms[k] = ms;
    if (energy_mj) energy_mj[k] = mj;
    if (mj < best_mj) {
      best_mj = mj;
      best = (int)k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LJ_OK) return st;
  if (best < 0)
    return efail(c, LJ_ERR_STATE, "no configuration ran long enough for two energy-counter updates (raise min_ms)");
  *chosen = all[best];
  return LJ_OK;
}

}  // extern "C"

// api.cu -- host implementation of the C ABI declared in include/ljgb.h.
//
// The context keeps every particle array on the device in cell order and
// drives the kernels on the caller's stream.  Linked Cells (Sec. 2.1.1)
// rebin at every force evaluation after the particles moved; Verlet lists are
// rebuilt when stale (other half mode or layout, a particle moved more than
// skin/2, or the integrator's rebuild period).  The full-search tuner (Sec.
// 2.3.2) times every valid configuration with CUDA events and picks the
// fastest by the mean of its samples.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>

#include "ljgb_internal.cuh"

using namespace ljgb;

namespace {

lj_status fail(Ctx& c, lj_status s, const std::string& msg) {
  c.err = msg;
  return s;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail(c, e_ == cudaErrorMemoryAllocation ? LJ_ERR_OOM : LJ_ERR_CUDA,                 \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

#define CKS(expr)                  \
  do {                             \
    lj_status s_ = (expr);         \
    if (s_ != LJ_OK) return s_;    \
  } while (0)

// floor((r / u)^2) with u = L / 2^32, exactly: with r = mr 2^er and
// L = mL 2^eL (53-bit integer mantissas), (r/u)^2 = mr^2 2^k / mL^2 with
// k = 2 (er - eL) + 64.  Long division of mr^2 by mL^2 produces the integer
// part and then one quotient bit per power of two.
uint64_t exact_cut2(double L, double r) {
  int er = 0, eL = 0;
  const double fr = std::frexp(r, &er), fL = std::frexp(L, &eL);
  const unsigned __int128 mr = (unsigned __int128)(uint64_t)std::ldexp(fr, 53);
  const unsigned __int128 mL = (unsigned __int128)(uint64_t)std::ldexp(fL, 53);
  const unsigned __int128 num = mr * mr, den = mL * mL;
  int k = 2 * (er - eL) + 64;
  unsigned __int128 q = num / den, rem = num - q * den;
  while (k > 0) {
    rem <<= 1;
    q <<= 1;
    if (rem >= den) {
      rem -= den;
      q |= 1;
    }
    if (q >> 64) return std::numeric_limits<uint64_t>::max();
    --k;
  }
  if (k < 0) q = (-k >= 128) ? 0 : (q >> -k);
  return (uint64_t)q;
}

template <typename T>
cudaError_t dalloc(T*& p, size_t count) {
  if (p) cudaFree(p);
  p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(&p, count * sizeof(T));
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

bool order_is_valid(const lj_config& g) {
  if (g.container == LJ_LC) {
    switch (g.order) {
      case LJ_ORD_IPT_SMEM:
      case LJ_ORD_IPT_TMA:
      case LJ_ORD_ROT32:
        if (g.param != 0) return false;
        break;
      case LJ_ORD_KI:
        if (g.param != 2 && g.param != 4) return false;
        break;
      case LJ_ORD_JSPLIT:
        if (g.param != 32 && g.param != 16 && g.param != 8 && g.param != 4 && g.param != 2) return false;
        break;
      default:
        return false;
    }
    return g.newton3 == LJ_N3_OFF || g.newton3 == LJ_N3_ATOMIC || g.newton3 == LJ_N3_ATOMIC_BWD;
  }
  if (g.container == LJ_LCS) {
    if (g.order != LJ_ORD_JSPLIT || (g.param != 8 && g.param != 4 && g.param != 2)) return false;
    return g.newton3 == LJ_N3_OFF || g.newton3 == LJ_N3_ATOMIC || g.newton3 == LJ_N3_ATOMIC_BWD;
  }
  if (g.container == LJ_VCL) {
    if (g.order != LJ_ORD_CL_TILE && g.order != LJ_ORD_CL_JLANE) return false;
    if (g.param != 4 && g.param != 6 && g.param != 8) return false;
    return g.newton3 == LJ_N3_OFF || g.newton3 == LJ_N3_ATOMIC;
  }
  if (g.container == LJ_VL) {
    if (g.order == LJ_ORD_VL_IPT) return g.param == 0 && g.newton3 >= LJ_N3_OFF && g.newton3 <= LJ_N3_TWOPASS;
    if (g.order == LJ_ORD_JSPLIT) {
      if (g.param != 32 && g.param != 16 && g.param != 8 && g.param != 4 && g.param != 2) return false;
      return g.newton3 == LJ_N3_OFF || g.newton3 == LJ_N3_ATOMIC;
    }
  }
  return false;
}

std::vector<lj_config> all_configs() {
  std::vector<lj_config> v;
  const int n3s[2] = {LJ_N3_OFF, LJ_N3_ATOMIC};
  for (int n3 : n3s) {
    v.push_back({LJ_LC, LJ_ORD_IPT_SMEM, 0, n3});
    v.push_back({LJ_LC, LJ_ORD_IPT_TMA, 0, n3});
    v.push_back({LJ_LC, LJ_ORD_KI, 2, n3});
    v.push_back({LJ_LC, LJ_ORD_KI, 4, n3});
    for (int w : {32, 16, 8, 4, 2}) v.push_back({LJ_LC, LJ_ORD_JSPLIT, w, n3});
    v.push_back({LJ_LC, LJ_ORD_ROT32, 0, n3});
  }
  for (int n3 : n3s) {
    v.push_back({LJ_VL, LJ_ORD_VL_IPT, 0, n3});
    for (int w : {32, 16, 8, 4, 2}) v.push_back({LJ_VL, LJ_ORD_JSPLIT, w, n3});
  }
  v.push_back({LJ_VL, LJ_ORD_VL_IPT, 0, LJ_N3_TWOPASS});
  // the backward half shell last, so that the indices above stay as they were
  v.push_back({LJ_LC, LJ_ORD_IPT_SMEM, 0, LJ_N3_ATOMIC_BWD});
  v.push_back({LJ_LC, LJ_ORD_IPT_TMA, 0, LJ_N3_ATOMIC_BWD});
  v.push_back({LJ_LC, LJ_ORD_KI, 2, LJ_N3_ATOMIC_BWD});
  v.push_back({LJ_LC, LJ_ORD_KI, 4, LJ_N3_ATOMIC_BWD});
  for (int w : {32, 16, 8, 4, 2}) v.push_back({LJ_LC, LJ_ORD_JSPLIT, w, LJ_N3_ATOMIC_BWD});
  v.push_back({LJ_LC, LJ_ORD_ROT32, 0, LJ_N3_ATOMIC_BWD});
  // cluster lists: order x cluster size x Newton-3
  for (int n3 : n3s)
    for (int ord : {LJ_ORD_CL_TILE, LJ_ORD_CL_JLANE})
      for (int m : {4, 6, 8}) v.push_back({LJ_VCL, ord, m, n3});
  // linked cells of edge >= r_c / 2 (sub-cells), JSPLIT x Newton-3 (forward and backward half)
  for (int n3 : {LJ_N3_OFF, LJ_N3_ATOMIC, LJ_N3_ATOMIC_BWD})
    for (int w : {8, 4, 2}) v.push_back({LJ_LCS, LJ_ORD_JSPLIT, w, n3});
  return v;
}

lj_status sync_status(Ctx& c) {
  CK(cudaMemcpyAsync(c.host_status, c.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  return LJ_OK;
}

// Reads and clears the device status word; maps sticky errors to codes.
lj_status take_status(Ctx& c, uint32_t ignore = 0) {
  CKS(sync_status(c));
  const uint32_t st = *c.host_status & ~ignore;
  if (*c.host_status) CK(cudaMemsetAsync(c.status, 0, sizeof(uint32_t), c.stream));
  if (st & ST_NONFINITE) return fail(c, LJ_ERR_NONFINITE, "non-finite force, energy or virial");
  if (st & ST_TIMEOUT) return fail(c, LJ_ERR_TIMEOUT, "a bounded device wait timed out");
  if (st & ST_OOB) return fail(c, LJ_ERR_CUDA, "device index check failed");
  return LJ_OK;
}

lj_status need_particles(Ctx& c) {
  if (!c.have_particles) return fail(c, LJ_ERR_STATE, "no particles loaded");
  return LJ_OK;
}

lj_status alloc_particles(Ctx& c, int64_t n) {
  if (n == c.n && c.pos) return LJ_OK;
  CK(dalloc(c.pos, n));
  CK(dalloc(c.inv, n));
  CK(dalloc(c.pos_alt, n));
  CK(dalloc(c.vel, 3 * n));
  CK(dalloc(c.vel_alt, 3 * n));
  CK(dalloc(c.frc, 3 * n));
  CK(dalloc(c.frc_alt, 3 * n));
  CK(dalloc(c.cell_of, n));
  CK(dalloc(c.slot, n));
  CK(dalloc(c.key, 2 * n));
  CK(dalloc(c.x_build, 3 * n));
  CK(dalloc(c.nnbr, n));
  CK(dalloc(c.rev_cnt, n + 1));
  CK(dalloc(c.rev_start, n + 1));
  dfree(c.nbr);
  c.nbr = nullptr;
  c.vl_cap = 0;
  c.n = n;
  return LJ_OK;
}

void reset_state_flags(Ctx& c) {
  c.kick_pending = false;  // new particles: nothing of the last step is due
  c.skin_pending = false;
  c.binned_nc = 0;
  c.binned_for = -1;
  c.vl_valid = false;
  c.rev_valid = false;
  c.vl_half = -1;
  c.vcl_valid = false;
  c.vcl_half = -1;
  c.vcl_M = 0;
  c.forces_valid = false;
  c.tiles_gen = ~0ull;
  c.moved = true;
}

lj_status do_bin(Ctx& c, int container) {
  const int nc = container == LJ_LC ? c.nc_lc : container == LJ_LCS ? c.nc_lcs : c.nc_vl;
  const int need = container == LJ_LCS ? 5 : 3;
  if (nc < need)
    return fail(c, LJ_ERR_ARG, "box holds fewer than " + std::to_string(need) +
                                   " cells per axis for this container (edge " + std::to_string(c.L / need) + ")");
  c.P.nc = nc;
  CK(bin_cells(c, nc));
  c.launches += 7;  // cell ids, 3 scan passes, scatter, per-cell sort, permute
  c.binned_for = container;
  c.vl_valid = false;
  c.rev_valid = false;
  c.moved = false;
  return LJ_OK;
}

int initial_cap(const Ctx& c, int half) {
  const double rl = c.rc + c.skin;
  const double rho = (double)c.n / (c.L * c.L * c.L);
  double m = 4.18879020478639 * rl * rl * rl * rho * 1.25 + 16.0;
  if (half) m *= 0.5;
  int cap = (int)std::ceil(m / 8.0) * 8;
  return std::max(cap, 16);
}

// Bins on the r_c + skin cells and builds the lists (regrowing on overflow).
lj_status do_build_verlet(Ctx& c, int half, int colmajor, bool twopass) {
  c.skin_pending = false;  // the new lists make an earlier skin check moot
  CKS(do_bin(c, LJ_VL));
  if (c.vl_cap == 0 || !c.nbr) {
    c.vl_cap = initial_cap(c, half);
    CK(dalloc(c.nbr, (size_t)c.vl_cap * c.n));
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    CK(cudaMemsetAsync(c.maxlen, 0, sizeof(uint32_t), c.stream));
    CK(launch_build_verlet(c, half, colmajor, c.maxlen));
    c.launches += 1;
    uint32_t ml = 0;
    CK(cudaMemcpyAsync(c.host_status, c.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(&ml, c.maxlen, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (!(*c.host_status & ST_CAPACITY)) break;
    CK(cudaMemsetAsync(c.status, 0, sizeof(uint32_t), c.stream));
    c.vl_cap = (int)((ml + 15) / 8) * 8;
    CK(dalloc(c.nbr, (size_t)c.vl_cap * c.n));
    c.counters[4] += 1;
    if (attempt == 3) return fail(c, LJ_ERR_CAPACITY, "Verlet list capacity could not be grown");
  }
  if (*c.host_status & ST_SKIN) {  // a fresh list makes an earlier skin flag stale
    *c.host_status &= ~ST_SKIN;
    CK(cudaMemcpyAsync(c.status, c.host_status, sizeof(uint32_t), cudaMemcpyHostToDevice, c.stream));
  }
  c.vl_half = half;
  c.vl_colmajor = colmajor;
  // 16-bit copy of the lists (halves the list bytes) when every entry
  // j - i, wrapped modulo n, is guaranteed to fit: n <= 65536.  In larger
  // boxes the neighbours across the periodic faces in y and x lie up to a
  // full z-layer of cells away in cell order.
  c.vl_idx16 = false;
  if (!twopass && c.n <= 65536) {
    CK(launch_list_to16(c, c.maxlen));
    c.launches += 1;
    uint32_t ovf = 1;
    CK(cudaMemcpyAsync(&ovf, c.maxlen, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    c.vl_idx16 = ovf == 0;
  }
  c.vl_valid = true;
  c.rev_valid = false;
  c.steps_since_build = 0;
  c.counters[2] += 1;
  if (twopass) {
    const size_t ne = (size_t)c.vl_cap * c.n;
    if (c.rev_cap < ne) {
      CK(dalloc(c.rev_slot, ne));
      CK(dalloc(c.rev_key, ne));
      CK(dalloc(c.rev_key2, ne));
      c.rev_cap = ne;
    }
    const size_t bytes = 3 * ne * (c.prec == LJ_PREC_FP64 ? sizeof(double) : sizeof(float));
    if (c.twopass_bytes < bytes) {
      dfree(c.twopass);
      c.twopass = nullptr;
      CK(cudaMalloc(&c.twopass, bytes));
      c.twopass_bytes = bytes;
    }
    CK(launch_reverse_index(c));
    c.launches += 6;  // count, 3 scan passes, scatter, per-segment sort
    c.rev_valid = true;
  }
  return LJ_OK;
}

// Cluster order and cluster-pair lists for cluster size M (regrowing on
// overflow); the cluster order's binning snapshots the positions for the
// skin/2 rule.
lj_status do_build_vcl(Ctx& c, int M, int half) {
  c.skin_pending = false;
  if (c.n >= (int64_t(1) << 29)) return fail(c, LJ_ERR_ARG, "cluster lists hold at most 2^29 - 1 particles");
  int64_t ncl = 0;
  CK(vcl_bin(c, M, &ncl));
  c.launches += 13;  // tower ids, 3 scan passes, keys, per-cell sort, permute, cluster count + 3 scan passes, ...
  c.binned_for = LJ_VCL;
  c.vl_valid = false;
  c.rev_valid = false;
  c.moved = false;
  if (c.vcl_cap == 0) {
    // neighbour clusters: the boxes' Minkowski sum with the r_l ball, about
    // (a + 2 r_l)^3 for a cluster edge a = (M / rho)^(1/3), over M per cluster
    const double rho = (double)c.n / (c.L * c.L * c.L), rl = c.rc + c.skin;
    const double a = std::cbrt((double)M / rho);
    const double m = std::pow(a + 2.0 * rl, 3.0) * rho / M * (half ? 0.6 : 1.2) + 16.0;
    c.vcl_cap = (int)std::min<double>(std::ceil(m / 8.0) * 8.0, (double)std::max<int64_t>(ncl, 8) + 8.0);
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (c.vcl_nbr_cap < (size_t)c.vcl_cap * ncl || !c.vcl_nbr || !c.vcl_mask) {
      dfree(c.vcl_nbr);
      dfree(c.vcl_mask);
      c.vcl_nbr = nullptr;
      c.vcl_mask = nullptr;
      c.vcl_nbr_cap = 0;
      CK(cudaMalloc(&c.vcl_nbr, (size_t)c.vcl_cap * ncl * sizeof(uint32_t)));
      CK(cudaMalloc(&c.vcl_mask, (size_t)c.vcl_cap * ncl * sizeof(uint64_t)));
      c.vcl_nbr_cap = (size_t)c.vcl_cap * ncl;
    }
    if (c.vcl_nn_cap < (size_t)ncl || !c.vcl_nn) {
      dfree(c.vcl_nn);
      c.vcl_nn = nullptr;
      CK(dalloc(c.vcl_nn, (size_t)ncl));
      c.vcl_nn_cap = (size_t)ncl;
    }
    CK(cudaMemsetAsync(c.maxlen, 0, sizeof(uint32_t), c.stream));
    CK(launch_vcl_build(c, half, c.maxlen));
    c.launches += 1;
    uint32_t ml = 0;
    CK(cudaMemcpyAsync(c.host_status, c.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(&ml, c.maxlen, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (!(*c.host_status & ST_CAPACITY)) break;
    CK(cudaMemsetAsync(c.status, 0, sizeof(uint32_t), c.stream));
    c.vcl_cap = (int)((ml + 15) / 8) * 8;
    c.counters[4] += 1;
    if (attempt == 3) return fail(c, LJ_ERR_CAPACITY, "cluster list capacity could not be grown");
  }
  if (*c.host_status & ST_SKIN) {  // a fresh list makes an earlier skin flag stale
    *c.host_status &= ~ST_SKIN;
    CK(cudaMemcpyAsync(c.status, c.host_status, sizeof(uint32_t), cudaMemcpyHostToDevice, c.stream));
  }
  c.vcl_half = half;
  c.vcl_valid = true;
  c.steps_since_build = 0;
  c.counters[2] += 1;
  return LJ_OK;
}

// Lists of either list container exist for the current storage order (their
// build snapshot is what the skin/2 rule compares against).
bool lists_current(const Ctx& c) {
  return (c.vl_valid && c.binned_for == LJ_VL) || (c.vcl_valid && c.binned_for == LJ_VCL);
}

// The current lists are the ones cfg evaluates on.
bool lists_match(const Ctx& c, const lj_config& cfg) {
  const int half = cfg.newton3 != LJ_N3_OFF ? 1 : 0;
  if (cfg.container == LJ_VL)
    return c.vl_valid && c.binned_for == LJ_VL && c.vl_half == half &&
           c.vl_colmajor == (cfg.order == LJ_ORD_VL_IPT ? 1 : 0) && (cfg.newton3 != LJ_N3_TWOPASS || c.rev_valid);
  if (cfg.container == LJ_VCL)
    return c.vcl_valid && c.binned_for == LJ_VCL && c.vcl_half == half && c.vcl_M == cfg.param;
  return false;
}

// (Re)builds the lists of a list container for cfg.
lj_status build_lists(Ctx& c, const lj_config& cfg) {
  const int half = cfg.newton3 != LJ_N3_OFF ? 1 : 0;
  if (cfg.container == LJ_VCL) {
    CKS(do_build_vcl(c, cfg.param, half));
    c.P.nc = c.vcl_nt;
  } else {
    CKS(do_build_verlet(c, half, cfg.order == LJ_ORD_VL_IPT ? 1 : 0, cfg.newton3 == LJ_N3_TWOPASS));
    c.P.nc = c.nc_vl;
  }
  c.moved_since_build = false;
  return LJ_OK;
}

// Displacement check since the last build (skin/2 rule), synchronous.
lj_status list_is_fresh(Ctx& c, bool& fresh) {
  fresh = lists_current(c);
  if (!fresh || !c.moved_since_build) return LJ_OK;
  CK(launch_kick_drift(c, 0.0, 0.0, false, true) == cudaSuccess ? cudaSuccess : cudaErrorUnknown);
  uint32_t st = 0;
  CK(cudaMemcpyAsync(c.host_status, c.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  st = *c.host_status;
  if (st & ST_SKIN) {
    CK(cudaMemsetAsync(c.status, 0, sizeof(uint32_t), c.stream));
    fresh = false;
  }
  return LJ_OK;
}

// Makes the container structures current for cfg.
lj_status prepare(Ctx& c, const lj_config& cfg, bool allow_rebuild_schedule) {
  (void)allow_rebuild_schedule;
  if (cfg.container == LJ_LC || cfg.container == LJ_LCS) {
    if (c.binned_for != cfg.container || c.moved) CKS(do_bin(c, cfg.container));
    c.P.nc = cfg.container == LJ_LC ? c.nc_lc : c.nc_lcs;
    return LJ_OK;
  }
  bool fresh = false;
  CKS(list_is_fresh(c, fresh));
  if (fresh && lists_match(c, cfg)) {
    c.P.nc = cfg.container == LJ_VCL ? c.vcl_nt : c.nc_vl;
    return LJ_OK;
  }
  if (lists_current(c) && c.moved_since_build) c.counters[3] += 1;
  return build_lists(c, cfg);
}

// Kernels launched by the force dispatch (pair kernel + tile build when
// needed, or pair kernel + gather for the two-pass variant).
int force_launches(const Ctx& c, const lj_config& cfg, bool tiles_rebuilt) {
  if (cfg.container == LJ_VL) return cfg.newton3 == LJ_N3_TWOPASS ? 2 : 1;
  if (cfg.container == LJ_VCL) return 1;
  if (cfg.order == LJ_ORD_JSPLIT) return 1;
  return 1 + (tiles_rebuilt ? 5 : 0);
}

// Applies the pending closing half kick of the last integrated step (with the
// forces it was due with); every reader of velocities and every recomputation
// of the forces comes here first.
lj_status settle_kick(Ctx& c) {
  if (!c.kick_pending) return LJ_OK;
  CK(launch_kick_drift(c, c.kick_hdtm, 0.0, true, false));
  c.kick_pending = false;
  c.launches += 1;
  return LJ_OK;
}

lj_status run_force(Ctx& c, const lj_config& cfg, bool ev, bool acc_zeroed = false) {
  CKS(settle_kick(c));
  if (!acc_zeroed)  // energy, virial and pair counter
    CK(cudaMemsetAsync(c.ev, 0, 2 * sizeof(double) + sizeof(unsigned long long), c.stream));
  c.P.n = (int32_t)c.n;
  cudaError_t e;
  const bool f64 = c.prec == LJ_PREC_FP64;
  const uint64_t tiles_before = c.tiles_gen;
  const int tiles_T_before = c.tiles_T;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (c.timing) {
    while (c.ev_pool.size() < c.ev_used + 2) {
      cudaEvent_t ev_;
      CK(cudaEventCreate(&ev_));
      c.ev_pool.push_back(ev_);
    }
    t0 = c.ev_pool[c.ev_used];
    t1 = c.ev_pool[c.ev_used + 1];
    c.ev_used += 2;
  }
  // the tile list of the linked-cell orders is built outside the timed region
  if (cfg.container == LJ_LC && cfg.order != LJ_ORD_JSPLIT) {
    const int T = cfg.order == LJ_ORD_KI ? 32 * cfg.param : 32;
    CK(build_tiles(c, T));
  }
  if (t0) CK(cudaEventRecord(t0, c.stream));
  if (cfg.container == LJ_LC || cfg.container == LJ_LCS)
    e = f64 ? force_lc_f64(c, cfg, ev) : force_lc_f32(c, cfg, ev);
  else if (cfg.container == LJ_VCL)
    e = f64 ? force_vcl_f64(c, cfg, ev) : force_vcl_f32(c, cfg, ev);
  else
    e = f64 ? force_vl_f64(c, cfg, ev) : force_vl_f32(c, cfg, ev);
  if (t1) CK(cudaEventRecord(t1, c.stream));
  CK(e);
  c.launches += force_launches(c, cfg, c.tiles_gen != tiles_before || c.tiles_T != tiles_T_before);
  if (cfg.newton3 == LJ_N3_ATOMIC || cfg.newton3 == LJ_N3_ATOMIC_BWD) {  // unscaled atomic sums
    CK(f64 ? launch_scale_check(c) : launch_fold_scale(c));
    c.launches += 1;
  } else if (!(cfg.container == LJ_VL && cfg.newton3 == LJ_N3_OFF)) {  // fused into the VL N3-off store
    CK(launch_check_finite(c));
    c.launches += 1;
  }
  c.forces_valid = true;
  c.counters[0] += 1;
  return LJ_OK;
}

lj_status force_eval(Ctx& c, const lj_config& cfg, double* energy, double* virial) {
  if (!order_is_valid(cfg)) return fail(c, LJ_ERR_ARG, "invalid configuration");
  CKS(need_particles(c));
  const bool ev = energy || virial;
  if (c.skin_pending && lists_match(c, cfg)) {
    // positions came from lj_update_positions, whose kernel checked the skin:
    // evaluate on the current lists at once and read the flag meanwhile; if a
    // particle left its skin, rebuild and evaluate again
    c.skin_pending = false;
    c.P.nc = cfg.container == LJ_VCL ? c.vcl_nt : c.nc_vl;
    CKS(run_force(c, cfg, ev));
    CK(cudaEventSynchronize(c.drift_done));
    if (*reinterpret_cast<volatile uint32_t*>(c.skin_host)) {
      c.counters[3] += 1;
      CK(cudaMemsetAsync(c.status, 0, sizeof(uint32_t), c.stream));  // the speculative run's status is void
      CKS(build_lists(c, cfg));
      CKS(run_force(c, cfg, ev));
    }
  } else {
    c.skin_pending = false;
    CKS(prepare(c, cfg, false));
    CKS(run_force(c, cfg, ev));
  }
  c.last_cfg = cfg;
  if (ev) {
    CK(cudaMemcpyAsync(c.host_ev, c.ev, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(c.host_np, c.npairs, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.stream));
    CKS(take_status(c));
    const double side = cfg.newton3 == LJ_N3_OFF ? 0.5 : 1.0;
    if (energy) *energy = side * c.eps * 4.0 * c.host_ev[0];
    if (virial) *virial = side * c.eps * 24.0 * c.host_ev[1];
    c.counters[1] = (int64_t)((double)*c.host_np * side + 0.5);
    if (!std::isfinite(c.host_ev[0]) || !std::isfinite(c.host_ev[1]))
      return fail(c, LJ_ERR_NONFINITE, "non-finite energy or virial");
  } else {
    CK(cudaMemcpyAsync(c.host_np, c.npairs, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.stream));
    c.np_side = cfg.newton3 == LJ_N3_OFF ? 0.5 : 1.0;
    c.np_pending = true;
  }
  return LJ_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

lj_status lj_init_domain(lj_ctx** out, const double box[3], double cutoff, double skin, double eps, double sigma,
                         lj_precision prec, void* cuda_stream) {
  if (!out || !box) return LJ_ERR_ARG;
  *out = nullptr;
  const double L = box[0];
  if (!(L > 0) || box[1] != L || box[2] != L) return LJ_ERR_ARG;
  if (!(cutoff > 0) || !(skin >= 0) || !(cutoff + skin < 0.5 * L) || !(eps > 0) || !(sigma > 0)) return LJ_ERR_ARG;
  if (prec != LJ_PREC_FP64 && prec != LJ_PREC_FP32_ACC64) return LJ_ERR_ARG;
  lj_ctx* h = new (std::nothrow) lj_ctx();
  if (!h) return LJ_ERR_OOM;
  Ctx& c = h->c;
  c.L = L;
  c.rc = cutoff;
  c.skin = skin;
  c.eps = eps;
  c.sigma = sigma;
  c.prec = prec;
  c.stream = (cudaStream_t)cuda_stream;
  c.nc_lc = (int)std::floor(L / cutoff);
  c.nc_vl = (int)std::floor(L / (cutoff + skin));
  c.nc_lcs = (int)std::floor(L / (0.5 * cutoff));
  const double u = std::ldexp(L, -32);
  LJParams& P = c.P;
  P.Rc2 = exact_cut2(L, cutoff);
  c.Rl2 = exact_cut2(L, cutoff + skin);
  coarse_band(P.Rc2, &P.rc2p_lo, &P.rc2p_hi);
  coarse_band(c.Rl2, &c.rl2p_lo, &c.rl2p_hi);
  P.S = (sigma * sigma) / (u * u);
  P.S_hi = (float)P.S;
  P.S_lo = (float)(P.S - (double)P.S_hi);
  P.e24u = 24.0 * eps / u;
  P.e24 = 24.0 * eps;
  P.e4 = 4.0 * eps;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&c.ev, 3 * sizeof(double));
  if (e == cudaSuccess) c.npairs = reinterpret_cast<unsigned long long*>(c.ev + 2);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.drift_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc(&c.skin_host, sizeof(uint32_t), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&c.skin_dev, c.skin_host, 0);
  if (e == cudaSuccess) e = cudaMalloc(&c.status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c.maxlen, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c.tile_ctr, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c.feat_stats, 80 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost(&c.host_ev, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&c.host_np, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost(&c.host_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(c.status, 0, sizeof(uint32_t), c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e == cudaSuccess) {
    // L2 set-aside for persisting accesses (this process's context only): the
    // Verlet-list kernels keep the gathered positions resident with it.
    // LJGB_L2_PERSIST_MB=0 disables it.
    int dev = 0, maxwin = 0, maxpers = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxwin, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    cudaDeviceGetAttribute(&maxpers, cudaDevAttrMaxPersistingL2CacheSize, dev);
    const char* env = std::getenv("LJGB_L2_PERSIST_MB");
    size_t want = (size_t)(env ? std::atoi(env) : 48) << 20;
    want = std::min(want, (size_t)std::min(maxwin, maxpers));
    size_t cur = 0;
    if (want > 0 && cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) == cudaSuccess) {
      if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) want = 0;
      c.l2_window_bytes = want;
    }
    cudaGetLastError();
  }
  if (e != cudaSuccess) {
    lj_destroy(h);
    return e == cudaErrorMemoryAllocation ? LJ_ERR_OOM : LJ_ERR_CUDA;
  }
  *out = h;
  return LJ_OK;
}

static lj_status set_particles_impl(lj_ctx* h, int64_t n, const void* pos, bool fixed, const double* vel,
                                    double mass, int on_device) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (n < 1 || n > 0x7fffffffLL || !pos) return fail(c, LJ_ERR_ARG, "need 1 <= n < 2^31 and positions");
  if (!(mass > 0)) return fail(c, LJ_ERR_ARG, "mass must be positive");
  CKS(alloc_particles(c, n));
  const size_t pbytes = 3 * (size_t)n * (fixed ? sizeof(uint32_t) : sizeof(double));
  const void* dpos = pos;
  const double* dvel = vel;
  if (!on_device) {
    // host arrays go through a persistent device staging buffer (no per-call allocation)
    const size_t vbytes = vel ? 3 * (size_t)n * sizeof(double) : 0;
    const size_t need = ((pbytes + 255) / 256) * 256 + vbytes;
    if (c.stage_bytes < need) {
      dfree(c.stage);
      c.stage = nullptr;
      c.stage_bytes = 0;
      CK(cudaMalloc(&c.stage, need));
      c.stage_bytes = need;
    }
    char* st = (char*)c.stage;
    CK(cudaMemcpyAsync(st, pos, pbytes, cudaMemcpyHostToDevice, c.stream));
    dpos = st;
    if (vel) {
      double* dv = (double*)(st + ((pbytes + 255) / 256) * 256);
      CK(cudaMemcpyAsync(dv, vel, vbytes, cudaMemcpyHostToDevice, c.stream));
      dvel = dv;
    }
  }
  cudaError_t e = fixed ? launch_load_fp((const uint32_t*)dpos, n, dvel, c.pos, c.vel, c.stream)
                        : launch_quantize((const double*)dpos, n, c.L, dvel, c.pos, c.vel, c.stream);
  if (e == cudaSuccess) e = launch_iota(c.inv, n, c.stream);
  c.launches += 2;
  if (e == cudaSuccess) e = cudaMemsetAsync(c.frc, 0, 3 * (size_t)n * sizeof(double), c.stream);
  CK(e);
  c.mass = mass;
  c.P.n = (int32_t)n;
  c.have_particles = true;
  reset_state_flags(c);
  c.moved_since_build = true;
  return LJ_OK;
}

lj_status lj_set_particles(lj_ctx* h, int64_t n, const double* pos, const double* vel, double mass,
                           int on_device) {
  return set_particles_impl(h, n, pos, false, vel, mass, on_device);
}

lj_status lj_set_particles_fp(lj_ctx* h, int64_t n, const uint32_t* pos_fp, const double* vel, double mass,
                              int on_device) {
  return set_particles_impl(h, n, pos_fp, true, vel, mass, on_device);
}

// Device address of a host pointer the GPU can read and write directly (the
// caller's pinned memory, mapped in the unified address space), or nullptr.
static void* host_mapped(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

lj_status lj_update_positions(lj_ctx* h, const double* pos, int32_t on_device) {
  if (!h || !pos) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  CKS(settle_kick(c));  // the pending kick belongs to the state being replaced
  const size_t pbytes = 3 * (size_t)c.n * sizeof(double);
  const double* dpos = pos;
  const double* mapped = on_device ? nullptr : (const double*)host_mapped(pos);
  if (mapped) {
    dpos = mapped;  // read by the kernel across the host link, no staging copy
  } else if (!on_device) {
    if (c.stage_bytes < pbytes) {
      dfree(c.stage);
      c.stage = nullptr;
      c.stage_bytes = 0;
      CK(cudaMalloc(&c.stage, pbytes));
      c.stage_bytes = pbytes;
    }
    CK(cudaMemcpyAsync(c.stage, pos, pbytes, cudaMemcpyHostToDevice, c.stream));
    dpos = (const double*)c.stage;
  }
  // with current lists the update kernel also checks the skin (mapped flag)
  const bool check = lists_current(c);
  const double hs = 0.5 * c.skin * 4294967296.0 / c.L;
  const uint64_t d2max = hs * hs >= 1.8e19 ? ~0ull : (uint64_t)(hs * hs);
  if (check) *reinterpret_cast<volatile uint32_t*>(c.skin_host) = 0u;
  CK(launch_update_pos(c.pos, c.inv, dpos, c.n, c.L, check ? c.x_build : nullptr, d2max, c.skin_dev, c.stream,
                       c.status));
  if (check) CK(cudaEventRecord(c.drift_done, c.stream));
  c.skin_pending = check;
  c.launches += 1;
  // the cell order and the lists stay; the next evaluation rebins (linked
  // cells) or checks the skin and rebuilds only when needed (Verlet lists)
  c.moved = true;
  c.moved_since_build = true;
  c.forces_valid = false;
  return LJ_OK;
}

lj_status lj_bin_cells(lj_ctx* h, int32_t container) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  if (container != LJ_LC && container != LJ_VL && container != LJ_LCS)
    return fail(c, LJ_ERR_ARG, "unknown container");
  CKS(do_bin(c, container));
  CK(cudaGetLastError());
  return LJ_OK;
}

lj_status lj_build_verlet(lj_ctx* h, int32_t half_list) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  CKS(do_build_verlet(c, half_list ? 1 : 0, 0, false));
  c.moved_since_build = false;
  return LJ_OK;
}

lj_status lj_build_clusters(lj_ctx* h, int32_t M, int32_t half_list) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  if (M != 4 && M != 6 && M != 8) return fail(c, LJ_ERR_ARG, "cluster size must be 4, 6 or 8");
  CKS(settle_kick(c));
  CKS(do_build_vcl(c, M, half_list ? 1 : 0));
  c.moved_since_build = false;
  return LJ_OK;
}

lj_status lj_get_clusters(lj_ctx* h, int64_t* ncl, uint32_t* cl_start, int32_t* ntower) {
  if (!h || !ncl) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (c.binned_for != LJ_VCL || c.vcl_M == 0) return fail(c, LJ_ERR_STATE, "no cluster order is current");
  *ncl = c.vcl_ncl;
  if (ntower) *ntower = c.vcl_nt;
  if (cl_start) {
    CK(cudaMemcpyAsync(cl_start, c.cl_start, ((size_t)c.vcl_ncl + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                       c.stream));
    CK(cudaStreamSynchronize(c.stream));
  }
  return LJ_OK;
}

lj_status lj_get_cluster_lists(lj_ctx* h, int32_t* nbr, int32_t* nn, int32_t* cap_out) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (!c.vcl_valid || c.binned_for != LJ_VCL) return fail(c, LJ_ERR_STATE, "no cluster list built");
  const size_t ncl = (size_t)c.vcl_ncl, cap = (size_t)c.vcl_cap;
  if (cap_out) *cap_out = c.vcl_cap;
  if (nn) CK(cudaMemcpyAsync(nn, c.vcl_nn, ncl * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  if (nbr) {
    // packed entries (first slot << 3 | size - 1) back to cluster indices
    std::vector<uint32_t> packed(ncl * cap), cs(ncl + 1);
    std::vector<int32_t> len(ncl);
    CK(cudaMemcpyAsync(packed.data(), c.vcl_nbr, ncl * cap * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(cs.data(), c.cl_start, (ncl + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(len.data(), c.vcl_nn, ncl * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    for (size_t I = 0; I < ncl; ++I)
      for (size_t k = 0; k < cap; ++k) {
        if ((int32_t)k >= len[I]) {
          nbr[I * cap + k] = -1;
          continue;
        }
        const uint32_t b = packed[I * cap + k] >> 3;
        nbr[I * cap + k] = (int32_t)(std::lower_bound(cs.begin(), cs.end() - 1, b) - cs.begin());
      }
  }
  CK(cudaStreamSynchronize(c.stream));
  return LJ_OK;
}

lj_status lj_get_cluster_masks(lj_ctx* h, uint64_t* masks) {
  if (!h || !masks) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (!c.vcl_valid || c.binned_for != LJ_VCL) return fail(c, LJ_ERR_STATE, "no cluster list built");
  const size_t ncl = (size_t)c.vcl_ncl, cap = (size_t)c.vcl_cap;
  std::vector<int32_t> len(ncl);
  CK(cudaMemcpyAsync(masks, c.vcl_mask, ncl * cap * sizeof(uint64_t), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(len.data(), c.vcl_nn, ncl * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  for (size_t I = 0; I < ncl; ++I)
    for (size_t k = (size_t)std::max(0, std::min(len[I], (int32_t)cap)); k < cap; ++k) masks[I * cap + k] = 0;
  return LJ_OK;
}

int32_t lj_config_valid(lj_config cfg) { return order_is_valid(cfg) ? 1 : 0; }

int32_t lj_config_list(lj_config* out, int32_t cap) {
  const std::vector<lj_config> v = all_configs();
  if (out)
    for (int32_t k = 0; k < cap && k < (int32_t)v.size(); ++k) out[k] = v[k];
  return (int32_t)v.size();
}

lj_status lj_compute_forces(lj_ctx* h, lj_config cfg, double* energy_out, double* virial_out) {
  if (!h) return LJ_ERR_ARG;
  return force_eval(h->c, cfg, energy_out, virial_out);
}

lj_status lj_integrate_step(lj_ctx* h, double dt, int32_t nsteps, int32_t rebuild_every, lj_config cfg) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  if (!order_is_valid(cfg)) return fail(c, LJ_ERR_ARG, "invalid configuration");
  if (!(dt > 0) || nsteps < 0 || rebuild_every < 1) return fail(c, LJ_ERR_ARG, "need dt > 0, nsteps >= 0, rebuild_every >= 1");
  const double hdtm = 0.5 * dt / c.mass;
  const double dtu = dt * 4294967296.0 / c.L;
  const bool vl = cfg.container == LJ_VL || cfg.container == LJ_VCL;  // a list container
  c.skin_pending = false;  // the steps below check the skin themselves
  if (!c.forces_valid || memcmp(&c.last_cfg, &cfg, sizeof(cfg)) != 0) {
    CKS(prepare(c, cfg, false));
    CKS(run_force(c, cfg, false));
    c.last_cfg = cfg;
  }
  // Each step's closing half kick is left pending and fused into the next
  // step's first kick (the next call's, or lj_get_state / lj_kinetic_energy /
  // a force evaluation apply it on their own): one kernel per step less.
  for (int s = 0; s < nsteps; ++s) {
    const bool track = vl && lists_match(c, cfg);
    const bool speculate = track && c.steps_since_build + 1 < rebuild_every;
    if (speculate) *reinterpret_cast<volatile uint32_t*>(c.skin_host) = 0u;
    CK(launch_kick_drift(c, hdtm, dtu, false, track, speculate ? c.skin_dev : nullptr,
                         speculate ? c.ev : nullptr, c.kick_pending, c.kick_hdtm));
    c.kick_pending = false;
    c.launches += 1;
    c.moved = true;
    c.moved_since_build = true;
    if (vl) {
      c.steps_since_build += 1;
      const bool scheduled = c.steps_since_build >= rebuild_every || !lists_match(c, cfg);
      bool rebuild = scheduled;
      if (!scheduled) {
        // The drift writes its skin flag to mapped host memory and the force
        // kernel is queued at once on the current lists (the drift kernel also
        // cleared its accumulators), so the host's wait for the flag overlaps
        // GPU work.  If a particle left its skin the lists are rebuilt and the
        // forces computed again, replacing the speculative ones (and any
        // status they raised).
        CK(cudaEventRecord(c.drift_done, c.stream));
        c.P.nc = cfg.container == LJ_VCL ? c.vcl_nt : c.nc_vl;
        CKS(run_force(c, cfg, false, true));
        CK(cudaEventSynchronize(c.drift_done));
        if (*reinterpret_cast<volatile uint32_t*>(c.skin_host)) {
          CK(cudaMemsetAsync(c.status, 0, sizeof(uint32_t), c.stream));
          rebuild = true;
          c.counters[3] += 1;
        }
      }
      if (rebuild) {
        CKS(build_lists(c, cfg));
        CKS(run_force(c, cfg, false));
      }
    } else {
      CKS(do_bin(c, cfg.container));
      c.P.nc = cfg.container == LJ_LCS ? c.nc_lcs : c.nc_lc;
      CKS(run_force(c, cfg, false));
    }
    c.kick_pending = true;
    c.kick_hdtm = hdtm;
  }
  CK(cudaMemcpyAsync(c.host_np, c.npairs, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.stream));
  c.np_side = cfg.newton3 == LJ_N3_OFF ? 0.5 : 1.0;
  c.np_pending = true;
  return LJ_OK;
}

lj_status lj_get_forces(lj_ctx* h, double* dst, int32_t on_device) {
  if (!h || !dst) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  if (!c.forces_valid) return fail(c, LJ_ERR_STATE, "no forces computed");
  if (on_device) {
    CK(launch_from_slots(c.inv, c.frc, c.n, dst, c.stream, c.status));
    return LJ_OK;
  }
  if (double* mapped = (double*)host_mapped(dst)) {  // written by the kernel across the host link
    CK(launch_from_slots(c.inv, c.frc, c.n, mapped, c.stream, c.status));
    return take_status(c);
  }
  CK(launch_from_slots(c.inv, c.frc, c.n, c.frc_alt, c.stream, c.status));
  CK(cudaMemcpyAsync(dst, c.frc_alt, 3 * (size_t)c.n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  return take_status(c);
}

lj_status lj_get_state(lj_ctx* h, uint32_t* pos_fp, double* vel, int32_t on_device) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  CKS(settle_kick(c));
  const size_t n = (size_t)c.n;
  if (pos_fp) {
    if (on_device) {
      CK(launch_pos_to_original(c.pos, c.n, pos_fp, c.stream, c.status));
    } else {
      uint32_t* tmp = (uint32_t*)c.vel_alt;  // 3n doubles of scratch hold 3n uint32
      CK(launch_pos_to_original(c.pos, c.n, tmp, c.stream, c.status));
      CK(cudaMemcpyAsync(pos_fp, tmp, 3 * n * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
      CK(cudaStreamSynchronize(c.stream));
    }
  }
  if (vel) {
    if (on_device) {
      CK(launch_to_original(c.pos, c.vel, c.n, vel, c.stream, c.status));
    } else {
      CK(launch_to_original(c.pos, c.vel, c.n, c.vel_alt, c.stream, c.status));
      CK(cudaMemcpyAsync(vel, c.vel_alt, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      CK(cudaStreamSynchronize(c.stream));
    }
  }
  return LJ_OK;
}

lj_status lj_get_pairs(lj_ctx* h, int32_t container, int64_t* n_pairs, int32_t* ij) {
  if (!h || !n_pairs) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  std::vector<std::pair<int32_t, int32_t>> pairs;
  if (container == LJ_LC) {
    if (c.binned_for != LJ_LC || c.moved) CKS(do_bin(c, LJ_LC));
    unsigned long long* dcount = (unsigned long long*)c.feat_stats;
    CK(launch_lc_pairs(c, dcount, nullptr, 0));
    unsigned long long m = 0;
    CK(cudaMemcpyAsync(&m, dcount, sizeof(m), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    *n_pairs = (int64_t)m;
    if (!ij) return LJ_OK;
    int2* dout = nullptr;
    CK(cudaMalloc(&dout, std::max<size_t>(m, 1) * sizeof(int2)));
    cudaError_t e = launch_lc_pairs(c, dcount, dout, m);
    std::vector<int2> hp(m);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(hp.data(), dout, m * sizeof(int2), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    cudaFree(dout);
    CK(e);
    pairs.reserve(m);
    for (const int2& p : hp) pairs.emplace_back(p.x, p.y);
  } else if (container == LJ_VL) {
    if (!c.vl_valid || c.binned_for != LJ_VL) return fail(c, LJ_ERR_STATE, "no Verlet list built");
    const size_t n = (size_t)c.n, cap = (size_t)c.vl_cap;
    std::vector<int32_t> nbr(n * cap), nn(n);
    std::vector<uint4> pos(n);
    CK(cudaMemcpyAsync(nbr.data(), c.nbr, n * cap * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(nn.data(), c.nnbr, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(pos.data(), c.pos, n * sizeof(uint4), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    for (size_t i = 0; i < n; ++i)
      for (int k = 0; k < std::min(nn[i], (int32_t)cap); ++k) {
        const int32_t j = c.vl_colmajor ? nbr[(size_t)k * n + i] : nbr[i * cap + k];
        const int32_t a = (int32_t)pos[i].w, b = (int32_t)pos[j].w;
        if (c.vl_half || a < b) pairs.emplace_back(std::min(a, b), std::max(a, b));
      }
    *n_pairs = (int64_t)pairs.size();
    if (!ij) return LJ_OK;
  } else if (container == LJ_VCL) {
    if (!c.vcl_valid || c.binned_for != LJ_VCL) return fail(c, LJ_ERR_STATE, "no cluster list built");
    const size_t n = (size_t)c.n, ncl = (size_t)c.vcl_ncl, cap = (size_t)c.vcl_cap;
    std::vector<uint32_t> nbr(ncl * cap), cs(ncl + 1);
    std::vector<int32_t> nn(ncl);
    std::vector<uint4> pos(n);
    CK(cudaMemcpyAsync(nbr.data(), c.vcl_nbr, ncl * cap * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(nn.data(), c.vcl_nn, ncl * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(cs.data(), c.cl_start, (ncl + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(pos.data(), c.pos, n * sizeof(uint4), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    for (size_t I = 0; I < ncl; ++I)
      for (int k = 0; k < std::min(nn[I], (int32_t)cap); ++k) {
        const uint32_t e = nbr[I * cap + k], jb = e >> 3, je = jb + (e & 7u) + 1u;
        for (uint32_t a = cs[I]; a < cs[I + 1]; ++a)
          for (uint32_t b = jb; b < je; ++b) {
            const uint4 p = pos[a], q = pos[b];
            const int dx = (int)(q.x - p.x), dy = (int)(q.y - p.y), dz = (int)(q.z - p.z);
            const uint64_t R2 = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                                (uint64_t)((int64_t)dz * dz);
            if (R2 == 0 || R2 > c.Rl2) continue;
            const int32_t oa = (int32_t)p.w, ob = (int32_t)q.w;
            if (c.vcl_half || oa < ob) pairs.emplace_back(std::min(oa, ob), std::max(oa, ob));
          }
      }
    if (c.vcl_half) {  // the base cluster's own pairs appear twice in its self entry
      std::sort(pairs.begin(), pairs.end());
      pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
    }
    *n_pairs = (int64_t)pairs.size();
    if (!ij) return LJ_OK;
  } else {
    return fail(c, LJ_ERR_ARG, "unknown container");
  }
  std::sort(pairs.begin(), pairs.end());
  for (size_t k = 0; k < pairs.size(); ++k) {
    ij[2 * k] = pairs[k].first;
    ij[2 * k + 1] = pairs[k].second;
  }
  *n_pairs = (int64_t)pairs.size();
  return LJ_OK;
}

lj_status lj_get_cells(lj_ctx* h, uint32_t* perm, uint32_t* cell_start, int32_t* nc_out) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  if (!c.binned_nc) return fail(c, LJ_ERR_STATE, "not binned");
  const size_t n = (size_t)c.n;
  if (nc_out) *nc_out = c.binned_nc;
  if (perm) {
    std::vector<uint4> pos(n);
    CK(cudaMemcpyAsync(pos.data(), c.pos, n * sizeof(uint4), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    for (size_t k = 0; k < n; ++k) perm[k] = pos[k].w;
  }
  if (cell_start) {
    const size_t m = (size_t)c.binned_nc * c.binned_nc * c.binned_nc + 1;
    CK(cudaMemcpyAsync(cell_start, c.cell_start, m * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
  }
  return LJ_OK;
}

lj_status lj_get_verlet(lj_ctx* h, int32_t* nbr, int32_t* nnbr, int32_t* cap_out) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (!c.vl_valid) return fail(c, LJ_ERR_STATE, "no Verlet list built");
  const size_t n = (size_t)c.n, cap = (size_t)c.vl_cap;
  if (cap_out) *cap_out = c.vl_cap;
  if (nnbr) CK(cudaMemcpyAsync(nnbr, c.nnbr, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  if (nbr) {
    if (!c.vl_colmajor) {
      CK(cudaMemcpyAsync(nbr, c.nbr, n * cap * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    } else {
      std::vector<int32_t> t(n * cap);
      CK(cudaMemcpyAsync(t.data(), c.nbr, n * cap * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
      CK(cudaStreamSynchronize(c.stream));
      for (size_t i = 0; i < n; ++i)
        for (size_t k = 0; k < cap; ++k) nbr[i * cap + k] = t[k * n + i];
    }
  }
  CK(cudaStreamSynchronize(c.stream));
  return LJ_OK;
}

lj_status lj_get_counters(lj_ctx* h, int64_t* cnt5) {
  if (!h || !cnt5) return LJ_ERR_ARG;
  Ctx& c = h->c;
  if (c.np_pending) {
    CK(cudaStreamSynchronize(c.stream));
    c.counters[1] = (int64_t)((double)*c.host_np * c.np_side + 0.5);
    c.np_pending = false;
  }
  for (int k = 0; k < 5; ++k) cnt5[k] = c.counters[k];
  return LJ_OK;
}

lj_status lj_timing(lj_ctx* h, int32_t enable, double* force_ms, int64_t* launches, int64_t* total_launches) {
  if (!h) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CK(cudaStreamSynchronize(c.stream));
  if (force_ms || launches) {
    double tot = 0.0;
    for (size_t k = 0; k + 1 < c.ev_used; k += 2) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c.ev_pool[k], c.ev_pool[k + 1]));
      tot += ms;
    }
    if (force_ms) *force_ms = tot;
    if (launches) *launches = (int64_t)(c.ev_used / 2);
  }
  if (total_launches) *total_launches = c.launches;
  if (enable >= 0) {
    c.timing = enable != 0;
    c.ev_used = 0;
  }
  return LJ_OK;
}

lj_status lj_kinetic_energy(lj_ctx* h, double* ke) {
  if (!h || !ke) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  CKS(settle_kick(c));
  CK(launch_ke(c, c.ev));
  CK(cudaMemcpyAsync(c.host_ev, c.ev, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  *ke = 0.5 * c.mass * c.host_ev[0];
  return LJ_OK;
}

lj_status lj_features(lj_ctx* h, double* out) {
  if (!h || !out) return LJ_ERR_ARG;
  Ctx& c = h->c;
  CKS(need_particles(c));
  if (c.nc_lc < 1) return fail(c, LJ_ERR_ARG, "box smaller than the cutoff");
  CK(launch_feature_stats(c, c.feat_stats));
  unsigned long long st[74];
  CK(cudaMemcpyAsync(st, c.feat_stats, sizeof(st), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  c.binned_for = -1;  // the per-cell counter array was reused
  c.binned_nc = 0;
  c.moved = true;
  c.vl_valid = false;
  c.vcl_valid = false;
  const double n = (double)c.n, L = c.L;
  const double ncell = (double)c.nc_lc * c.nc_lc * c.nc_lc;
  const double s1 = (double)st[0], s2 = (double)st[1];
  const double mean = s1 / ncell;
  const double var = s2 / ncell - mean * mean;
  double bm = n / 64.0, bv = 0.0;
  for (int b = 0; b < 64; ++b) bv += ((double)st[10 + b] - bm) * ((double)st[10 + b] - bm);
  bv /= 64.0;
  const double edge = L / c.nc_lc, rl = c.rc + c.skin;
  out[0] = std::log(n / (L * L * L));
  out[1] = std::log(n);
  out[2] = mean;
  out[3] = std::sqrt(var > 0 ? var : 0.0);
  out[4] = (double)st[2] / ncell;
  for (int b = 0; b < 8; ++b) out[5 + b] = (double)st[2 + b] / ncell;
  out[13] = std::sqrt(bv) / bm;
  out[14] = c.rc / edge;
  out[15] = (s2 / n) * (4.0 / 3.0 * 3.14159265358979323846 * rl * rl * rl) / (edge * edge * edge);
  return LJ_OK;
}

const char* lj_last_error(const lj_ctx* h) {
  if (!h) return "null context";
  return h->c.err.c_str();
}

void lj_destroy(lj_ctx* h) {
  if (!h) return;
  Ctx& c = h->c;
  cudaStreamSynchronize(c.stream);
  void* dev[] = {c.pos, c.inv, c.pos_alt, c.vel, c.vel_alt, c.frc, c.frc_alt, c.cell_start, c.cnt, c.cell_of, c.slot,
                 c.key, c.scan_tmp, c.tiles, c.row_tiles, c.nbr, c.nnbr, c.x_build, c.maxlen, c.twopass,
                 c.rev_cnt, c.rev_start, c.rev_slot, c.rev_key, c.rev_key2, c.ev, c.status,
                 c.feat_stats, c.tile_ctr, c.stage, c.nbr16, c.tower_cl, c.cl_start, c.cl_lo, c.cl_hi, c.cl_z,
                 c.vcl_nbr, c.vcl_mask, c.vcl_nn, c.jacc};
  for (void* p : dev) dfree(p);
  if (c.host_ev) cudaFreeHost(c.host_ev);
  if (c.host_np) cudaFreeHost(c.host_np);
  if (c.host_status) cudaFreeHost(c.host_status);
  for (cudaEvent_t e : c.ev_pool) cudaEventDestroy(e);
  if (c.drift_done) cudaEventDestroy(c.drift_done);
  if (c.skin_host) cudaFreeHost(c.skin_host);
  delete h;
}

}  // extern "C"

// ljgb_internal.cuh -- shared definitions of the CUDA library (device helpers,
// parameter block, context).  Not part of the public ABI (include/ljgb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/ljgb.h"

namespace ljgb {

// ---------------------------------------------------------------------------
// Device status word bits (sticky until read by the host).
// ---------------------------------------------------------------------------
enum : uint32_t {
  ST_CAPACITY = 1u,   // a Verlet list overflowed
  ST_SKIN = 2u,       // a particle moved more than skin/2 since the list build
  ST_NONFINITE = 4u,  // NaN/Inf force
  ST_OOB = 8u,        // index out of range (defensive checks)
  ST_TIMEOUT = 16u,   // a bounded wait gave up
};

// Index checks of the LJGB_CHECKS build (build.py): an index read from data
// (a list entry, a segment bound, a cluster entry, a permutation slot) that
// falls outside its array sets ST_OOB, and the kernel skips or substitutes the
// access.  In the default build the test compiles away.
#ifdef LJGB_CHECKS
#define LJ_IDX_OK(cond, status) ((cond) ? true : (atomicOr((status), ST_OOB), false))
#else
#define LJ_IDX_OK(cond, status) true
#endif

// ---------------------------------------------------------------------------
// Parameter block, passed by value to the force kernels.
//
// Distances are handled in fixed-point units u = L / 2^32 (Sec. 2.1 cutoff
// rule read as an exact integer test).  The pair kernel works with
// r2u = R^2 in units u^2 and the dimensionless s2 = sigma^2 / r^2 = S / r2u,
// S = sigma^2 / u^2.  The force on i is F_i = -(24 eps / u) sum_j fac'_ij a_ij
// with fac' = s6 (2 s6 - 1) / r2u and a_ij the fixed-point difference, which
// equals the textbook -(24 eps / r^2) s6 (2 s6 - 1) dx.
// ---------------------------------------------------------------------------
struct LJParams {
  int32_t n;          // particles
  int32_t nc;         // cells per axis of the active container
  uint64_t Rc2;       // floor((r_c/u)^2)
  float rc2p_lo, rc2p_hi;  // coarse_r2 thresholds: certainly inside below lo, outside above hi
  float S_hi, S_lo;   // S = sigma^2/u^2 as an unevaluated float sum
  double S;           // S in FP64
  double e24u;        // 24 eps / u
  double e24;         // 24 eps
  double e4;          // 4 eps
};

// ---------------------------------------------------------------------------
// Small device helpers.
// ---------------------------------------------------------------------------

// Exact conversion of an FP32 value to FP64 done with integer operations on
// the IEEE-754 bit fields (sign kept, exponent rebiased 127 -> 1023, mantissa
// shifted into place).  GB300's FP64 pipe runs at ~1/80 of FP32 and hardware
// float->double conversions at under one per clock per SM, so the per-particle
// FP64 fold uses this instead.  FP32 subnormals (|x| < 1.2e-38) become signed
// zero; Inf and NaN are preserved.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t m = b & 0x7fffffu;
  const uint32_t sgn = b & 0x80000000u;
  uint32_t ex = (e == 255u) ? 0x7ffu : (e + 896u);
  uint32_t hi = sgn | (ex << 20) | (m >> 3);
  uint32_t lo = m << 29;
  hi = (e == 0u) ? sgn : hi;
  lo = (e == 0u) ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over aligned groups of W lanes (W a power of two <= 32); every lane of a
// group ends with the group's total.
template <int W>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exact membership test: 0 < R^2 <= Rc2 with R^2 in 64-bit integers.
__device__ __forceinline__ bool in_cut_exact(int a, int b, int c, uint64_t Rc2) {
  const uint64_t R2 = (uint64_t)((long long)a * a) + (uint64_t)((long long)b * b) +
                      (uint64_t)((long long)c * c);
  return (R2 != 0ull) & (R2 <= Rc2);
}

// 1/x for positive normal x: the hardware approximation refined by one
// Newton-Raphson step x0 (2 - x x0), written as two fused multiply-adds.
__device__ __forceinline__ float rcp_nr(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  const float e = fmaf(-x, y, 1.0f);
  return fmaf(y, e, y);
}

// ---------------------------------------------------------------------------
// The pair kernel (Algorithm 1's ForceKernel), FP32 and FP64 variants.
//
// Input: the fixed-point difference (a,b,c) = x_j - x_i (minimum image).
// Membership is the exact integer rule 0 < R^2 <= Rc2 with R^2 = a^2 + b^2 +
// c^2 in 64-bit integers.  The same exact R^2, rounded once to the pair
// precision, is the r^2 of the force: near the zero of F(r) (r = 2^(1/6)
// sigma) the force is ill-conditioned in r (|r F'/F| ~ 40), so r^2 carries one
// rounding instead of the several of a float sum of rounded squares (this
// cuts the worst FP32 force error relative to RMS|F| about 3x on dilute boxes).
// Output: fac' (0 outside the cutoff) and the converted differences; the
// caller accumulates fac' * (af,bf,cf).  With EV it also accumulates
// s6 (s6 - 1) (energy / 4 eps) and s6 (2 s6 - 1) (virial / 24 eps).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t r2_exact(int a, int b, int c) {
  return (uint64_t)((long long)a * a) + (uint64_t)((long long)b * b) + (uint64_t)((long long)c * c);
}

// Coarse r^2 for screening candidates without 64-bit arithmetic: each
// difference is shifted right by 9 (|a >> 9| < 2^22) and converted exactly by
// the magic-number method (the bits of 1.5 2^23 + v read as a float are
// 1.5 2^23 + v), giving A = floor(a / 512).  Since |(a/512)^2 - A^2| <= 2|A| + 1,
// the exact R^2 / 2^18 lies within 2 (|A|+|B|+|C|) + 3 + rounding of the
// returned sum; coarse_band() turns that into thresholds below which a pair is
// certainly inside and above which it is certainly outside.
__device__ __forceinline__ float coarse_r2(int a, int b, int c) {
  const float x = __int_as_float((a >> 9) + 0x4B400000) - 12582912.0f;
  const float y = __int_as_float((b >> 9) + 0x4B400000) - 12582912.0f;
  const float z = __int_as_float((c >> 9) + 0x4B400000) - 12582912.0f;
  return fmaf(z, z, fmaf(y, y, x * x));
}

// SELECT evaluates the pair unconditionally and selects the result, so the
// warp takes no branch (for list orders where most entries are inside and the
// branch is always taken by some lane); otherwise a pair outside the cutoff
// returns early, and SCREEN first rejects candidates by the coarse r^2.
template <bool EV, bool SCREEN = false, bool SELECT = false>
__device__ __forceinline__ float pair_f32(int a, int b, int c, const LJParams& P, float& af, float& bf,
                                          float& cf, float& eu, float& ew, int& cnt) {
  if (SCREEN) {
    const float r2p = coarse_r2(a, b, c);
    if (r2p > P.rc2p_hi) {  // certainly outside the cutoff
      af = bf = cf = 0.0f;
      return 0.0f;
    }
  }
  const uint64_t R2 = r2_exact(a, b, c);
  const bool in = R2 - 1ull < P.Rc2;  // 0 < R2 <= Rc2 (R2 = 0 wraps to the largest value)
  if (!SELECT && !in) {
    af = bf = cf = 0.0f;
    return 0.0f;
  }
  // R2 to FP32 from its two 32-bit words: 64-bit conversions run on the FP64
  // pipe (1/80 rate on GB300); the high word is below 2^24 whenever r_c < L/16,
  // so the sum carries a single rounding
  const float r2 = fmaf(__uint2float_rn((uint32_t)(R2 >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)R2));
  af = __int2float_rn(a);
  bf = __int2float_rn(b);
  cf = __int2float_rn(c);
  const float inv = rcp_nr(r2);
  const float s2 = fmaf(inv, P.S_hi, inv * P.S_lo);
  const float s6 = s2 * s2 * s2;
  const float t = fmaf(2.0f, s6, -1.0f);
  const bool keep = SELECT ? in : true;
  const float fac = keep ? s6 * t * inv : 0.0f;
  if (EV) {
    eu += keep ? fmaf(s6, s6, -s6) : 0.0f;
    ew += keep ? s6 * t : 0.0f;
  }
  cnt += keep ? 1 : 0;
  return fac;
}

template <bool EV>
__device__ __forceinline__ double pair_f64(int a, int b, int c, const LJParams& P, double& ad,
                                           double& bd, double& cd, double& eu, double& ew, int& cnt) {
  const uint64_t R2 = r2_exact(a, b, c);
  double fac = 0.0;
  ad = bd = cd = 0.0;
  if (R2 - 1ull < P.Rc2) {
    ad = (double)a;
    bd = (double)b;
    cd = (double)c;
    const double r2 = __ull2double_rn(R2);
    const double inv = 1.0 / r2;
    const double s2 = P.S * inv;
    const double s6 = s2 * s2 * s2;
    const double t = fma(2.0, s6, -1.0);
    fac = s6 * t * inv;
    if (EV) {
      eu += fma(s6, s6, -s6);
      ew += s6 * t;
    }
    cnt += 1;
  }
  return fac;
}

// Precision traits: the accumulator type of a pair chunk and its FP64 fold.
template <typename R>
struct Prec;
template <>
struct Prec<float> {
  template <bool EV, bool SCREEN = false, bool SELECT = false>
  __device__ __forceinline__ static float pair(int a, int b, int c, const LJParams& P, float& af, float& bf,
                                               float& cf, float& eu, float& ew, int& cnt) {
    return pair_f32<EV, SCREEN, SELECT>(a, b, c, P, af, bf, cf, eu, ew, cnt);
  }
  __device__ __forceinline__ static double to_d(float v) { return f2d_exact(v); }
};
template <>
struct Prec<double> {
  template <bool EV, bool SCREEN = false, bool SELECT = false>
  __device__ __forceinline__ static double pair(int a, int b, int c, const LJParams& P, double& ad,
                                                double& bd, double& cd, double& eu, double& ew, int& cnt) {
    return pair_f64<EV>(a, b, c, P, ad, bd, cd, eu, ew, cnt);
  }
  __device__ __forceinline__ static double to_d(double v) { return v; }
};

__device__ __forceinline__ int mimg(uint32_t xi, uint32_t xj) { return (int)(xj - xi); }

// Output block of a force evaluation: sorted-order FP64 forces plus global
// accumulators.
struct ForceOut {
  double* fx;
  double* fy;
  double* fz;
  double* ev;             // [0] = sum s6(s6-1), [1] = sum s6(2s6-1) (each pair counted per side visited)
  unsigned long long* npairs;  // pair evaluations counted (per side visited)
  uint32_t* status;
  float* jacc;  // FP32 Newton-3 evaluations: [n][4] partial sums (x, y, z, unused), else null
};

// One 16-byte vector reduction of (a, b, c, 0) into the float4 at p (16-byte
// aligned), performed in L2.
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(0.0f)
               : "memory");
}

// A Newton-3 contribution to particle k, unscaled (the factor 24 eps / u is
// applied once per particle afterwards): a j's share of one pair, or an i's
// sum over its pairs.  FP32 evaluations add it to k's FP32 partial sum with
// one vector reduction (the only record of k's force until launch_fold_scale
// writes the FP64 force from it); FP64 evaluations add it to the FP64 force
// with three atomics.
template <typename R>
__device__ __forceinline__ void n3_add(const ForceOut& out, int64_t k, R x, R y, R z) {
  if constexpr (sizeof(R) == 4) {
    if (x != 0.0f || y != 0.0f || z != 0.0f) red_add_v4(out.jacc + 4 * k, x, y, z);
  } else {
    if (x != 0.0) atomicAdd(out.fx + k, x);
    if (y != 0.0) atomicAdd(out.fy + k, y);
    if (z != 0.0) atomicAdd(out.fz + k, z);
  }
}

// Block-level reduction of the energy/virial partials and pair counts; one
// atomic per block.  Every thread of the block must call it.
template <typename R>
__device__ __forceinline__ void block_flush(double eu, double ew, int cnt, const ForceOut& out, bool EV) {
  __shared__ double s_e[2][32];
  __shared__ unsigned long long s_c[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  unsigned long long c = (unsigned long long)cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (EV) {
    eu = warp_sum_d(eu);
    ew = warp_sum_d(ew);
  }
  if (lane == 0) {
    s_c[wid] = c;
    if (EV) {
      s_e[0][wid] = eu;
      s_e[1][wid] = ew;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tc = 0;
    double te = 0.0, tw = 0.0;
    for (int w = 0; w < nw; ++w) {
      tc += s_c[w];
      if (EV) {
        te += s_e[0][w];
        tw += s_e[1][w];
      }
    }
    atomicAdd(out.npairs, tc);
    if (EV) {
      atomicAdd(&out.ev[0], te);
      atomicAdd(&out.ev[1], tw);
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side context.
// ---------------------------------------------------------------------------
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
};

struct Ctx {
  // geometry and model
  double L = 0, rc = 0, skin = 0, eps = 1, sigma = 1, mass = 1;
  int prec = LJ_PREC_FP32_ACC64;
  cudaStream_t stream = nullptr;
  int nc_lc = 0, nc_vl = 0, nc_lcs = 0;  // cells per axis: edge >= r_c, >= r_c + skin, >= r_c / 2
  LJParams P{};            // params with the cutoff r_c
  uint64_t Rl2 = 0;        // floor((r_l/u)^2)
  float rl2p_lo = 0, rl2p_hi = 0;  // coarse_r2 screening thresholds for r_l
  int64_t n = 0;
  bool have_particles = false;
  bool moved = true;             // particles moved since the last binning
  bool moved_since_build = true; // particles moved since the last list build
  lj_config last_cfg{-1, -1, -1, -1};
  double np_side = 1.0;          // pair-count scale of the pending evaluation
  bool np_pending = false;
  int rebuild_every = 10;        // list period assumed by the tuner's cost

  // particle state in the current (cell) order
  uint4* pos = nullptr;    // x, y, z fixed point, w = original index
  uint32_t* inv = nullptr; // original index -> current slot (inverse of pos[].w)
  uint4* pos_alt = nullptr;
  double* vel = nullptr;   // [3][n]
  double* vel_alt = nullptr;
  double* frc = nullptr;   // [3][n] forces of the last evaluation
  double* frc_alt = nullptr;
  float* jacc = nullptr;    // [n][4] FP32 Newton-3 partial sums
  size_t jacc_cap = 0;      // particles it holds
  bool forces_valid = false;
  // closing half kick of the last integrated step, not yet applied: velocities
  // are at the half step and v += kick_hdtm * F is due (see lj_integrate_step)
  bool kick_pending = false;
  double kick_hdtm = 0.0;
  // lj_update_positions checked the skin into skin_host (event drift_done):
  // the next list evaluation runs at once and rebuilds only if it was exceeded
  bool skin_pending = false;

  // binning
  int binned_nc = 0;       // n_c of the current cell order (0 = not binned)
  int binned_for = -1;     // container the order belongs to
  uint32_t* cell_start = nullptr;
  size_t cell_cap = 0;     // capacity of cell_start (entries)
  uint32_t* cnt = nullptr; // per-cell counters
  size_t cnt_cap = 0;
  uint32_t* cell_of = nullptr;
  uint32_t* slot = nullptr;
  unsigned long long* key = nullptr;  // (orig << 32) | source slot
  uint32_t* scan_tmp = nullptr;
  size_t scan_tmp_cap = 0;

  // tiles of the linked-cell kernels (per tile size)
  int tiles_T = 0;
  int tiles_for_nc = 0;
  uint64_t tiles_gen = 0;
  uint4* tiles = nullptr;  // (begin, end, row, cx_first | cx_last << 16)
  size_t tiles_cap = 0;
  int ntiles = 0;
  uint32_t* row_tiles = nullptr;  // per row (per cell for single-cell tiles) tile counts / offsets
  const uint32_t* ntiles_dev = nullptr;  // device count of the current tiles
  size_t row_tiles_cap = 0;
  uint64_t bin_gen = 0;    // increments at every binning
  uint32_t* tile_ctr = nullptr;  // device work counter of the tile kernels

  // Verlet lists
  int32_t* nbr = nullptr;  // row-major [n][cap] (JSPLIT) or column-major [cap][n] (IPT)
  int32_t* nnbr = nullptr;
  int16_t* nbr16 = nullptr;  // 16-bit copy of nbr (j - i wrapped modulo n) when every entry fits
  size_t nbr16_cap = 0;
  bool vl_idx16 = false;
  int vl_cap = 0;
  int vl_half = -1;        // half mode of the current list, -1 = none
  int vl_colmajor = 0;
  bool vl_valid = false;
  uint32_t* x_build = nullptr;  // [3][n] positions at the last build
  uint32_t* maxdisp = nullptr;  // device max |displacement| (units)
  int steps_since_build = 0;

  // Verlet cluster lists (k_vcl.cu): cluster order for cluster size vcl_M,
  // clusters [cl_start[c], cl_start[c+1]) with boxes cl_lo / cl_hi, and the
  // row-major cluster-pair lists [ncl][vcl_cap] of packed entries
  // (begin << 3) | (size - 1) with their member masks
  int vcl_M = 0;
  int vcl_nt = 0;               // towers per axis
  int64_t vcl_ncl = 0;
  int vcl_half = -1;
  bool vcl_valid = false;
  uint32_t* tower_cl = nullptr; // first cluster of each tower (nt^2 + 1)
  size_t tower_cl_cap = 0;
  uint32_t* cl_start = nullptr;
  size_t cl_start_cap = 0;
  uint4* cl_lo = nullptr;
  size_t cl_lo_cap = 0;
  uint4* cl_hi = nullptr;
  size_t cl_hi_cap = 0;
  uint32_t* cl_z = nullptr;     // zmin of every cluster, then zmax
  size_t cl_z_cap = 0;
  uint32_t* vcl_nbr = nullptr;
  uint64_t* vcl_mask = nullptr;  // [ncl][cap]: member pairs within r_l, bit a * M + b
  int32_t* vcl_nn = nullptr;
  int vcl_cap = 0;
  size_t vcl_nbr_cap = 0, vcl_nn_cap = 0;

  // two-pass Newton-3: per-entry slots R[3][cap*n] and the reverse index
  void* twopass = nullptr;
  size_t twopass_bytes = 0;
  uint32_t* rev_cnt = nullptr;    // n + 1
  uint32_t* rev_start = nullptr;  // n + 1
  uint32_t* rev_slot = nullptr;   // cap * n
  unsigned long long* rev_key = nullptr;   // cap * n
  unsigned long long* rev_key2 = nullptr;  // cap * n
  size_t rev_cap = 0;             // entries allocated in rev_slot / rev_key
  bool rev_valid = false;
  uint32_t* maxlen = nullptr;     // device: longest list of the last build, when it overflowed the capacity

  // accumulators and status
  double* ev = nullptr;    // 2 doubles, then the pair counter (one allocation, cleared by one memset)
  unsigned long long* npairs = nullptr;  // = (unsigned long long*)(ev + 2)
  uint32_t* status = nullptr;
  double* host_ev = nullptr;  // pinned mirror
  unsigned long long* host_np = nullptr;
  uint32_t* host_status = nullptr;
  // skin flag of the integrator's drift in mapped pinned memory (host view and
  // device alias): the drift kernel writes it, the host reads it after an event
  uint32_t* skin_host = nullptr;
  uint32_t* skin_dev = nullptr;
  cudaEvent_t drift_done = nullptr;

  // L2 persisting window over the positions for the Verlet-list kernels (0 = off)
  size_t l2_window_bytes = 0;

  // staging buffer for host uploads
  void* stage = nullptr;
  size_t stage_bytes = 0;

  // feature statistics scratch
  unsigned long long* feat_stats = nullptr;

  // learned tuner
  std::vector<float> mlp_params;
  int mlp_C = 0;
  std::vector<float> mlp_mean, mlp_std;
  std::vector<lj_config> mlp_cfgs;

  // counters
  int64_t counters[5] = {0, 0, 0, 0, 0};
  int64_t launches = 0;          // kernels launched by this context
  // optional CUDA-event timing of the force kernel (lj_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::string err;
};

// ---------------------------------------------------------------------------
// Kernel launchers (one translation unit each).
// ---------------------------------------------------------------------------
cudaError_t launch_quantize(const double* pos, int64_t n, double L, const double* vel, uint4* out_pos,
                            double* out_vel, cudaStream_t s);
cudaError_t launch_load_fp(const uint32_t* pos_fp, int64_t n, const double* vel, uint4* out_pos, double* out_vel,
                           cudaStream_t s);
cudaError_t bin_cells(Ctx& c, int nc);
cudaError_t build_tiles(Ctx& c, int T);
cudaError_t excl_scan_u32(Ctx& c, const uint32_t* in, uint32_t* out, int64_t n);
cudaError_t sort_segments(Ctx& c, const uint32_t* starts, int64_t nseg, unsigned long long* key,
                          unsigned long long* key2);
cudaError_t launch_build_verlet(Ctx& c, int half, int colmajor, uint32_t* maxlen);
cudaError_t launch_update_pos(uint4* pos, const uint32_t* inv, const double* x, int64_t n, double L,
                              const uint32_t* xb, uint64_t disp2_max, uint32_t* skin_flag, cudaStream_t s,
                              uint32_t* status);
cudaError_t launch_iota(uint32_t* inv, int64_t n, cudaStream_t s);
cudaError_t launch_from_slots(const uint32_t* inv, const double* src3, int64_t n, double* dst3, cudaStream_t s,
                              uint32_t* status);
cudaError_t launch_reverse_index(Ctx& c);
cudaError_t launch_list_to16(Ctx& c, uint32_t* overflow);
int vcl_ntower(int64_t n, int M);
cudaError_t vcl_bin(Ctx& c, int M, int64_t* ncl_out);
cudaError_t launch_vcl_build(Ctx& c, int half, uint32_t* maxlen);
cudaError_t force_vcl_f32(Ctx& c, const lj_config& cfg, bool ev);
cudaError_t force_vcl_f64(Ctx& c, const lj_config& cfg, bool ev);

// Thresholds for coarse_r2 (units of 2^18 u^2) around the integer threshold
// R2max: certainly inside below *lo, certainly outside above *hi.  The band
// half-width covers the flooring bound 2 (|A|+|B|+|C|) + 3 <= 2 sqrt(3 x) + 3
// at x = R2max / 2^18, plus float rounding of the sum, doubled for safety.
inline void coarse_band(uint64_t R2max, float* lo, float* hi) {
  const double x = (double)R2max / 262144.0;
  const double d = 2.0 * (2.0 * std::sqrt(3.0 * x) + 3.0) + 4.0e-7 * x + 8.0;
  *lo = (float)std::max(0.0, x - d) * (1.0f - 1e-6f);
  *hi = (float)(x + d) * (1.0f + 1e-6f);
}
cudaError_t launch_twopass_gather(Ctx& c);
cudaError_t force_lc_f32(Ctx& c, const lj_config& cfg, bool ev);
cudaError_t force_lc_f64(Ctx& c, const lj_config& cfg, bool ev);
cudaError_t force_vl_f32(Ctx& c, const lj_config& cfg, bool ev);
cudaError_t force_vl_f64(Ctx& c, const lj_config& cfg, bool ev);
cudaError_t launch_kick_drift(Ctx& c, double hdtm, double dtu, bool kick_only, bool track,
                              uint32_t* skin_flag = nullptr, double* zero_acc = nullptr, bool pre = false,
                              double hpre = 0.0);
cudaError_t launch_to_original(const uint4* pos, const double* src3, int64_t n, double* dst3, cudaStream_t s,
                               uint32_t* status);
cudaError_t launch_pos_to_original(const uint4* pos, int64_t n, uint32_t* dst3, cudaStream_t s,
                                   uint32_t* status);
cudaError_t launch_feature_stats(Ctx& c, unsigned long long* stats);
cudaError_t launch_ke(Ctx& c, double* out);
cudaError_t launch_check_finite(Ctx& c);
cudaError_t launch_scale_check(Ctx& c);
cudaError_t launch_fold_scale(Ctx& c);
cudaError_t n3_begin(Ctx& c, ForceOut& out, bool fp32);
cudaError_t launch_lc_pairs(Ctx& c, unsigned long long* count, int2* out, size_t cap);

}  // namespace ljgb

// The opaque handle of the C ABI.
struct lj_ctx {
  ljgb::Ctx c;
};

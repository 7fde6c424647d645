// k_integrate.cu -- velocity Verlet (Sec. 2.1: Verlet integration of Newton's
// equations), reorder back to the caller's particle order, tuner feature
// statistics, and small reductions.
#include "k_force_lc.cuh"

namespace ljgb {

static inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// v = fma(dt/2m, F, v) (one rounding); with drift, x += rne(v * dtu) mod 2^32,
// where rne(v * dtu) is the exact product rounded once to the nearest integer:
// fma(v, dtu, 1.5 * 2^52) lies in [2^52, 2^53) where the spacing is 1, and its
// low 32 bits are the displacement modulo 2^32.  With track, particles whose
// displacement since the last list build exceeds skin/2 set ST_SKIN (and the
// mapped host word skin_flag, when given).  zero_acc, when given, is cleared
// (two doubles and a counter) for the force evaluation queued next.  With pre,
// the previous step's closing half kick (hpre) is applied first, as its own
// rounded FMA, so that fusing the two kicks leaves the arithmetic unchanged.
__global__ void k_kick_drift(uint4* __restrict__ pos, double* __restrict__ vel, const double* __restrict__ frc,
                             int64_t n, double hdtm, double dtu, int drift, const uint32_t* __restrict__ xb,
                             uint64_t disp2_max, uint32_t* __restrict__ status, uint32_t* skin_flag,
                             double* __restrict__ zero_acc, int pre, double hpre) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (zero_acc && i == 0) {  // energy, virial and pair counter of the force evaluation that follows
    zero_acc[0] = 0.0;
    zero_acc[1] = 0.0;
    reinterpret_cast<unsigned long long*>(zero_acc)[2] = 0ull;
  }
  if (i >= n) return;
  const double f0 = frc[i], f1 = frc[n + i], f2 = frc[2 * n + i];
  double v0 = vel[i], v1 = vel[n + i], v2 = vel[2 * n + i];
  if (pre) {  // the previous step's closing half kick, then this step's first
    v0 = __fma_rn(hpre, f0, v0);
    v1 = __fma_rn(hpre, f1, v1);
    v2 = __fma_rn(hpre, f2, v2);
  }
  v0 = __fma_rn(hdtm, f0, v0);
  v1 = __fma_rn(hdtm, f1, v1);
  v2 = __fma_rn(hdtm, f2, v2);
  vel[i] = v0;
  vel[n + i] = v1;
  vel[2 * n + i] = v2;
  if (!drift) return;
  const double M = 6755399441055744.0;  // 1.5 * 2^52
  uint4 p = pos[i];
  p.x += (uint32_t)__double2loint(__fma_rn(v0, dtu, M));
  p.y += (uint32_t)__double2loint(__fma_rn(v1, dtu, M));
  p.z += (uint32_t)__double2loint(__fma_rn(v2, dtu, M));
  pos[i] = p;
  if (xb) {
    const int a = (int)(p.x - xb[i]), b = (int)(p.y - xb[n + i]), c = (int)(p.z - xb[2 * n + i]);
    const uint64_t d2 = (uint64_t)((long long)a * a) + (uint64_t)((long long)b * b) + (uint64_t)((long long)c * c);
    if (d2 > disp2_max) {
      atomicOr(status, ST_SKIN);
      if (skin_flag) *skin_flag = 1u;  // mapped host word: any writer sets it
    }
  }
}

cudaError_t launch_kick_drift(Ctx& c, double hdtm, double dtu, bool kick_only, bool track, uint32_t* skin_flag,
                              double* zero_acc, bool pre, double hpre) {
  const double half_skin_u = 0.5 * c.skin * 4294967296.0 / c.L;
  const double d2 = half_skin_u * half_skin_u;
  const uint64_t d2max = d2 >= 1.8e19 ? ~0ull : (uint64_t)d2;
  k_kick_drift<<<nb(c.n, 256), 256, 0, c.stream>>>(c.pos, c.vel, c.frc, c.n, hdtm, dtu, kick_only ? 0 : 1,
                                                   track ? c.x_build : nullptr, d2max, c.status, skin_flag,
                                                   zero_acc, pre ? 1 : 0, hpre);
  return cudaGetLastError();
}

// dst[a][orig(s)] = src[a][s]
__global__ void k_to_original(const uint4* __restrict__ pos, const double* __restrict__ src, int64_t n,
                              double* __restrict__ dst, uint32_t* status) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t o = pos[s].w;
  if (!LJ_IDX_OK(o < (uint64_t)n, status)) return;
  dst[o] = src[s];
  dst[n + o] = src[n + s];
  dst[2 * n + o] = src[2 * n + s];
}

__global__ void k_pos_to_original(const uint4* __restrict__ pos, int64_t n, uint32_t* __restrict__ dst,
                                  uint32_t* status) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint4 p = pos[s];
  if (!LJ_IDX_OK(p.w < (uint64_t)n, status)) return;
  dst[p.w] = p.x;
  dst[n + p.w] = p.y;
  dst[2 * n + p.w] = p.z;
}

// dst[a][o] = src[a][inv[o]]: writes in the caller's order (coalesced), so dst
// may also be the caller's pinned host memory written across the host link.
__global__ void k_from_slots(const uint32_t* __restrict__ inv, const double* __restrict__ src, int64_t n,
                             double* __restrict__ dst, uint32_t* status) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const uint32_t s = inv[o];
  if (!LJ_IDX_OK(s < (uint64_t)n, status)) return;
  dst[o] = src[s];
  dst[n + o] = src[n + s];
  dst[2 * n + o] = src[2 * n + s];
}

cudaError_t launch_from_slots(const uint32_t* inv, const double* src3, int64_t n, double* dst3, cudaStream_t s,
                              uint32_t* status) {
  k_from_slots<<<nb(n, 256), 256, 0, s>>>(inv, src3, n, dst3, status);
  return cudaGetLastError();
}

cudaError_t launch_to_original(const uint4* pos, const double* src3, int64_t n, double* dst3, cudaStream_t s,
                               uint32_t* status) {
  k_to_original<<<nb(n, 256), 256, 0, s>>>(pos, src3, n, dst3, status);
  return cudaGetLastError();
}

cudaError_t launch_pos_to_original(const uint4* pos, int64_t n, uint32_t* dst3, cudaStream_t s,
                                   uint32_t* status) {
  k_pos_to_original<<<nb(n, 256), 256, 0, s>>>(pos, n, dst3, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tuner feature statistics (exact integers): per-cell counts on the r_c cells,
// then sum occ, sum occ^2, the 8-bin occupancy histogram and the 64
// coarse-block counts (top two bits of each coordinate).
// stats layout: [0] sum occ, [1] sum occ^2, [2..9] histogram, [10..73] blocks.
// ---------------------------------------------------------------------------
__global__ void k_feat_count(const uint4* __restrict__ pos, int64_t n, uint32_t nc, uint32_t* __restrict__ occ,
                             unsigned long long* __restrict__ stats) {
  __shared__ unsigned int s_blk[64];
  if (threadIdx.x < 64) s_blk[threadIdx.x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint4 p = pos[i];
    const uint32_t c = (cx_of(p.z, nc) * nc + cx_of(p.y, nc)) * nc + cx_of(p.x, nc);
    atomicAdd(&occ[c], 1u);
    atomicAdd(&s_blk[((p.z >> 30) * 4 + (p.y >> 30)) * 4 + (p.x >> 30)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 64 && s_blk[threadIdx.x]) atomicAdd(&stats[10 + threadIdx.x], (unsigned long long)s_blk[threadIdx.x]);
}

__global__ void k_feat_cells(const uint32_t* __restrict__ occ, int64_t ncell, unsigned long long* __restrict__ stats) {
  __shared__ unsigned long long s_acc[10];
  if (threadIdx.x < 10) s_acc[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long s1 = 0, s2 = 0;
  unsigned int h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long o = occ[c];
    s1 += o;
    s2 += o * o;
    const int b = o == 0 ? 0 : o <= 2 ? 1 : o <= 4 ? 2 : o <= 8 ? 3 : o <= 16 ? 4 : o <= 32 ? 5 : o <= 64 ? 6 : 7;
    h[b] += 1;
  }
  atomicAdd(&s_acc[0], s1);
  atomicAdd(&s_acc[1], s2);
#pragma unroll
  for (int b = 0; b < 8; ++b)
    if (h[b]) atomicAdd(&s_acc[2 + b], (unsigned long long)h[b]);
  __syncthreads();
  if (threadIdx.x < 10 && s_acc[threadIdx.x]) atomicAdd(&stats[threadIdx.x], s_acc[threadIdx.x]);
}

cudaError_t launch_feature_stats(Ctx& c, unsigned long long* stats) {
  const int nc = c.nc_lc;
  const int64_t ncell = (int64_t)nc * nc * nc;
  cudaError_t e;
  if ((e = cudaMemsetAsync(stats, 0, 74 * sizeof(unsigned long long), c.stream)) != cudaSuccess) return e;
  // the per-cell counter array of the binning is free between binnings
  if (c.cnt_cap < (size_t)ncell + 1) {
    if (c.cnt) cudaFree(c.cnt);
    c.cnt = nullptr;
    c.cnt_cap = 0;
    if ((e = cudaMalloc(&c.cnt, ((size_t)ncell + 1) * sizeof(uint32_t))) != cudaSuccess) return e;
    c.cnt_cap = (size_t)ncell + 1;
  }
  if ((e = cudaMemsetAsync(c.cnt, 0, (size_t)ncell * sizeof(uint32_t), c.stream)) != cudaSuccess) return e;
  k_feat_count<<<nb(c.n, 256), 256, 0, c.stream>>>(c.pos, c.n, (uint32_t)nc, c.cnt, stats);
  k_feat_cells<<<(unsigned)std::min<int64_t>(nb(ncell, 256), 1024), 256, 0, c.stream>>>(c.cnt, ncell, stats);
  return cudaGetLastError();
}

// 1/2 m sum v^2 (FP64)
__global__ void k_ke(const double* __restrict__ vel, int64_t n, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
    s += vel[i] * vel[i];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

cudaError_t launch_ke(Ctx& c, double* out) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), c.stream);
  if (e != cudaSuccess) return e;
  k_ke<<<std::min<unsigned>(nb(3 * c.n, 256), 1024), 256, 0, c.stream>>>(c.vel, c.n, out);
  return cudaGetLastError();
}

__global__ void k_check_finite(const double* __restrict__ f, int64_t m, uint32_t* __restrict__ status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(f[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

cudaError_t launch_check_finite(Ctx& c) {
  k_check_finite<<<nb(3 * c.n, 256), 256, 0, c.stream>>>(c.frc, 3 * c.n, c.status);
  return cudaGetLastError();
}

// f *= scale, then the finiteness check: the Newton-3 kernels leave unscaled
// FP64 sums (one multiply per particle here instead of one per contribution).
__global__ void k_scale_check(double* __restrict__ f, int64_t m, double scale, uint32_t* __restrict__ status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = f[i] * scale;
    f[i] = v;
    bad |= !isfinite(v);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// f = scale * the FP32 partial sums, then the finiteness check: the fold of
// an FP32 Newton-3 evaluation, whose kernels add both sides of every pair to
// the partial sums.
__global__ void k_fold_scale(double* __restrict__ f, const float4* __restrict__ jacc, int64_t n, double scale,
                             uint32_t* __restrict__ status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = jacc[i];
    const double v0 = (double)a.x * scale, v1 = (double)a.y * scale, v2 = (double)a.z * scale;
    f[i] = v0;
    f[n + i] = v1;
    f[2 * n + i] = v2;
    bad |= !isfinite(v0) || !isfinite(v1) || !isfinite(v2);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

cudaError_t launch_fold_scale(Ctx& c) {
  k_fold_scale<<<nb(c.n, 256), 256, 0, c.stream>>>(c.frc, (const float4*)c.jacc, c.n, c.P.e24u, c.status);
  return cudaGetLastError();
}

// Start of a Newton-3 evaluation: the sums it accumulates into are zeroed,
// the FP64 forces for FP64 pair arithmetic, else the FP32 partial sums (grown
// to n particles when needed, and named in out).
cudaError_t n3_begin(Ctx& c, ForceOut& out, bool fp32) {
  cudaError_t e;
  if (!fp32) return cudaMemsetAsync(c.frc, 0, 3 * (size_t)c.n * sizeof(double), c.stream);
  if (c.jacc_cap < (size_t)c.n) {
    if (c.jacc) cudaFree(c.jacc);
    c.jacc = nullptr;
    c.jacc_cap = 0;
    if ((e = cudaMalloc(&c.jacc, 4 * sizeof(float) * (size_t)c.n)) != cudaSuccess) return e;
    c.jacc_cap = (size_t)c.n;
  }
  out.jacc = c.jacc;
  return cudaMemsetAsync(c.jacc, 0, 4 * sizeof(float) * (size_t)c.n, c.stream);
}

cudaError_t launch_scale_check(Ctx& c) {
  k_scale_check<<<nb(3 * c.n, 256), 256, 0, c.stream>>>(c.frc, 3 * c.n, c.P.e24u, c.status);
  return cudaGetLastError();
}

// Pair set of the linked-cell scan: every (i, j) with orig(i) < orig(j),
// 0 < R^2 <= Rc2, j in the 27 cells around i.  With out == nullptr only counts.
__global__ void k_lc_pairs(const uint4* __restrict__ pos, const uint32_t* __restrict__ cs, int nc, int64_t n,
                           uint64_t Rc2, unsigned long long* __restrict__ count, int2* __restrict__ out,
                           unsigned long long cap, uint32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 pi = pos[i];
  const int cx = (int)cx_of(pi.x, nc), cy = (int)cx_of(pi.y, nc), cz = (int)cx_of(pi.z, nc);
  Seg segs[18];
  const int ns = make_segments<false>(cs, nc, cz * nc + cy, cx, cx, 0u, 0u, segs);
  check_segs(segs, ns, (uint32_t)n, status);
  for (int s = 0; s < ns; ++s)
    for (uint32_t j = segs[s].b; j < segs[s].e; ++j) {
      const uint4 pj = pos[j];
      if (pj.w <= pi.w) continue;
      if (!in_cut_exact(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), Rc2)) continue;
      const unsigned long long k = atomicAdd(count, 1ull);
      if (out && k < cap) out[k] = make_int2((int)pi.w, (int)pj.w);
    }
}

cudaError_t launch_lc_pairs(Ctx& c, unsigned long long* count, int2* out, size_t cap) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), c.stream);
  if (e != cudaSuccess) return e;
  k_lc_pairs<<<nb(c.n, 128), 128, 0, c.stream>>>(c.pos, c.cell_start, c.binned_nc, c.n, c.P.Rc2, count, out,
                                                (unsigned long long)cap, c.status);
  return cudaGetLastError();
}

}  // namespace ljgb

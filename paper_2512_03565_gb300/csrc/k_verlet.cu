// k_verlet.cu -- Verlet-list construction (Sec. 2.1.1: neighbour lists of the
// particles within cutoff + skin, built with the help of the linked-cell
// structure and rebuilt every few steps).
//
// The tile scan (bv_tile, k_build.cuh) is shared with the batched ensemble.
// Lists longer than the capacity keep counting, set ST_CAPACITY and report
// the longest list so the host can regrow and rebuild.
#include "k_build.cuh"
#include "k_force_lc.cuh"

namespace ljgb {

// One tile per warp, taken from a global counter; the scan is bv_tile.
template <bool HALF, bool COLMAJOR>
__global__ void __launch_bounds__(256) k_build_verlet(const uint4* __restrict__ pos, const uint32_t* __restrict__ cs,
                                                      int nc, int n, uint64_t Rl2, int cap,
                                                      const uint4* __restrict__ tiles,
                                                      const uint32_t* __restrict__ ntiles_ptr,
                                                      uint32_t* __restrict__ tile_ctr, int32_t* __restrict__ nbr,
                                                      int32_t* __restrict__ nnbr, uint32_t* __restrict__ xb,
                                                      uint32_t* __restrict__ maxlen, uint32_t* __restrict__ status,
                                                      float rl2p_lo, float rl2p_hi) {
  __shared__ uint4 s_i[8][32];
  __shared__ float4 s_c[8][32];  // coarse coordinates of the tile's particles
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t ntiles = *ntiles_ptr;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(tile_ctr, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntiles) break;
    const uint4 tile = tiles[t];
    const int cx = (int)(tile.w & 0xffffu);  // single-cell tiles: cx_first == cx_last
    const int ni = (int)(tile.y - tile.x);
    if (lane < ni) {
      const uint4 p = pos[tile.x + lane];
      s_i[wib][lane] = p;
      s_c[wib][lane] = make_float4(coarse_coord(p.x), coarse_coord(p.y), coarse_coord(p.z), 0.0f);
      xb[tile.x + lane] = p.x;
      xb[(int64_t)n + tile.x + lane] = p.y;
      xb[2 * (int64_t)n + tile.x + lane] = p.z;
    }
    BSeg segs[18];
    const int ns = builder_segments(cs, nc, (int)tile.z, cx, segs);
#ifdef LJGB_CHECKS
    for (int s = 0; s < ns; ++s)
      if (!LJ_IDX_OK(segs[s].b <= segs[s].e && segs[s].e <= (uint32_t)n, status)) segs[s].b = segs[s].e = 0u;
#endif
    const uint32_t my_cnt = bv_tile<HALF, COLMAJOR>(pos, segs, ns, tile.x, ni, s_i[wib], s_c[wib], n, cap, Rl2,
                                                     rl2p_lo, rl2p_hi, nbr);
    if (lane < ni) {
      nnbr[tile.x + lane] = (int32_t)my_cnt;
      if (my_cnt > (uint32_t)cap) {  // only an overflow needs the longest length (for the regrowth)
        atomicOr(status, ST_CAPACITY);
        atomicMax(maxlen, my_cnt);
      }
    }
    __syncwarp();
  }
}

// Reverse index of a half list for the two-pass Newton-3 reduction:
// rstart[j]..rstart[j+1] holds the entry ids e = k * n + i (column-major
// slots) of all entries with nbr[e] = j, in ascending e.
__global__ void k_rev_count(const int32_t* __restrict__ nbr, const int32_t* __restrict__ nnbr, int n, int cap,
                            uint32_t* __restrict__ rcnt, uint32_t* __restrict__ rslot, uint32_t* status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)cap * n) return;
  const int k = (int)(e / n), i = (int)(e % n);
  if (k >= min(nnbr[i], cap)) return;
  if (!LJ_IDX_OK((unsigned)nbr[e] < (unsigned)n, status)) return;
  rslot[e] = atomicAdd(&rcnt[nbr[e]], 1u);
}

__global__ void k_rev_scatter(const int32_t* __restrict__ nbr, const int32_t* __restrict__ nnbr, int n, int cap,
                              const uint32_t* __restrict__ rstart, const uint32_t* __restrict__ rslot,
                              unsigned long long* __restrict__ rkey, uint32_t* status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)cap * n) return;
  const int k = (int)(e / n), i = (int)(e % n);
  if (k >= min(nnbr[i], cap)) return;
  if (!LJ_IDX_OK((unsigned)nbr[e] < (unsigned)n, status)) return;
  rkey[rstart[nbr[e]] + rslot[e]] = (unsigned long long)e;
}

// Pass 2: F_j += (24 eps / u) * sum of j's slots, summed in ascending entry order.
template <typename R>
__global__ void k_twopass_gather(int n, int cap, const uint32_t* __restrict__ rstart,
                                 const unsigned long long* __restrict__ rkey, const R* __restrict__ slot,
                                 double e24u, double* __restrict__ fx, double* __restrict__ fy,
                                 double* __restrict__ fz, uint32_t* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t ne = (int64_t)cap * n;
  R sx = 0, sy = 0, sz = 0;
  for (uint32_t q = rstart[j]; q < rstart[j + 1]; ++q) {
    const int64_t e = (int64_t)rkey[q];
    if (!LJ_IDX_OK(e < ne, status)) break;
    sx += slot[e];
    sy += slot[ne + e];
    sz += slot[2 * ne + e];
  }
  fx[j] += e24u * Prec<R>::to_d(sx);
  fy[j] += e24u * Prec<R>::to_d(sy);
  fz[j] += e24u * Prec<R>::to_d(sz);
}

static inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_build_verlet(Ctx& c, int half, int colmajor, uint32_t* maxlen) {
  const int64_t n = c.n;
  cudaError_t e = build_tiles(c, -32);  // single-cell tiles: exact 27-cell candidate sets
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.tile_ctr, 0, sizeof(uint32_t), c.stream)) != cudaSuccess) return e;
  const uint32_t* ntiles = c.ntiles_dev;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256 + 1, 152 * 8);
  auto k = half ? (colmajor ? k_build_verlet<true, true> : k_build_verlet<true, false>)
                : (colmajor ? k_build_verlet<false, true> : k_build_verlet<false, false>);
  k<<<blocks, 256, 0, c.stream>>>(c.pos, c.cell_start, c.binned_nc, (int)n, c.Rl2, c.vl_cap, c.tiles, ntiles,
                                  c.tile_ctr, c.nbr, c.nnbr, c.x_build, maxlen, c.status, c.rl2p_lo, c.rl2p_hi);
  return cudaGetLastError();
}

// 16-bit copy of the lists: entry j stored as j - i wrapped into [-n/2, n/2);
// any entry outside the int16 range sets *overflow (the 32-bit list is used).
__global__ void k_list_to16(const int32_t* __restrict__ nbr, const int32_t* __restrict__ nnbr, int64_t n, int cap,
                            int colmajor, int16_t* __restrict__ out, uint32_t* __restrict__ overflow,
                            uint32_t* status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)cap * n) return;
  const int64_t i = colmajor ? e % n : e / cap;
  const int k = colmajor ? (int)(e / n) : (int)(e % cap);
  if (k >= min(nnbr[i], cap)) return;
  if (!LJ_IDX_OK((uint64_t)(uint32_t)nbr[e] < (uint64_t)n, status)) return;
  int64_t d = (int64_t)nbr[e] - i;
  if (d >= (n + 1) / 2) d -= n;
  if (d < -(n / 2)) d += n;
  if (d < -32768 || d > 32767) {
    atomicOr(overflow, 1u);
    return;
  }
  out[e] = (int16_t)d;
}

cudaError_t launch_list_to16(Ctx& c, uint32_t* overflow) {
  const int64_t ne = (int64_t)c.vl_cap * c.n;
  if ((size_t)ne > c.nbr16_cap) {
    if (c.nbr16) cudaFree(c.nbr16);
    c.nbr16 = nullptr;
    c.nbr16_cap = 0;
    cudaError_t e = cudaMalloc(&c.nbr16, (size_t)ne * sizeof(int16_t));
    if (e != cudaSuccess) return e;
    c.nbr16_cap = (size_t)ne;
  }
  cudaError_t e = cudaMemsetAsync(overflow, 0, sizeof(uint32_t), c.stream);
  if (e != cudaSuccess) return e;
  k_list_to16<<<nb(ne, 256), 256, 0, c.stream>>>(c.nbr, c.nnbr, c.n, c.vl_cap, c.vl_colmajor, c.nbr16, overflow,
                                                  c.status);
  return cudaGetLastError();
}

cudaError_t launch_reverse_index(Ctx& c) {
  const int64_t n = c.n, ne = (int64_t)c.vl_cap * n;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c.rev_cnt, 0, (size_t)(n + 1) * sizeof(uint32_t), c.stream)) != cudaSuccess) return e;
  k_rev_count<<<nb(ne, 256), 256, 0, c.stream>>>(c.nbr, c.nnbr, (int)n, c.vl_cap, c.rev_cnt, c.rev_slot,
                                                 c.status);
  if ((e = excl_scan_u32(c, c.rev_cnt, c.rev_start, n)) != cudaSuccess) return e;
  k_rev_scatter<<<nb(ne, 256), 256, 0, c.stream>>>(c.nbr, c.nnbr, (int)n, c.vl_cap, c.rev_start, c.rev_slot,
                                                   c.rev_key, c.status);
  if ((e = sort_segments(c, c.rev_start, n, c.rev_key, c.rev_key2)) != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_twopass_gather(Ctx& c) {
  const int64_t n = c.n;
  if (c.prec == LJ_PREC_FP64)
    k_twopass_gather<double><<<nb(n, 256), 256, 0, c.stream>>>((int)n, c.vl_cap, c.rev_start, c.rev_key2,
                                                               (const double*)c.twopass, c.P.e24u, c.frc,
                                                               c.frc + n, c.frc + 2 * n, c.status);
  else
    k_twopass_gather<float><<<nb(n, 256), 256, 0, c.stream>>>((int)n, c.vl_cap, c.rev_start, c.rev_key2,
                                                              (const float*)c.twopass, c.P.e24u, c.frc, c.frc + n,
                                                              c.frc + 2 * n, c.status);
  return cudaGetLastError();
}

}  // namespace ljgb

// k_verlet.cu -- Verlet-list construction (Sec. 2.1.1: neighbour lists of the
// particles within cutoff + skin, built with the help of the linked-cell
// structure and rebuilt every few steps).
//
// The builder walks tiles of <= 32 consecutive particles of one cell (so a
// tile's candidates are exactly the 27 cells around it): a warp loads each
// 32-particle chunk of
// the tile's neighbour segments once, then for every i of the tile tests the
// chunk's 32 j's (one per lane) with the exact integer rule, keeps j != i with
// 0 < R^2 <= floor((r_l/u)^2) (half lists: j > i), and compacts the survivors
// with a warp ballot: each kept lane's slot is i's running count plus the
// number of kept lanes below it.  Every i therefore receives its j's in the
// scan order of rows (dz, dy) and ascending index, and its entries of one chunk
// are written as consecutive stores.  The tile's running counts live in lane
// registers (lane q holds the q-th particle's), and the coarse float screen
// (coarse_r2) settles every candidate except those in a thin band around r_l,
// which get the exact 64-bit test.  Lists longer than the capacity keep
// counting, set ST_CAPACITY and report the longest list so the host can
// regrow and rebuild.
#include "k_force_lc.cuh"

namespace ljgb {

__global__ void __launch_bounds__(256) k_build_verlet(const uint4* __restrict__ pos, const uint32_t* __restrict__ cs,
                                                      int nc, int n, uint64_t Rl2, int half, int cap, int colmajor,
                                                      const uint4* __restrict__ tiles,
                                                      const uint32_t* __restrict__ ntiles_ptr,
                                                      uint32_t* __restrict__ tile_ctr, int32_t* __restrict__ nbr,
                                                      int32_t* __restrict__ nnbr, uint32_t* __restrict__ xb,
                                                      uint32_t* __restrict__ maxlen, uint32_t* __restrict__ status,
                                                      float rl2p_lo, float rl2p_hi) {
  __shared__ uint4 s_i[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t ntiles = *ntiles_ptr;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(tile_ctr, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntiles) break;
    const uint4 tile = tiles[t];
    const int cf = (int)(tile.w & 0xffffu), cl = (int)(tile.w >> 16);
    const uint32_t ni = tile.y - tile.x;
    if (lane < (int)ni) {
      const uint4 p = pos[tile.x + lane];
      s_i[wib][lane] = p;
      xb[tile.x + lane] = p.x;
      xb[(int64_t)n + tile.x + lane] = p.y;
      xb[2 * (int64_t)n + tile.x + lane] = p.z;
    }
    uint32_t my_cnt = 0;  // lane q counts the list of the tile's q-th particle
    __syncwarp();
    Seg segs[18];
    const int ns = make_segments<false>(cs, nc, (int)tile.z, cf, cl, tile.x, segs);
#pragma unroll 1
    for (int s = 0; s < ns; ++s) {
#pragma unroll 1
      for (uint32_t jb = segs[s].b; jb < segs[s].e; jb += 32) {
        const uint32_t j = jb + lane;
        const bool vj = j < segs[s].e;
        const uint4 pj = vj ? pos[j] : make_uint4(0, 0, 0, 0);
#pragma unroll 4
        for (uint32_t q = 0; q < ni; ++q) {
          const uint4 pi = s_i[wib][q];
          const uint32_t i = tile.x + q;
          const int da = mimg(pi.x, pj.x), db = mimg(pi.y, pj.y), dc = mimg(pi.z, pj.z);
          const float r2p = coarse_r2(da, db, dc);
          // coarse screen decides both sides; only the thin band needs the exact test
          bool in = vj && ((da | db | dc) != 0) && (!half || j > i) && r2p <= rl2p_hi;
          if (in && r2p >= rl2p_lo) in = in_cut_exact(da, db, dc, Rl2);
          const unsigned mask = __ballot_sync(0xffffffffu, in);
          const uint32_t base = __shfl_sync(0xffffffffu, my_cnt, (int)q);
          if (in) {
            const uint32_t k = base + __popc(mask & lt);
            if (k < (uint32_t)cap) {
              if (colmajor)
                nbr[(int64_t)k * n + i] = (int32_t)j;
              else
                nbr[(int64_t)i * cap + k] = (int32_t)j;
            }
          }
          if (lane == (int)q) my_cnt += __popc(mask);
        }
      }
    }
    if (lane < (int)ni) {
      nnbr[tile.x + lane] = (int32_t)my_cnt;
      if (my_cnt > (uint32_t)cap) atomicOr(status, ST_CAPACITY);
      atomicMax(maxlen, my_cnt);
    }
    __syncwarp();
  }
}

// Reverse index of a half list for the two-pass Newton-3 reduction:
// rstart[j]..rstart[j+1] holds the entry ids e = k * n + i (column-major
// slots) of all entries with nbr[e] = j, in ascending e.
__global__ void k_rev_count(const int32_t* __restrict__ nbr, const int32_t* __restrict__ nnbr, int n, int cap,
                            uint32_t* __restrict__ rcnt, uint32_t* __restrict__ rslot) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)cap * n) return;
  const int k = (int)(e / n), i = (int)(e % n);
  if (k >= min(nnbr[i], cap)) return;
  rslot[e] = atomicAdd(&rcnt[nbr[e]], 1u);
}

__global__ void k_rev_scatter(const int32_t* __restrict__ nbr, const int32_t* __restrict__ nnbr, int n, int cap,
                              const uint32_t* __restrict__ rstart, const uint32_t* __restrict__ rslot,
                              unsigned long long* __restrict__ rkey) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)cap * n) return;
  const int k = (int)(e / n), i = (int)(e % n);
  if (k >= min(nnbr[i], cap)) return;
  rkey[rstart[nbr[e]] + rslot[e]] = (unsigned long long)e;
}

// Pass 2: F_j += (24 eps / u) * sum of j's slots, summed in ascending entry order.
template <typename R>
__global__ void k_twopass_gather(int n, int cap, const uint32_t* __restrict__ rstart,
                                 const unsigned long long* __restrict__ rkey, const R* __restrict__ slot,
                                 double e24u, double* __restrict__ fx, double* __restrict__ fy,
                                 double* __restrict__ fz) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t ne = (int64_t)cap * n;
  R sx = 0, sy = 0, sz = 0;
  for (uint32_t q = rstart[j]; q < rstart[j + 1]; ++q) {
    const int64_t e = (int64_t)rkey[q];
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
  const int blocks = (int)std::min<int64_t>((n + 255) / 256 + 1, 152 * 8);
  k_build_verlet<<<blocks, 256, 0, c.stream>>>(c.pos, c.cell_start, c.binned_nc, (int)n, c.Rl2, half, c.vl_cap,
                                                colmajor, c.tiles, c.row_tiles + (size_t)c.binned_nc * c.binned_nc,
                                                c.tile_ctr, c.nbr, c.nnbr, c.x_build, maxlen, c.status, c.rl2p_lo,
                                                c.rl2p_hi);
  return cudaGetLastError();
}

// 16-bit copy of the lists: entry j stored as j - i wrapped into [-n/2, n/2);
// any entry outside the int16 range sets *overflow (the 32-bit list is used).
__global__ void k_list_to16(const int32_t* __restrict__ nbr, const int32_t* __restrict__ nnbr, int64_t n, int cap,
                            int colmajor, int16_t* __restrict__ out, uint32_t* __restrict__ overflow) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)cap * n) return;
  const int64_t i = colmajor ? e % n : e / cap;
  const int k = colmajor ? (int)(e / n) : (int)(e % cap);
  if (k >= min(nnbr[i], cap)) return;
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
  k_list_to16<<<nb(ne, 256), 256, 0, c.stream>>>(c.nbr, c.nnbr, c.n, c.vl_cap, c.vl_colmajor, c.nbr16, overflow);
  return cudaGetLastError();
}

cudaError_t launch_reverse_index(Ctx& c) {
  const int64_t n = c.n, ne = (int64_t)c.vl_cap * n;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c.rev_cnt, 0, (size_t)(n + 1) * sizeof(uint32_t), c.stream)) != cudaSuccess) return e;
  k_rev_count<<<nb(ne, 256), 256, 0, c.stream>>>(c.nbr, c.nnbr, (int)n, c.vl_cap, c.rev_cnt, c.rev_slot);
  if ((e = excl_scan_u32(c, c.rev_cnt, c.rev_start, n)) != cudaSuccess) return e;
  k_rev_scatter<<<nb(ne, 256), 256, 0, c.stream>>>(c.nbr, c.nnbr, (int)n, c.vl_cap, c.rev_start, c.rev_slot,
                                                   c.rev_key);
  if ((e = sort_segments(c, c.rev_start, n, c.rev_key, c.rev_key2)) != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_twopass_gather(Ctx& c) {
  const int64_t n = c.n;
  if (c.prec == LJ_PREC_FP64)
    k_twopass_gather<double><<<nb(n, 256), 256, 0, c.stream>>>((int)n, c.vl_cap, c.rev_start, c.rev_key2,
                                                               (const double*)c.twopass, c.P.e24u, c.frc,
                                                               c.frc + n, c.frc + 2 * n);
  else
    k_twopass_gather<float><<<nb(n, 256), 256, 0, c.stream>>>((int)n, c.vl_cap, c.rev_start, c.rev_key2,
                                                              (const float*)c.twopass, c.P.e24u, c.frc, c.frc + n,
                                                              c.frc + 2 * n);
  return cudaGetLastError();
}

}  // namespace ljgb

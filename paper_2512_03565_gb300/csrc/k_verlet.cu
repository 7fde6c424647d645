// k_verlet.cu -- Verlet-list construction (Sec. 2.1.1: neighbour lists of the
// particles within cutoff + skin, built with the help of the linked-cell
// structure and rebuilt every few steps).
//
// The builder walks tiles of <= 32 consecutive particles of one cell (so a
// tile's candidates are exactly the 27 cells around it), keeps j != i with
// 0 < R^2 <= floor((r_l/u)^2) by the exact integer rule (half lists: j > i),
// and gives every i its j's in the scan order of rows (dz, dy) and ascending
// index.  A coarse float screen settles every candidate except those in a thin
// band around r_l, which get the exact 64-bit test: each particle's
// coordinates floor(x / 512) are exact floats, the segment's periodic image is
// one addition per loaded j, and a test is three exact subtractions and an FMA
// sum (the same bound as coarse_r2, since floor(x_j/512) - floor(x_i/512) is
// within 1 of (x_j - x_i)/512).
// The warp holds 32 j's, one per lane, and takes the tile's i's in turn;
// survivors are compacted with a warp ballot (lane q holds the q-th particle's
// running count), so each i's entries of one chunk are consecutive stores.
// Lists longer than the capacity keep counting, set ST_CAPACITY and report
// the longest list so the host can regrow and rebuild.
#include "k_force_lc.cuh"

namespace ljgb {

// Coarse coordinate of a fixed-point value: floor(x / 512) as an exact float
// (the bits of 2^23 + v read as a float are 2^23 + v for v < 2^23).
__device__ __forceinline__ float coarse_coord(uint32_t x) {
  return __int_as_float((int)((x >> 9) | 0x4B000000u)) - 8388608.0f;
}

// Segments of a single-cell tile's 27-cell neighbourhood with the periodic
// shift (in coarse units, 2^23 per box edge) that brings each segment's j's to
// the image nearest the tile; mixed = the segment covers a whole row whose
// images differ per pair (only when nc = 3), which uses the integer path.
struct BSeg {
  uint32_t b, e;
  float sx, sy, sz;
  int mixed;
};

__device__ __forceinline__ int builder_segments(const uint32_t* __restrict__ cs, int nc, int row, int cx,
                                                BSeg* out) {
  const int cy = row % nc, cz = row / nc;
  const float E = 8388608.0f;  // 2^23 coarse units per box edge
  int ns = 0;
#pragma unroll 1
  for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll 1
    for (int dy = -1; dy <= 1; ++dy) {
      const int zz = cz + dz, yy = cy + dy;
      const float sz = zz < 0 ? -E : (zz >= nc ? E : 0.0f);
      const float sy = yy < 0 ? -E : (yy >= nc ? E : 0.0f);
      const int r = ((zz + nc) % nc) * nc + (yy + nc) % nc;
      const int64_t base = (int64_t)r * nc;
      const int lo = cx - 1, hi = cx + 1;
      if (hi - lo + 1 >= nc) {
        out[ns++] = {cs[base], cs[base + nc], 0.0f, sy, sz, 1};
      } else if (lo < 0) {
        out[ns++] = {cs[base], cs[base + hi + 1], 0.0f, sy, sz, 0};
        out[ns++] = {cs[base + nc - 1], cs[base + nc], -E, sy, sz, 0};
      } else if (hi >= nc) {
        out[ns++] = {cs[base], cs[base + 1], E, sy, sz, 0};
        out[ns++] = {cs[base + lo], cs[base + nc], 0.0f, sy, sz, 0};
      } else {
        out[ns++] = {cs[base + lo], cs[base + hi + 1], 0.0f, sy, sz, 0};
      }
    }
  }
  return ns;
}

// One candidate test of the builder for lane j against the tile's q-th
// particle i, ballot compaction and the store of the survivors.
template <bool HALF, bool COLMAJOR, bool EXACT>
__device__ __forceinline__ void bv_test(const float4& ci, const uint4& pi, float jx, float jy, float jz,
                                        const uint4& pj, int j, uint32_t i, int q, int lane, unsigned lt, int n,
                                        int cap, uint64_t Rl2, float rl2p_lo, float rl2p_hi,
                                        int32_t* __restrict__ nbr, uint32_t& my_cnt) {
  bool in;
  if (!EXACT) {
    const float dx = jx - ci.x, dy = jy - ci.y, dz = jz - ci.z;  // exact (integers < 2^24)
    const float r2p = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    in = (HALF ? j > (int)i : j != (int)i) && r2p <= rl2p_hi;
    if (in && r2p >= rl2p_lo) in = in_cut_exact(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), Rl2);
  } else {
    in = j >= 0 && (HALF ? j > (int)i : j != (int)i) &&
         in_cut_exact(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), Rl2);
  }
  const unsigned mask = __ballot_sync(0xffffffffu, in);
  const uint32_t base = __shfl_sync(0xffffffffu, my_cnt, q);
  if (in) {
    const uint32_t k = base + __popc(mask & lt);
    if (k < (uint32_t)cap) {
      if (COLMAJOR)
        nbr[(int64_t)k * n + i] = j;
      else
        nbr[(int64_t)i * cap + k] = j;
    }
  }
  if (lane == q) my_cnt += __popc(mask);
}

// Chunks of 32 j's are packed across segment boundaries (each lane carries its
// own periodic shift), so a tile's ~27 cells take ceil(total / 32) chunks;
// lanes past the end sit at coarse -1e30 with j = -1 and are never accepted.
// A tile whose neighbourhood has a whole-row segment (n_c = 3) takes the
// per-segment path with the integer test for those rows.
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
  const unsigned lt = (1u << lane) - 1u;
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
    uint32_t my_cnt = 0;  // lane q counts the list of the tile's q-th particle
    __syncwarp();
    BSeg segs[18];
    const int ns = builder_segments(cs, nc, (int)tile.z, cx, segs);
    bool mixed = false;
    uint32_t total = 0;
    for (int s = 0; s < ns; ++s) {
      mixed |= segs[s].mixed != 0;
      total += segs[s].e - segs[s].b;
    }
    if (!mixed) {
      int sl = 0;
      uint32_t off = lane;  // this lane's position within segment sl
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        while (sl < ns && off >= segs[sl].e - segs[sl].b) {
          off -= segs[sl].e - segs[sl].b;
          ++sl;
        }
        int j = -1;
        uint4 pj = make_uint4(0, 0, 0, 0);
        float jx = -1e30f, jy = -1e30f, jz = -1e30f;
        if (sl < ns) {
          const BSeg& sg = segs[sl];
          j = (int)(sg.b + off);
          pj = pos[j];
          jx = coarse_coord(pj.x) + sg.sx;
          jy = coarse_coord(pj.y) + sg.sy;
          jz = coarse_coord(pj.z) + sg.sz;
        }
#pragma unroll 4
        for (int q = 0; q < ni; ++q)
          bv_test<HALF, COLMAJOR, false>(s_c[wib][q], s_i[wib][q], jx, jy, jz, pj, j, tile.x + q, q, lane, lt, n,
                                         cap, Rl2, rl2p_lo, rl2p_hi, nbr, my_cnt);
        off += 32;
      }
    } else {
#pragma unroll 1
      for (int s = 0; s < ns; ++s) {
        const BSeg sg = segs[s];
#pragma unroll 1
        for (uint32_t jb = sg.b; jb < sg.e; jb += 32) {
          const bool vj = jb + lane < sg.e;
          const int j = vj ? (int)(jb + lane) : -1;
          const uint4 pj = vj ? pos[j] : make_uint4(0, 0, 0, 0);
          const float jx = vj ? coarse_coord(pj.x) + sg.sx : -1e30f;
          const float jy = vj ? coarse_coord(pj.y) + sg.sy : -1e30f;
          const float jz = vj ? coarse_coord(pj.z) + sg.sz : -1e30f;
#pragma unroll 1
          for (int q = 0; q < ni; ++q) {
            if (sg.mixed)
              bv_test<HALF, COLMAJOR, true>(s_c[wib][q], s_i[wib][q], jx, jy, jz, pj, j, tile.x + q, q, lane, lt,
                                            n, cap, Rl2, rl2p_lo, rl2p_hi, nbr, my_cnt);
            else
              bv_test<HALF, COLMAJOR, false>(s_c[wib][q], s_i[wib][q], jx, jy, jz, pj, j, tile.x + q, q, lane, lt,
                                             n, cap, Rl2, rl2p_lo, rl2p_hi, nbr, my_cnt);
          }
        }
      }
    }
    if (lane < ni) {
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
  const uint32_t* ntiles = c.row_tiles + (size_t)c.binned_nc * c.binned_nc;
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

// k_verlet.cu -- Verlet-list construction (Sec. 2.1.1: neighbour lists of the
// particles within cutoff + skin, built with the help of the linked-cell
// structure and rebuilt every few steps).
//
// One warp per particle i scans the 27 cells of edge >= r_c + skin around its
// cell (9 rows, each an ascending run of cells) in strides of 32 candidates,
// keeps j != i with 0 < R^2 <= floor((r_l/u)^2) (half lists: j > i), and
// compacts the survivors with a warp ballot: each kept lane's slot is the
// running count plus the number of kept lanes below it, so the list keeps the
// scan order.  Lists longer than the capacity keep counting, set ST_CAPACITY
// and report the longest list so the host can regrow and rebuild.
#include "k_force_lc.cuh"

namespace ljgb {

__global__ void __launch_bounds__(256) k_build_verlet(const uint4* __restrict__ pos, const uint32_t* __restrict__ cs,
                                                      int nc, int n, uint64_t Rl2, int half, int cap, int colmajor,
                                                      int32_t* __restrict__ nbr, int32_t* __restrict__ nnbr,
                                                      uint32_t* __restrict__ xb, uint32_t* __restrict__ maxlen,
                                                      uint32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += nwarps) {
    const uint32_t i = (uint32_t)w;
    const uint4 pi = pos[i];
    const int cx = (int)cx_of(pi.x, nc), cy = (int)cx_of(pi.y, nc), cz = (int)cx_of(pi.z, nc);
    uint32_t count = 0;
#pragma unroll 1
    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll 1
      for (int dy = -1; dy <= 1; ++dy) {
        const int r = ((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc;
        Seg sg[2];
        const int ns = row_segments(cs, nc, r, cx - 1, cx + 1, sg);
#pragma unroll 1
        for (int s = 0; s < ns; ++s) {
#pragma unroll 1
          for (uint32_t jb = sg[s].b; jb < sg[s].e; jb += 32) {
            const uint32_t j = jb + lane;
            bool in = false;
            if (j < sg[s].e && j != i && (!half || j > i)) {
              const uint4 pj = pos[j];
              in = in_cut_exact(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), Rl2);
            }
            const unsigned mask = __ballot_sync(0xffffffffu, in);
            if (in) {
              const uint32_t k = count + __popc(mask & lt);
              if (k < (uint32_t)cap) {
                if (colmajor)
                  nbr[(int64_t)k * n + i] = (int32_t)j;
                else
                  nbr[(int64_t)i * cap + k] = (int32_t)j;
              }
            }
            count += __popc(mask);
          }
        }
      }
    }
    if (lane == 0) {
      nnbr[i] = (int32_t)count;
      if (count > (uint32_t)cap) atomicOr(status, ST_CAPACITY);
      atomicMax(maxlen, count);
    }
    if (lane < 3) xb[(int64_t)lane * n + i] = lane == 0 ? pi.x : (lane == 1 ? pi.y : pi.z);
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
  const int blocks = (int)std::min<int64_t>((n * 32 + 255) / 256, 152 * 64);
  k_build_verlet<<<blocks, 256, 0, c.stream>>>(c.pos, c.cell_start, c.binned_nc, (int)n, c.Rl2, half, c.vl_cap,
                                                colmajor, c.nbr, c.nnbr, c.x_build, maxlen, c.status);
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

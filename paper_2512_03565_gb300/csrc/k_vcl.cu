// k_vcl.cu -- Verlet cluster lists (Sec. 2.1.1: particles grouped into
// clusters of a fixed size, neighbour lists of whole clusters rebuilt every
// few steps; Sec. 5.1: cluster sizes 4, 6 and 8 and the interaction order
// aligned to them).
//
// Cluster order.  The box is cut into n_t x n_t towers over (x, y), n_t the
// largest k >= 1 with k^3 M <= n, so that a tower holds about n_t M particles
// and a cluster of M is about as tall as it is wide.  Particles are stored by
// tower (id cx n_t + cy), then z, then original index: a stable counting sort
// into n_t^3 tower cells (z-slabs of the towers, about M particles each) and a
// sort of each cell by (z, original index).  A tower's run is cut into
// clusters of M consecutive particles, the last one shorter.  No cluster wraps
// in x or y (a tower is one cell column) or in z (z ascends along the tower).
//
// Cluster pairs.  The box of a cluster is the min/max of its fixed-point
// coordinates.  I and J are neighbours iff sum_a d_a^2 <= floor((r_l/u)^2),
// with d_a the periodic distance of the two boxes' intervals on the 2^32
// circle, decided in 64-bit integers (so the lists are exact and equal the
// CPU oracle's).  The search visits the towers whose x and y ranges come
// within r_l of I's box and, in each, the z-window of clusters found by
// binary search; one warp per i-cluster appends with ballots.
//
// Member masks (reading R21).  A cluster pair found by the box test is kept
// only if some member pair (a-th particle of I, b-th of J, two different
// particles; for a half list's J = I only b > a) lies within r_l in the same
// exact integer rule, and its entry carries the mask of those member pairs,
// bit a * M + b.  The force kernels take a lane's pair only when its bit is
// set, and about a fifth of the box-test survivors (clusters of 4 at density
// 0.75) have an empty mask and are not listed at all.
//
// A list entry packs the j-cluster's first particle and its size:
// (begin << 3) | (size - 1), so the force kernels read one word per cluster,
// and its mask is a parallel 64-bit word.
#include "ljgb_internal.cuh"

namespace ljgb {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ uint32_t tcoord(uint32_t x, uint32_t nt) {
  return (uint32_t)(((unsigned long long)x * nt) >> 32);
}

// tower cell id (cx nt + cy) nt + cz and the slot within the cell
__global__ void k_tower_ids(const uint4* __restrict__ pos, int64_t n, uint32_t nt, uint32_t* __restrict__ cell_of,
                            uint32_t* __restrict__ slot, uint32_t* __restrict__ cnt) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint4 p = pos[s];
  const uint32_t c = (tcoord(p.x, nt) * nt + tcoord(p.y, nt)) * nt + tcoord(p.z, nt);
  cell_of[s] = c;
  slot[s] = atomicAdd(&cnt[c], 1u);
}

// key = (z << 32) | original index: the per-cell sort then orders by z with
// ties by original index
__global__ void k_tower_keys(const uint4* __restrict__ pos, int64_t n, const uint32_t* __restrict__ cell_of,
                             const uint32_t* __restrict__ slot, const uint32_t* __restrict__ cell_start,
                             unsigned long long* __restrict__ key) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint4 p = pos[s];
  key[cell_start[cell_of[s]] + slot[s]] = ((unsigned long long)p.z << 32) | (unsigned long long)p.w;
}

// Moves the state into the sorted order; the source slot of original index o
// is inv[o] (each thread reads and then rewrites only its own particle's entry).
__global__ void k_permute_orig(const unsigned long long* __restrict__ key, int64_t n, const uint4* __restrict__ pos,
                               const double* __restrict__ vel, const double* __restrict__ frc,
                               uint4* __restrict__ pos2, double* __restrict__ vel2, double* __restrict__ frc2,
                               uint32_t* __restrict__ inv, uint32_t* __restrict__ xb, uint32_t* status) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const uint32_t o = (uint32_t)(key[d] & 0xffffffffull);
  if (!LJ_IDX_OK(o < (uint64_t)n, status)) return;
  const uint32_t s = inv[o];
  if (!LJ_IDX_OK(s < (uint64_t)n, status)) return;
  const uint4 p = pos[s];
  pos2[d] = p;
  inv[o] = (uint32_t)d;
  xb[d] = p.x;  // positions at the build, for the skin/2 rule
  xb[n + d] = p.y;
  xb[2 * n + d] = p.z;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vel2[a * n + d] = vel[a * n + s];
    frc2[a * n + d] = frc[a * n + s];
  }
}

// clusters per tower: ceil(count / M)
__global__ void k_tower_ncl(const uint32_t* __restrict__ cell_start, int64_t ntow, uint32_t nt, int M,
                            uint32_t* __restrict__ ncl) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntow) return;
  const uint32_t c = cell_start[(t + 1) * nt] - cell_start[t * nt];
  ncl[t] = (c + (uint32_t)M - 1u) / (uint32_t)M;
}

// cluster boundaries of each tower; cl_start[ncl] = n is written by tower ntow-1
__global__ void k_tower_clusters(const uint32_t* __restrict__ cell_start, int64_t ntow, uint32_t nt, int M,
                                 const uint32_t* __restrict__ tower_cl, uint32_t* __restrict__ cl_start, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntow) return;
  const uint32_t b = cell_start[t * nt], e = cell_start[(t + 1) * nt];
  uint32_t k = tower_cl[t];
  for (uint32_t p = b; p < e; p += (uint32_t)M, ++k) cl_start[k] = p;
  if (t == ntow - 1) cl_start[tower_cl[ntow]] = (uint32_t)n;
}

// box of each cluster: lo = (xmin, ymin, zmin), hi = (xmax, ymax, zmax)
__global__ void k_cluster_boxes(const uint4* __restrict__ pos, const uint32_t* __restrict__ cl_start, int64_t ncl,
                                uint4* __restrict__ lo, uint4* __restrict__ hi) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncl) return;
  const uint32_t b = cl_start[c], e = cl_start[c + 1];
  uint4 p = pos[b];
  uint4 l = make_uint4(p.x, p.y, p.z, 0u), h = l;
  for (uint32_t k = b + 1; k < e; ++k) {
    p = pos[k];
    l.x = min(l.x, p.x);
    l.y = min(l.y, p.y);
    l.z = min(l.z, p.z);
    h.x = max(h.x, p.x);
    h.y = max(h.y, p.y);
    h.z = max(h.z, p.z);
  }
  lo[c] = l;
  hi[c] = h;
}

// periodic distance of two non-wrapping intervals on the 2^32 circle
__device__ __forceinline__ uint64_t ivgap(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
  if (a0 <= b1 && b0 <= a1) return 0ull;
  const uint32_t g1 = b0 - a1, g2 = a0 - b1;
  return (uint64_t)(g1 < g2 ? g1 : g2);
}

// Towers whose coordinate range meets [lo - R, hi + R] on one axis: the first
// tower and the count (cyclic); all towers when the widened interval could
// wrap onto its first tower.
__device__ __forceinline__ void tower_range(uint32_t lo, uint32_t hi, uint32_t R, uint32_t nt, uint32_t& first,
                                            uint32_t& count) {
  const uint64_t span = (uint64_t)(hi - lo) + 2ull * R;
  const uint64_t W = (4294967296ull + nt - 1) / nt;
  if (span + W >= 4294967296ull) {
    first = 0;
    count = nt;
    return;
  }
  first = tcoord(lo - R, nt);
  const uint32_t last = tcoord(hi + R, nt);
  count = (last + nt - first) % nt + 1u;
}

// first index in [b, e) with key[idx] >= v (keys non-decreasing)
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ key, uint32_t b, uint32_t e,
                                                    uint32_t v) {
  while (b < e) {
    const uint32_t m = (b + e) >> 1;
    if (key[m] < v) b = m + 1;
    else e = m;
  }
  return b;
}

struct VclBuildArgs {
  const uint4* pos;
  const uint32_t* cl_start;
  const uint4* lo;
  const uint4* hi;
  const uint32_t* zlo;   // per cluster zmin (for the binary searches)
  const uint32_t* zhi;   // per cluster zmax
  const uint32_t* tower_cl;
  int64_t ncl;
  uint32_t nt;
  uint64_t Rl2;
  uint32_t Rl;           // floor(sqrt(Rl2))
  int cap;
  int M;                 // cluster size (bit a * M + b of a mask)
  uint32_t* nbr;
  uint64_t* mask;
  int32_t* nn;
  uint32_t* maxlen;
  uint32_t* status;
};

// Mask of the member pairs of clusters I and J within r_l (exact integer
// rule); for J = I only the pairs b > a (half lists) or b != a (full lists).
template <bool HALF>
__device__ __forceinline__ uint64_t member_mask(const VclBuildArgs& A, uint32_t I, uint32_t J) {
  const uint32_t ib = A.cl_start[I], ni = A.cl_start[I + 1] - ib;
  const uint32_t jb = A.cl_start[J], nj = A.cl_start[J + 1] - jb;
  uint64_t m = 0;
  for (uint32_t b = 0; b < nj; ++b) {
    const uint4 q = A.pos[jb + b];
    for (uint32_t a = 0; a < ni; ++a) {
      if (J == I && (HALF ? b <= a : b == a)) continue;
      const uint4 p = A.pos[ib + a];
      if (in_cut_exact((int)(q.x - p.x), (int)(q.y - p.y), (int)(q.z - p.z), A.Rl2))
        m |= 1ull << (a * (uint32_t)A.M + b);
    }
  }
  return m;
}

// Cluster ranges of tower t whose z interval meets [zl - R, zh + R]
// (periodic): up to two index ranges [s1, e1) and [s2, e2).
__device__ __forceinline__ void z_window(const VclBuildArgs& A, uint32_t t, uint32_t zl, uint32_t zh, uint32_t& s1,
                                         uint32_t& e1, uint32_t& s2, uint32_t& e2) {
  const uint32_t b = A.tower_cl[t], e = A.tower_cl[t + 1];
  s2 = e2 = b;
  const uint64_t span = (uint64_t)(zh - zl) + 2ull * A.Rl;
  if (span >= 4294967295ull) {
    s1 = b;
    e1 = e;
    return;
  }
  const int64_t wlo = (int64_t)zl - (int64_t)A.Rl, whi = (int64_t)zh + (int64_t)A.Rl;
  if (wlo >= 0 && whi <= 4294967295ll) {
    s1 = lower_bound_u32(A.zhi, b, e, (uint32_t)wlo);          // first with zmax >= lo
    e1 = lower_bound_u32(A.zlo, s1, e, (uint32_t)whi + 1u);    // first with zmin > hi
    if ((uint32_t)whi == 0xffffffffu) e1 = e;
    return;
  }
  // the window wraps: [a, 2^32 - 1] and [0, c]
  const uint32_t a = (uint32_t)(wlo < 0 ? wlo + 4294967296ll : wlo);
  const uint32_t cc = (uint32_t)(whi > 4294967295ll ? whi - 4294967296ll : whi);
  s1 = lower_bound_u32(A.zhi, b, e, a);
  e1 = e;
  s2 = b;
  e2 = lower_bound_u32(A.zlo, b, e, cc + 1u);
  if (e2 > s1) {  // the two ranges meet: every cluster once
    s1 = b;
    e1 = e;
    s2 = e2 = b;
  }
}

template <bool HALF>
__global__ void __launch_bounds__(256) k_vcl_build(VclBuildArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < A.ncl; I += nwarps) {
    const uint4 li = A.lo[I], hi = A.hi[I];
    uint32_t fx, cx_n, fy, cy_n;
    tower_range(li.x, hi.x, A.Rl, A.nt, fx, cx_n);
    tower_range(li.y, hi.y, A.Rl, A.nt, fy, cy_n);
    const uint32_t ntw = cx_n * cy_n;
    uint32_t count = 0;
    for (uint32_t tb = 0; tb < ntw; tb += 32) {
      // this lane's tower and its (up to two) z-window ranges
      uint32_t s1 = 0, e1 = 0, s2 = 0, e2 = 0;
      const uint32_t q = tb + (uint32_t)lane;
      if (q < ntw) {
        const uint32_t ix = q % cx_n, iy = q / cx_n;
        const uint32_t tx = (fx + ix) % A.nt, ty = (fy + iy) % A.nt;
        z_window(A, tx * A.nt + ty, li.z, hi.z, s1, e1, s2, e2);
      }
      const uint32_t l1 = e1 - s1, len = l1 + (e2 - s2);
      // exclusive prefix of the lanes' candidate counts
      uint32_t incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t excl = incl - len;
      for (uint32_t cb = 0; cb < total; cb += 32) {
        const uint32_t k = cb + (uint32_t)lane;
        // owner lane: the last lane whose exclusive prefix is <= k
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t ex = __shfl_sync(0xffffffffu, excl, owner + step);
          if (ex <= k) owner += step;
        }
        const uint32_t o_ex = __shfl_sync(0xffffffffu, excl, owner);
        const uint32_t o_s1 = __shfl_sync(0xffffffffu, s1, owner);
        const uint32_t o_l1 = __shfl_sync(0xffffffffu, l1, owner);
        const uint32_t o_s2 = __shfl_sync(0xffffffffu, s2, owner);
        bool take = false;
        uint32_t J = 0;
        uint64_t mk = 0;
        if (k < total) {
          const uint32_t r = k - o_ex;
          J = r < o_l1 ? o_s1 + r : o_s2 + (r - o_l1);
          if ((!HALF || J >= (uint32_t)I) && LJ_IDX_OK((int64_t)J < A.ncl, A.status)) {
            const uint4 lj = A.lo[J], hj = A.hi[J];
            const uint64_t dx = ivgap(li.x, hi.x, lj.x, hj.x);
            const uint64_t dy = ivgap(li.y, hi.y, lj.y, hj.y);
            const uint64_t dz = ivgap(li.z, hi.z, lj.z, hj.z);
            if (dx * dx + dy * dy + dz * dz <= A.Rl2) {
              mk = member_mask<HALF>(A, (uint32_t)I, J);
              take = mk != 0ull;
            }
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (take) {
          const uint32_t p = count + (uint32_t)__popc(m & ((1u << lane) - 1u));
          if (p < (uint32_t)A.cap) {
            const uint32_t jb = A.cl_start[J], je = A.cl_start[J + 1];
            A.nbr[(int64_t)I * A.cap + p] = (jb << 3) | (je - jb - 1u);
            A.mask[(int64_t)I * A.cap + p] = mk;
          }
        }
        count += (uint32_t)__popc(m);
      }
    }
    if (lane == 0) {
      A.nn[I] = (int32_t)count;
      if (count > (uint32_t)A.cap) {
        atomicOr(A.status, ST_CAPACITY);
        atomicMax(A.maxlen, count);
      }
    }
  }
}

__global__ void k_split_z(const uint4* __restrict__ lo, const uint4* __restrict__ hi, int64_t ncl,
                          uint32_t* __restrict__ zlo, uint32_t* __restrict__ zhi) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncl) return;
  zlo[c] = lo[c].z;
  zhi[c] = hi[c].z;
}

template <typename T>
cudaError_t grow(T*& p, size_t& cap, size_t need) {
  if (need <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&p, need * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

}  // namespace

int vcl_ntower(int64_t n, int M) {
  if (M < 1 || n < 1) return 1;
  int64_t k = 1;
  while ((k + 1) * (k + 1) * (k + 1) * (int64_t)M <= n) ++k;
  return (int)k;
}

// Sorts the particles into cluster order for cluster size M, forms the
// clusters and their boxes, and snapshots the positions for the skin rule.
// Returns the number of clusters in *ncl_out (one host synchronisation).
cudaError_t vcl_bin(Ctx& c, int M, int64_t* ncl_out) {
  const int64_t n = c.n;
  const int nt = vcl_ntower(n, M);
  const int64_t ntow = (int64_t)nt * nt, ncell = ntow * nt;
  cudaError_t e;
  if ((e = grow(c.cell_start, c.cell_cap, (size_t)ncell + 1)) != cudaSuccess) return e;
  if ((e = grow(c.cnt, c.cnt_cap, (size_t)ncell + 1)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.cnt, 0, (size_t)ncell * sizeof(uint32_t), c.stream)) != cudaSuccess) return e;
  k_tower_ids<<<nblk(n, 256), 256, 0, c.stream>>>(c.pos, n, (uint32_t)nt, c.cell_of, c.slot, c.cnt);
  if ((e = excl_scan_u32(c, c.cnt, c.cell_start, ncell)) != cudaSuccess) return e;
  k_tower_keys<<<nblk(n, 256), 256, 0, c.stream>>>(c.pos, n, c.cell_of, c.slot, c.cell_start, c.key);
  unsigned long long* key2 = c.key + n;
  if ((e = sort_segments(c, c.cell_start, ncell, c.key, key2)) != cudaSuccess) return e;
  k_permute_orig<<<nblk(n, 256), 256, 0, c.stream>>>(key2, n, c.pos, c.vel, c.frc, c.pos_alt, c.vel_alt, c.frc_alt,
                                                      c.inv, c.x_build, c.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  std::swap(c.pos, c.pos_alt);
  std::swap(c.vel, c.vel_alt);
  std::swap(c.frc, c.frc_alt);
  c.binned_nc = nt;
  c.bin_gen += 1;
  // clusters
  if ((e = grow(c.tower_cl, c.tower_cl_cap, (size_t)ntow + 1)) != cudaSuccess) return e;
  k_tower_ncl<<<nblk(ntow, 256), 256, 0, c.stream>>>(c.cell_start, ntow, (uint32_t)nt, M, c.tower_cl);
  if ((e = excl_scan_u32(c, c.tower_cl, c.tower_cl, ntow)) != cudaSuccess) return e;
  uint32_t ncl = 0;
  if ((e = cudaMemcpyAsync(&ncl, c.tower_cl + ntow, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
  if ((e = grow(c.cl_start, c.cl_start_cap, (size_t)ncl + 1)) != cudaSuccess) return e;
  if ((e = grow(c.cl_lo, c.cl_lo_cap, (size_t)ncl + 1)) != cudaSuccess) return e;
  if ((e = grow(c.cl_hi, c.cl_hi_cap, (size_t)ncl + 1)) != cudaSuccess) return e;
  if ((e = grow(c.cl_z, c.cl_z_cap, 2 * ((size_t)ncl + 1))) != cudaSuccess) return e;
  k_tower_clusters<<<nblk(ntow, 256), 256, 0, c.stream>>>(c.cell_start, ntow, (uint32_t)nt, M, c.tower_cl,
                                                          c.cl_start, n);
  k_cluster_boxes<<<nblk(ncl, 256), 256, 0, c.stream>>>(c.pos, c.cl_start, ncl, c.cl_lo, c.cl_hi);
  k_split_z<<<nblk(ncl, 256), 256, 0, c.stream>>>(c.cl_lo, c.cl_hi, ncl, c.cl_z, c.cl_z + ncl + 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  c.vcl_nt = nt;
  c.vcl_ncl = ncl;
  c.vcl_M = M;
  *ncl_out = ncl;
  return cudaSuccess;
}

// Cluster-pair lists of the current cluster order (half: J >= I only).
cudaError_t launch_vcl_build(Ctx& c, int half, uint32_t* maxlen) {
  VclBuildArgs A;
  A.cl_start = c.cl_start;
  A.lo = c.cl_lo;
  A.hi = c.cl_hi;
  A.zlo = c.cl_z;
  A.zhi = c.cl_z + c.vcl_ncl + 1;
  A.tower_cl = c.tower_cl;
  A.ncl = c.vcl_ncl;
  A.nt = (uint32_t)c.vcl_nt;
  A.Rl2 = c.Rl2;
  uint64_t r = (uint64_t)std::sqrt((double)c.Rl2);
  while (r * r > c.Rl2) --r;
  while ((r + 1) * (r + 1) <= c.Rl2) ++r;
  A.Rl = (uint32_t)std::min<uint64_t>(r, 0xffffffffull);
  A.cap = c.vcl_cap;
  A.M = c.vcl_M;
  A.pos = c.pos;
  A.nbr = c.vcl_nbr;
  A.mask = c.vcl_mask;
  A.nn = c.vcl_nn;
  A.maxlen = maxlen;
  A.status = c.status;
  const int64_t threads = std::max<int64_t>(32, c.vcl_ncl * 32);
  const unsigned g = (unsigned)std::min<int64_t>((threads + 255) / 256, 152 * 8);
  if (half)
    k_vcl_build<true><<<g, 256, 0, c.stream>>>(A);
  else
    k_vcl_build<false><<<g, 256, 0, c.stream>>>(A);
  return cudaGetLastError();
}

}  // namespace ljgb

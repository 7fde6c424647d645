// k_bin.cu -- particle upload and Linked Cells binning (Sec. 2.1.1).
//
// The cell order is a stable counting sort by cell id: cell ids and per-cell
// slots from atomic counters, an exclusive scan of the counts (cell_start),
// a scatter, and a per-cell sort by original index, which makes the order
// unique (ties keep ascending original index) and independent of the order of
// the atomics.  All particle state is then permuted into cell order, which is
// the order every force kernel reads (structure of arrays, Sec. 2.3.1).
#include <mutex>

#include "ljgb_internal.cuh"

namespace ljgb {

// -------------------------------------------------------------------------
// upload
// -------------------------------------------------------------------------

// x_fp = floor(x / L * 2^32) mod 2^32 (the division and floors are exact
// IEEE-754 operations, so the host oracle's identical formula agrees bit for bit).
__device__ __forceinline__ uint32_t quantize_coord(double x, double L) {
  double t = x / L;
  t = t - floor(t);
  double s = floor(t * 4294967296.0);
  if (s >= 4294967296.0) s = 0.0;
  return (uint32_t)s;
}

__global__ void k_quantize(const double* __restrict__ pos, int64_t n, double L, const double* __restrict__ vel,
                           uint4* __restrict__ out, double* __restrict__ vout) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    q[a] = quantize_coord(pos[a * n + i], L);
    vout[a * n + i] = vel ? vel[a * n + i] : 0.0;
  }
  out[i] = make_uint4(q[0], q[1], q[2], (uint32_t)i);
}

// New coordinates in the caller's order written into the current (cell)
// order through the inverse permutation: particle o goes to slot inv[o],
// quantised as above.  x is read in the caller's order (coalesced), so it may
// also be the caller's pinned host memory read across the host link.
// With xb, the displacement since the last list build is checked as in the
// integrator's drift (skin/2) and a particle beyond it sets the mapped host
// word skin_flag.
__global__ void k_update_pos(uint4* __restrict__ pos, const uint32_t* __restrict__ inv, const double* __restrict__ x,
                             int64_t n, double L, const uint32_t* __restrict__ xb, uint64_t disp2_max,
                             uint32_t* skin_flag, uint32_t* status) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const uint32_t s = inv[o];
  if (!LJ_IDX_OK(s < (uint64_t)n, status)) return;
  const uint4 p = make_uint4(quantize_coord(x[o], L), quantize_coord(x[n + o], L), quantize_coord(x[2 * n + o], L),
                             (uint32_t)o);
  pos[s] = p;
  if (xb) {
    const int a = (int)(p.x - xb[s]), b = (int)(p.y - xb[n + s]), c = (int)(p.z - xb[2 * n + s]);
    const uint64_t d2 = (uint64_t)((long long)a * a) + (uint64_t)((long long)b * b) + (uint64_t)((long long)c * c);
    if (d2 > disp2_max) *skin_flag = 1u;
  }
}

// inv[o] = o: the order right after a load
__global__ void k_iota(uint32_t* __restrict__ inv, int64_t n) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n) inv[o] = (uint32_t)o;
}

__global__ void k_load_fp(const uint32_t* __restrict__ pos, int64_t n, const double* __restrict__ vel,
                          uint4* __restrict__ out, double* __restrict__ vout) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = make_uint4(pos[i], pos[n + i], pos[2 * n + i], (uint32_t)i);
#pragma unroll
  for (int a = 0; a < 3; ++a) vout[a * n + i] = vel ? vel[a * n + i] : 0.0;
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_quantize(const double* pos, int64_t n, double L, const double* vel, uint4* out_pos,
                            double* out_vel, cudaStream_t s) {
  k_quantize<<<nblk(n, 256), 256, 0, s>>>(pos, n, L, vel, out_pos, out_vel);
  return cudaGetLastError();
}

cudaError_t launch_update_pos(uint4* pos, const uint32_t* inv, const double* x, int64_t n, double L,
                              const uint32_t* xb, uint64_t disp2_max, uint32_t* skin_flag, cudaStream_t s,
                              uint32_t* status) {
  k_update_pos<<<nblk(n, 256), 256, 0, s>>>(pos, inv, x, n, L, xb, disp2_max, skin_flag, status);
  return cudaGetLastError();
}

cudaError_t launch_iota(uint32_t* inv, int64_t n, cudaStream_t s) {
  k_iota<<<nblk(n, 256), 256, 0, s>>>(inv, n);
  return cudaGetLastError();
}

cudaError_t launch_load_fp(const uint32_t* pos_fp, int64_t n, const double* vel, uint4* out_pos, double* out_vel,
                           cudaStream_t s) {
  k_load_fp<<<nblk(n, 256), 256, 0, s>>>(pos_fp, n, vel, out_pos, out_vel);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// exclusive scan of uint32 counts: out[k] = sum_{m<k} in[k], out[n] = total
// (in and out may alias).  Three passes: block scans of 4096 items, a scan of
// the block totals, and the carry-in add.
// -------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_TILE = SCAN_T * SCAN_I;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  uint32_t base = wid ? s_warp[wid - 1] : 0u;
  __syncthreads();
  return base + x - v;
}

__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                             uint32_t* __restrict__ block_tot) {
  __shared__ uint32_t s_warp[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
  uint32_t v[SCAN_I], sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    sum += v[k];
  }
  uint32_t tot;
  uint32_t off = block_excl_scan(sum, s_warp, tot);
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    if (base + k < n) out[base + k] = off;
    off += v[k];
  }
  if (threadIdx.x == 0) block_tot[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block totals, in place; writes the grand
// total to *total_out.
__global__ void k_scan_totals(uint32_t* __restrict__ tot, int64_t nb, uint32_t* __restrict__ total_out) {
  __shared__ uint32_t s_warp[32];
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += SCAN_TILE) {
    const int64_t base = b0 + (int64_t)threadIdx.x * SCAN_I;
    uint32_t v[SCAN_I], sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
      v[k] = (base + k < nb) ? tot[base + k] : 0u;
      sum += v[k];
    }
    uint32_t t;
    uint32_t off = block_excl_scan(sum, s_warp, t) + carry;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
      if (base + k < nb) tot[base + k] = off;
      off += v[k];
    }
    carry += t;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ block_off) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
  const uint32_t add = block_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k)
    if (base + k < n) out[base + k] += add;
}

// out has n + 1 entries.
cudaError_t excl_scan_u32(Ctx& c, const uint32_t* in, uint32_t* out, int64_t n) {
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if ((size_t)nb + 1 > c.scan_tmp_cap) {
    if (c.scan_tmp) cudaFree(c.scan_tmp);
    c.scan_tmp = nullptr;
    size_t cap = (size_t)nb + 1024;
    cudaError_t e = cudaMalloc(&c.scan_tmp, cap * sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    c.scan_tmp_cap = cap;
  }
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint32_t), c.stream);
  k_scan_tiles<<<(unsigned)nb, SCAN_T, 0, c.stream>>>(in, out, n, c.scan_tmp);
  k_scan_totals<<<1, SCAN_T, 0, c.stream>>>(c.scan_tmp, nb, out + n);
  k_scan_add<<<(unsigned)nb, SCAN_T, 0, c.stream>>>(out, n, c.scan_tmp);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// counting sort by cell
// -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cell_coord(uint32_t x, uint32_t nc) {
  return (uint32_t)(((unsigned long long)x * nc) >> 32);
}

__global__ void k_cell_ids(const uint4* __restrict__ pos, int64_t n, uint32_t nc, uint32_t* __restrict__ cell_of,
                           uint32_t* __restrict__ slot, uint32_t* __restrict__ cnt) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint4 p = pos[s];
  const uint32_t c = (cell_coord(p.z, nc) * nc + cell_coord(p.y, nc)) * nc + cell_coord(p.x, nc);
  cell_of[s] = c;
  slot[s] = atomicAdd(&cnt[c], 1u);
}

__global__ void k_scatter_keys(const uint4* __restrict__ pos, int64_t n, const uint32_t* __restrict__ cell_of,
                               const uint32_t* __restrict__ slot, const uint32_t* __restrict__ cell_start,
                               unsigned long long* __restrict__ key) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t d = cell_start[cell_of[s]] + slot[s];
  key[d] = ((unsigned long long)pos[s].w << 32) | (unsigned long long)s;
}

// One warp per cell.  Cells of <= 32 particles: bitonic sort in registers.
// Larger cells: each key's rank is the number of smaller keys in the cell
// (keys are distinct), written to the second buffer.
__global__ void k_sort_cells(const uint32_t* __restrict__ cell_start, int64_t ncell,
                             unsigned long long* __restrict__ key, unsigned long long* __restrict__ key2) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= ncell) return;
  const uint32_t b = cell_start[w], e = cell_start[w + 1];
  const uint32_t cnt = e - b;
  if (cnt <= 1u) {
    if (cnt == 1u && lane == 0) key2[b] = key[b];
    return;
  }
  if (cnt <= 32u) {
    unsigned long long v = (lane < (int)cnt) ? key[b + lane] : ~0ull;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
        const bool up = (lane & k) == 0;
        const bool low = (lane & j) == 0;
        v = (low == up) ? (v < o ? v : o) : (v > o ? v : o);
      }
    }
    if (lane < (int)cnt) key2[b + lane] = v;
    return;
  }
  for (uint32_t t = lane; t < cnt; t += 32) {
    const unsigned long long v = key[b + t];
    uint32_t r = 0;
    for (uint32_t q = 0; q < cnt; ++q) r += (key[b + q] < v) ? 1u : 0u;
    key2[b + r] = v;
  }
}

cudaError_t sort_segments(Ctx& c, const uint32_t* starts, int64_t nseg, unsigned long long* key,
                          unsigned long long* key2) {
  if (nseg <= 0) return cudaSuccess;
  k_sort_cells<<<nblk(nseg * 32, 256), 256, 0, c.stream>>>(starts, nseg, key, key2);
  return cudaGetLastError();
}

__global__ void k_permute(const unsigned long long* __restrict__ key, int64_t n, const uint4* __restrict__ pos,
                          const double* __restrict__ vel, const double* __restrict__ frc, uint4* __restrict__ pos2,
                          double* __restrict__ vel2, double* __restrict__ frc2, uint32_t* __restrict__ inv,
                          uint32_t* status) {
  int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const uint32_t s = (uint32_t)(key[d] & 0xffffffffull);
  if (!LJ_IDX_OK(s < (uint64_t)n, status)) return;
  const uint4 p = pos[s];
  pos2[d] = p;
  if (LJ_IDX_OK(p.w < (uint64_t)n, status)) inv[p.w] = (uint32_t)d;  // original index -> new slot
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vel2[a * n + d] = vel[a * n + s];
    frc2[a * n + d] = frc[a * n + s];
  }
}

template <typename T>
static cudaError_t grow(T*& p, size_t& cap, size_t need) {
  if (need <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&p, need * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

cudaError_t bin_cells(Ctx& c, int nc) {
  const int64_t n = c.n;
  const int64_t ncell = (int64_t)nc * nc * nc;
  cudaError_t e;
  if ((e = grow(c.cell_start, c.cell_cap, (size_t)ncell + 1)) != cudaSuccess) return e;
  if ((e = grow(c.cnt, c.cnt_cap, (size_t)ncell + 1)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.cnt, 0, (size_t)ncell * sizeof(uint32_t), c.stream)) != cudaSuccess) return e;
  k_cell_ids<<<nblk(n, 256), 256, 0, c.stream>>>(c.pos, n, (uint32_t)nc, c.cell_of, c.slot, c.cnt);
  if ((e = excl_scan_u32(c, c.cnt, c.cell_start, ncell)) != cudaSuccess) return e;
  k_scatter_keys<<<nblk(n, 256), 256, 0, c.stream>>>(c.pos, n, c.cell_of, c.slot, c.cell_start, c.key);
  unsigned long long* key2 = c.key + n;
  if ((e = sort_segments(c, c.cell_start, ncell, c.key, key2)) != cudaSuccess) return e;
  k_permute<<<nblk(n, 256), 256, 0, c.stream>>>(key2, n, c.pos, c.vel, c.frc, c.pos_alt, c.vel_alt, c.frc_alt,
                                                 c.inv, c.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  std::swap(c.pos, c.pos_alt);
  std::swap(c.vel, c.vel_alt);
  std::swap(c.frc, c.frc_alt);
  c.binned_nc = nc;
  c.bin_gen += 1;
  return cudaSuccess;
}

// -------------------------------------------------------------------------
// Row tiles for the linked-cell kernels.
//
// A row is the run of cells (0..nc-1, cy, cz); its particles are contiguous
// in cell order.  A tile is a run of at most T consecutive particles of one
// row whose cells span cx_first..cx_last with cx_last - cx_first <= nc - 3, so
// that the union of the tile's neighbour cells never wraps onto itself and
// the Newton-3 half shell stays exact (see k_force_lc.cu).
// tile = (begin, end, row, cx_first | cx_last << 16).
// -------------------------------------------------------------------------
template <bool WRITE>
__global__ void k_row_tiles(const uint32_t* __restrict__ cs, int nc, int Tsigned, uint32_t* __restrict__ row_cnt,
                            uint4* __restrict__ tiles) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nc * nc) return;
  // T < 0: tiles of at most |T| particles of a single cell
  const int T = Tsigned < 0 ? -Tsigned : Tsigned;
  const int maxspan = Tsigned < 0 ? 0 : nc - 3;
  uint32_t k = WRITE ? row_cnt[r] : 0u;
  uint32_t tb = 0, tn = 0;
  int cf = 0, cl = 0;
  bool open = false;
  for (int cx = 0; cx < nc; ++cx) {
    uint32_t a = cs[(int64_t)r * nc + cx], b = cs[(int64_t)r * nc + cx + 1];
    while (a < b) {
      if (open && (tn == (uint32_t)T || cx - cf > maxspan)) {
        if (WRITE) tiles[k] = make_uint4(tb, tb + tn, (uint32_t)r, (uint32_t)cf | ((uint32_t)cl << 16));
        ++k;
        open = false;
      }
      if (!open) {
        open = true;
        tb = a;
        tn = 0;
        cf = cx;
      }
      uint32_t m = min(b - a, (uint32_t)T - tn);
      tn += m;
      a += m;
      cl = cx;
    }
  }
  if (open) {
    if (WRITE) tiles[k] = make_uint4(tb, tb + tn, (uint32_t)r, (uint32_t)cf | ((uint32_t)cl << 16));
    ++k;
  }
  if (!WRITE) row_cnt[r] = k;
}

// Single-cell tiles (T < 0), one thread per cell: the same tiles as the row
// scan above, in the same (cell) order, from per-cell counts and their scan.
template <bool WRITE>
__global__ void k_cell_tiles(const uint32_t* __restrict__ cs, int64_t ncell, int nc, uint32_t T,
                             uint32_t* __restrict__ cnt_off, uint4* __restrict__ tiles) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const uint32_t b = cs[c], e = cs[c + 1];
  if (!WRITE) {
    cnt_off[c] = (e - b + T - 1u) / T;
    return;
  }
  const uint32_t row = (uint32_t)(c / nc), cx = (uint32_t)(c % nc);
  uint32_t k = cnt_off[c];
  for (uint32_t p = b; p < e; p += T) tiles[k++] = make_uint4(p, min(p + T, e), row, cx | (cx << 16));
}

cudaError_t build_tiles(Ctx& c, int T) {
  if (c.tiles_T == T && c.tiles_gen == c.bin_gen && c.tiles_for_nc == c.binned_nc) return cudaSuccess;
  const int nc = c.binned_nc;
  const int64_t nrow = (int64_t)nc * nc, ncell = nrow * nc;
  cudaError_t e;
  // worst case: one tile per particle plus one per row
  if ((e = grow(c.tiles, c.tiles_cap, (size_t)(c.n + nrow + 1))) != cudaSuccess) return e;
  if (T < 0) {
    if ((e = grow(c.row_tiles, c.row_tiles_cap, (size_t)ncell + 1)) != cudaSuccess) return e;
    k_cell_tiles<false><<<nblk(ncell, 256), 256, 0, c.stream>>>(c.cell_start, ncell, nc, (uint32_t)(-T),
                                                                c.row_tiles, c.tiles);
    if ((e = excl_scan_u32(c, c.row_tiles, c.row_tiles, ncell)) != cudaSuccess) return e;
    k_cell_tiles<true><<<nblk(ncell, 256), 256, 0, c.stream>>>(c.cell_start, ncell, nc, (uint32_t)(-T),
                                                               c.row_tiles, c.tiles);
    c.ntiles_dev = c.row_tiles + ncell;
  } else {
    if ((e = grow(c.row_tiles, c.row_tiles_cap, (size_t)nrow + 1)) != cudaSuccess) return e;
    k_row_tiles<false><<<nblk(nrow, 128), 128, 0, c.stream>>>(c.cell_start, nc, T, c.row_tiles, c.tiles);
    if ((e = excl_scan_u32(c, c.row_tiles, c.row_tiles, nrow)) != cudaSuccess) return e;
    k_row_tiles<true><<<nblk(nrow, 128), 128, 0, c.stream>>>(c.cell_start, nc, T, c.row_tiles, c.tiles);
    c.ntiles_dev = c.row_tiles + nrow;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  c.tiles_T = T;
  c.tiles_gen = c.bin_gen;
  c.tiles_for_nc = nc;
  return cudaSuccess;
}

}  // namespace ljgb

// ---------------------------------------------------------------------------
// Allocation-free binning entry point (lj_bin_cells_static).
//
// Some callers cannot allocate device memory at the moment they need cell
// lists: code that runs while another allocator owns the whole device pool
// (a framework's caching allocator sized to the card), real-time loops where
// a cudaMalloc's implicit synchronisation is not allowed, or host code that
// must not fail on allocation after start-up.  This variant of the binning
// kernels takes device inputs and outputs from the caller and keeps its own
// scratch (per-cell counters, per-particle cell ids and slots, sort keys and
// the scan's block totals) in the file-scope device array below, sized for at
// most LJ_STATIC_MAX_N particles and LJ_STATIC_MAX_CELLS cells.  Every GPU that
// loads the library holds this array until the process exits.
// ---------------------------------------------------------------------------
namespace ljgb {
namespace {

constexpr int64_t kStaticMaxN = 65536;       // LJ_STATIC_MAX_N
constexpr int64_t kStaticMaxCells = 32768;   // LJ_STATIC_MAX_CELLS (n_c <= 32)
constexpr int64_t kStaticScanBlocks = (kStaticMaxCells + SCAN_TILE - 1) / SCAN_TILE + 1;
// byte offsets of the scratch regions (each 256-byte aligned)
constexpr size_t kOffCnt = 0;
constexpr size_t kOffCellOf = kOffCnt + 256 * ((4 * (kStaticMaxCells + 1) + 255) / 256);
constexpr size_t kOffSlot = kOffCellOf + 4 * kStaticMaxN;
constexpr size_t kOffKey = kOffSlot + 4 * kStaticMaxN;
constexpr size_t kOffKey2 = kOffKey + 8 * kStaticMaxN;
constexpr size_t kOffScan = kOffKey2 + 8 * kStaticMaxN;
constexpr size_t kStaticBytes = kOffScan + 256 * ((4 * kStaticScanBlocks + 255) / 256);

static __device__ __align__(256) unsigned char g_bin_scratch[kStaticBytes];

// Device address of g_bin_scratch per device, looked up once per device with
// that device current.  In host code the symbol g_bin_scratch is only a
// host-side stand-in and must never be passed to a kernel.
std::mutex g_scratch_mu;
void* g_scratch_addr[128] = {nullptr};

cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_bin_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void k_cell_ids_soa(const uint32_t* __restrict__ pos, int64_t n, uint32_t nc, uint32_t* __restrict__ cell_of,
                               uint32_t* __restrict__ slot, uint32_t* __restrict__ cnt) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t c = (cell_coord(pos[2 * n + s], nc) * nc + cell_coord(pos[n + s], nc)) * nc + cell_coord(pos[s], nc);
  cell_of[s] = c;
  slot[s] = atomicAdd(&cnt[c], 1u);
}

__global__ void k_scatter_keys_soa(int64_t n, const uint32_t* __restrict__ cell_of, const uint32_t* __restrict__ slot,
                                   const uint32_t* __restrict__ cell_start, unsigned long long* __restrict__ key) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  key[cell_start[cell_of[s]] + slot[s]] = (unsigned long long)s << 32;
}

__global__ void k_keys_to_perm(const unsigned long long* __restrict__ key, int64_t n, uint32_t* __restrict__ perm) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) perm[k] = (uint32_t)(key[k] >> 32);
}

}  // namespace
}  // namespace ljgb

extern "C" lj_status lj_bin_cells_static(const uint32_t* pos_fp, int64_t n, int32_t nc, uint32_t* perm,
                                         uint32_t* cell_start, void* cuda_stream) {
  using namespace ljgb;
  if (!pos_fp || !perm || !cell_start || n < 1 || n > kStaticMaxN || nc < 1) return LJ_ERR_ARG;
  const int64_t ncell = (int64_t)nc * nc * nc;
  if (ncell > kStaticMaxCells) return LJ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // an error left by earlier, unrelated work on this thread is not this
  // call's: clear it, so that the launch checks below see only these launches
  (void)cudaGetLastError();
  void* base = nullptr;
  if (static_scratch(&base) != cudaSuccess) return LJ_ERR_CUDA;
  unsigned char* b = (unsigned char*)base;
  uint32_t* cnt = (uint32_t*)(b + kOffCnt);
  uint32_t* cell_of = (uint32_t*)(b + kOffCellOf);
  uint32_t* slot = (uint32_t*)(b + kOffSlot);
  unsigned long long* key = (unsigned long long*)(b + kOffKey);
  unsigned long long* key2 = (unsigned long long*)(b + kOffKey2);
  uint32_t* scan_tot = (uint32_t*)(b + kOffScan);
  // the counters keep the previous call's values: clear them first
  if (cudaMemsetAsync(cnt, 0, (size_t)ncell * sizeof(uint32_t), s) != cudaSuccess) return LJ_ERR_CUDA;
  k_cell_ids_soa<<<nblk(n, 256), 256, 0, s>>>(pos_fp, n, (uint32_t)nc, cell_of, slot, cnt);
  if (cudaGetLastError() != cudaSuccess) return LJ_ERR_CUDA;
  const int64_t nb = (ncell + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tiles<<<(unsigned)nb, SCAN_T, 0, s>>>(cnt, cell_start, ncell, scan_tot);
  if (cudaGetLastError() != cudaSuccess) return LJ_ERR_CUDA;
  k_scan_totals<<<1, SCAN_T, 0, s>>>(scan_tot, nb, cell_start + ncell);
  if (cudaGetLastError() != cudaSuccess) return LJ_ERR_CUDA;
  k_scan_add<<<(unsigned)nb, SCAN_T, 0, s>>>(cell_start, ncell, scan_tot);
  if (cudaGetLastError() != cudaSuccess) return LJ_ERR_CUDA;
  k_scatter_keys_soa<<<nblk(n, 256), 256, 0, s>>>(n, cell_of, slot, cell_start, key);
  if (cudaGetLastError() != cudaSuccess) return LJ_ERR_CUDA;
  k_sort_cells<<<nblk(ncell * 32, 256), 256, 0, s>>>(cell_start, ncell, key, key2);
  if (cudaGetLastError() != cudaSuccess) return LJ_ERR_CUDA;
  k_keys_to_perm<<<nblk(n, 256), 256, 0, s>>>(key2, n, perm);
  return cudaGetLastError() == cudaSuccess ? LJ_OK : LJ_ERR_CUDA;
}

// k_ensemble.cu -- many independent periodic boxes of uneven sizes advanced
// together by one persistent kernel launch (captured as a CUDA graph).
//
// The paper tunes one simulation; this batch path applies the same force
// functor (Sec. 4.1, Algorithm 1, here the JSPLIT<w> order over linked cells,
// Sec. 2.1.1) and velocity Verlet (Sec. 2.1) to a set of boxes at once.  All
// boxes' particles live in one set of arrays (box b owns [off_b, off_b + n_b)),
// and all boxes' cells in one cell space (box b owns [cell_off_b, ... + nc_b^3)),
// so every phase of an MD step is one grid-wide sweep over all boxes:
//
//   kick + drift  ->  cell ids + counts  ->  exclusive scan of the counts (3
//   sweeps)  ->  scatter of sort keys  ->  per-cell sort by original index  ->
//   permutation of the state into cell order  ->  forces  ->  closing kick
//
// The phases are separated by a grid barrier of this file (arrival counter +
// generation word in global memory).  The kernel is launched cooperatively, so
// every block is resident; each barrier wait is bounded and a wait that gives
// up sets ST_TIMEOUT and makes every block leave the kernel.  Boxes too small
// for 3 cells per axis (edge >= r_c) use an all-pairs loop over their box.
#include <cmath>
#include <vector>

#include "k_build.cuh"
#include "k_force_lc.cuh"

namespace ljgb {

struct EnsBox {
  double L;
  double dtu;       // dt 2^32 / L
  double e24u;      // 24 eps / u
  uint64_t Rc2;
  float S_hi, S_lo;
  float rc2p_lo, rc2p_hi;
  int32_t nc;       // cells per axis (1 = all-pairs box)
  int32_t n;
  int64_t off;      // first particle
  int64_t cell_off; // first cell
  // Verlet-list mode (lj_ensemble_set_lists): cells of edge >= r_c + skin
  int32_t ncv;      // cells per axis (1 = the whole box is one cell)
  int64_t cell_off_v;
  uint64_t Rl2;     // floor(((r_c + skin)/u)^2)
  float rl2p_lo, rl2p_hi;
  uint64_t skin2;   // (skin / 2 / u)^2: displacement that forces a rebuild
};

struct EnsArgs {
  int nboxes;
  int64_t ntot;
  int64_t ncells;
  const EnsBox* boxes;
  const uint16_t* box_of;  // per particle (constant: particles never leave their box)
  uint4* pos;
  uint4* pos_alt;
  double* vel;
  double* vel_alt;
  double* frc;
  double* frc_alt;
  uint32_t* cnt;         // ncells + 1
  uint32_t* cell_start;  // ncells + 1
  uint32_t* cell_of;
  uint32_t* slot;
  unsigned long long* key;
  unsigned long long* key2;
  uint32_t* scan_tot;    // per scan tile
  unsigned* bar;         // [0] arrivals, [1] generation
  uint32_t* status;
  unsigned long long* npairs;  // in-cutoff pair evaluations (each pair counted from both sides)
  double hdtm;
  int nsteps;
  int first_force;       // compute forces at the initial positions first
  uint32_t spin_limit;   // barrier wait bound (iterations of ~0.1 us)
  int skip_block;        // test hook: this block leaves before the first barrier (-1 = none)
  // Verlet-list mode
  int vl;                // 0: linked cells rebinned every step; 1: Verlet lists
  int rebuild_every;
  int cap;               // list capacity (row-major rows of cap entries)
  int64_t ncells_v;
  const uint16_t* cell_box_v;  // box of each list-grid cell
  int32_t* nbr;
  int32_t* nnbr;
  uint32_t* xb;          // [3][ntot] positions at the last build
  uint32_t* since_build; // steps since the last build (device word)
  uint32_t* skin_flag;   // a particle moved beyond skin/2 (device word)
};

constexpr int ENS_SCAN_I = 8;  // items per thread of the in-kernel scan

// Grid barrier.  Returns false when the kernel must stop (a wait timed out
// here or elsewhere).  gen counts the barriers this block has passed.
__device__ __forceinline__ bool ens_barrier(const EnsArgs& A, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    if (*((volatile uint32_t*)A.status) & ST_TIMEOUT) {
      ok = 0;
    } else {
      const unsigned arrived = atomicAdd(&A.bar[0], 1u);
      if (arrived == gridDim.x - 1) {
        A.bar[0] = 0u;
        __threadfence();
        atomicAdd(&A.bar[1], 1u);
      } else {
        ok = 0;
        for (uint32_t it = 0; it < A.spin_limit; ++it) {
          if (*((volatile unsigned*)&A.bar[1]) != gen) {
            ok = 1;
            break;
          }
          if (*((volatile uint32_t*)A.status) & ST_TIMEOUT) break;
          __nanosleep(100);
        }
        if (!ok) atomicOr(A.status, ST_TIMEOUT);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  gen += 1;
  return s_ok != 0;
}

__device__ __forceinline__ LJParams box_params(const EnsBox& B) {
  LJParams P;
  P.n = B.n;
  P.nc = B.nc;
  P.Rc2 = B.Rc2;
  P.S_hi = B.S_hi;
  P.S_lo = B.S_lo;
  P.rc2p_lo = B.rc2p_lo;
  P.rc2p_hi = B.rc2p_hi;
  P.S = 0.0;
  P.e24u = B.e24u;
  P.e24 = P.e4 = 0.0;
  return P;
}

// Block-wide exclusive scan of ENS_SCAN_I * blockDim.x items starting at base.
__device__ void ens_scan_tile(const uint32_t* in, uint32_t* out, int64_t n, int64_t base, uint32_t* tot_out) {
  __shared__ uint32_t s_w[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t b0 = base + (int64_t)threadIdx.x * ENS_SCAN_I;
  uint32_t v[ENS_SCAN_I], sum = 0;
#pragma unroll
  for (int k = 0; k < ENS_SCAN_I; ++k) {
    v[k] = (b0 + k < n) ? in[b0 + k] : 0u;
    sum += v[k];
  }
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < nw ? s_w[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_w[lane] = w;
  }
  __syncthreads();
  uint32_t off = (wid ? s_w[wid - 1] : 0u) + x - sum;
  if (tot_out && threadIdx.x == 0) *tot_out = s_w[nw - 1];
#pragma unroll
  for (int k = 0; k < ENS_SCAN_I; ++k) {
    if (b0 + k < n) out[b0 + k] = off;
    off += v[k];
  }
  __syncthreads();
}

// One atomic per warp and force phase for the pair counter (a per-iteration
// atomic on the single counter serialised in L2).
__device__ __forceinline__ void flush_pairs(const EnsArgs& A, uint32_t pairs) {
  unsigned long long wc = pairs;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);
  if ((threadIdx.x & 31) == 0 && wc) atomicAdd(A.npairs, wc);
}

template <int W>
__device__ __forceinline__ void ens_forces(const EnsArgs& A, const uint4* __restrict__ pos,
                                           const uint32_t* __restrict__ cs, double* __restrict__ fx) {
  constexpr int G = 32 / W;
  const int lane = threadIdx.x & 31, g = lane / W, sub = lane % W;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = A.ntot;
  uint32_t pairs = 0;  // this lane's in-cutoff pairs of the phase, added once per warp at its end
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * G < n; w += nwarps) {
    const int64_t i = w * G + g;
    const bool vi = i < n;
    const int b = vi ? (int)A.box_of[i] : 0;
    const EnsBox B = A.boxes[b];
    const LJParams P = box_params(B);
    const uint4 pi = vi ? pos[i] : make_uint4(0, 0, 0, 0);
    Seg segs[18];
    int ns = 0;
    if (vi) {
      if (B.nc >= 3) {
        const int nc = B.nc;
        const int cx = (int)cx_of(pi.x, nc), cy = (int)cx_of(pi.y, nc), cz = (int)cx_of(pi.z, nc);
        ns = make_segments<false>(cs + B.cell_off, nc, cz * nc + cy, cx, cx, (uint32_t)i, (uint32_t)i + 1u, segs);
        check_segs(segs, ns, (uint32_t)A.ntot, A.status);
      } else {
        segs[0] = {(uint32_t)B.off, (uint32_t)(B.off + B.n), 0};
        ns = 1;
      }
    }
    const int nsmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)ns);
    float ax = 0.f, ay = 0.f, az = 0.f, eu = 0.f, ew = 0.f;
    int cnt = 0;
#pragma unroll 1
    for (int s = 0; s < nsmax; ++s) {
      const Seg sg = (s < ns) ? segs[s] : Seg{0u, 0u, 0};
      const uint32_t trips = (sg.e - sg.b + W - 1) / W;
      const uint32_t tmax = __reduce_max_sync(0xffffffffu, trips);
#pragma unroll 1
      for (uint32_t q = 0; q < tmax; ++q) {
        const uint32_t j = sg.b + q * W + sub;
        if (j < sg.e) {
          const uint4 pj = pos[j];
          float af, bf, cf;
          const float fac = pair_f32<false, true>(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), P, af,
                                                  bf, cf, eu, ew, cnt);
          ax += fac * af;
          ay += fac * bf;
          az += fac * cf;
        }
      }
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    pairs += (uint32_t)cnt;
    if (vi && sub == 0) {
      const double f0 = -B.e24u * f2d_exact(ax), f1 = -B.e24u * f2d_exact(ay), f2 = -B.e24u * f2d_exact(az);
      fx[i] = f0;
      fx[n + i] = f1;
      fx[2 * n + i] = f2;
      if (!isfinite(f0) || !isfinite(f1) || !isfinite(f2)) atomicOr(A.status, ST_NONFINITE);
    }
  }
  flush_pairs(A, pairs);
}

// Forces over the Verlet lists (JSPLIT<W>: W lanes per particle stride over
// its row), the pair arithmetic of the single-box list kernels with the box's
// parameters.
template <int W>
__device__ __forceinline__ void ens_forces_vl(const EnsArgs& A, const uint4* __restrict__ pos,
                                              double* __restrict__ fx) {
  constexpr int G = 32 / W;
  const int lane = threadIdx.x & 31, g = lane / W, sub = lane % W;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = A.ntot;
  uint32_t pairs = 0;  // this lane's in-cutoff pairs of the phase, added once per warp at its end
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * G < n; w += nwarps) {
    const int64_t i = w * G + g;
    const bool vi = i < n;
    const EnsBox B = A.boxes[vi ? (int)A.box_of[i] : 0];
    const LJParams P = box_params(B);
    float ax = 0.f, ay = 0.f, az = 0.f, eu = 0.f, ew = 0.f;
    int cnt = 0;
    if (vi) {
      const uint4 pi = pos[i];
      const int m = min(A.nnbr[i], A.cap);
      const int32_t* row = A.nbr + i * A.cap;
      // the next batch's entries are loaded while this batch's pairs are
      // computed, as in the single-box list kernel
      int jc[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        jc[t] = (sub + t * W < m) ? __ldcs(row + sub + t * W) : (int)i;
        if (!LJ_IDX_OK((uint64_t)(uint32_t)jc[t] < (uint64_t)A.ntot, A.status)) jc[t] = (int)i;
      }
      for (int k0 = sub; k0 < m; k0 += W * 4) {
        uint4 pj[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) pj[t] = __ldg(pos + jc[t]);
        int jn[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int k = k0 + W * 4 + t * W;
          jn[t] = (k < m) ? __ldcs(row + k) : (int)i;
          if (!LJ_IDX_OK((uint64_t)(uint32_t)jn[t] < (uint64_t)A.ntot, A.status)) jn[t] = (int)i;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          float af, bf, cf;
          const float fac = pair_f32<false, false, true>(mimg(pi.x, pj[t].x), mimg(pi.y, pj[t].y),
                                                         mimg(pi.z, pj[t].z), P, af, bf, cf, eu, ew, cnt);
          ax += fac * af;
          ay += fac * bf;
          az += fac * cf;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) jc[t] = jn[t];
      }
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    pairs += (uint32_t)cnt;
    if (vi && sub == 0) {
      const double f0 = -B.e24u * f2d_exact(ax), f1 = -B.e24u * f2d_exact(ay), f2 = -B.e24u * f2d_exact(az);
      fx[i] = f0;
      fx[n + i] = f1;
      fx[2 * n + i] = f2;
      if (!isfinite(f0) || !isfinite(f1) || !isfinite(f2)) atomicOr(A.status, ST_NONFINITE);
    }
  }
  flush_pairs(A, pairs);
}

// The list build of every box: one warp per cell of the list grid, the cell's
// particles in tiles of <= 32 (bv_tile), against the 27 cells around it (the
// whole box when it holds fewer than 3 cells per axis).  Records the build
// positions for the skin check.
__device__ __forceinline__ void ens_build_lists(const EnsArgs& A, const uint4* __restrict__ pos,
                                                const uint32_t* __restrict__ cs) {
  __shared__ uint4 s_i[16][32];  // blocks of at most 512 threads
  __shared__ float4 s_c[16][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = A.ntot;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < A.ncells_v; c += nwarps) {
    const uint32_t cb = cs[c], ce = cs[c + 1];
    if (cb == ce) continue;
    const EnsBox& B = A.boxes[A.cell_box_v[c]];
    BSeg segs[18];
    int ns;
    if (B.ncv >= 3) {
      const int nc = B.ncv;
      const int64_t local = c - B.cell_off_v;
      ns = builder_segments(cs + B.cell_off_v, nc, (int)(local / nc), (int)(local % nc), segs);
    } else {
      segs[0] = {(uint32_t)B.off, (uint32_t)(B.off + B.n), 0.0f, 0.0f, 0.0f, 1};
      ns = 1;
    }
    for (uint32_t first = cb; first < ce; first += 32) {
      const int ni = (int)min(32u, ce - first);
      if (lane < ni) {
        const uint4 p = pos[first + lane];
        s_i[wib][lane] = p;
        s_c[wib][lane] = make_float4(coarse_coord(p.x), coarse_coord(p.y), coarse_coord(p.z), 0.0f);
        A.xb[first + lane] = p.x;
        A.xb[n + first + lane] = p.y;
        A.xb[2 * n + first + lane] = p.z;
      }
      const uint32_t cnt = bv_tile<false, false>(pos, segs, ns, first, ni, s_i[wib], s_c[wib], (int)n, A.cap, B.Rl2,
                                                 B.rl2p_lo, B.rl2p_hi, A.nbr);
      if (lane < ni) {
        A.nnbr[first + lane] = (int32_t)cnt;
        if (cnt > (uint32_t)A.cap) atomicOr(A.status, ST_CAPACITY);
      }
      __syncwarp();
    }
  }
}

template <int W, bool VL>
__global__ void k_ensemble(EnsArgs A) {
  unsigned gen = 0;
  const int64_t n = A.ntot;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t scan_tile = (int64_t)blockDim.x * ENS_SCAN_I;
  const double M = 6755399441055744.0;  // 1.5 * 2^52: fma(v, dtu, M) rounds v dtu to an integer
  if ((int)blockIdx.x == A.skip_block) return;
  uint4 *pos = A.pos, *pos2 = A.pos_alt;
  double *vel = A.vel, *vel2 = A.vel_alt, *frc = A.frc, *frc2 = A.frc_alt;
  const int total = A.nsteps + (A.first_force ? 1 : 0);
  for (int step = 0; step < total; ++step) {
    const bool move = !(A.first_force && step == 0);
    // ---- kick + drift (and, from the second step on, the previous closing kick);
    // with lists, the displacement since the last build is checked (skin/2)
    if (move) {
      for (int64_t i = tid; i < n; i += nthr) {
        const EnsBox& B = A.boxes[A.box_of[i]];
        const double dtu = B.dtu;
        uint4 p = pos[i];
        uint32_t* pc = &p.x;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double v = __fma_rn(A.hdtm, frc[a * n + i], vel[a * n + i]);
          vel[a * n + i] = v;
          pc[a] += (uint32_t)__double2loint(__fma_rn(v, dtu, M));
        }
        pos[i] = p;
        if (VL) {
          const int a = (int)(p.x - A.xb[i]), b = (int)(p.y - A.xb[n + i]), c = (int)(p.z - A.xb[2 * n + i]);
          const uint64_t d2 = (uint64_t)((long long)a * a) + (uint64_t)((long long)b * b) +
                              (uint64_t)((long long)c * c);
          if (d2 > B.skin2) *((volatile uint32_t*)A.skin_flag) = 1u;
        }
      }
    }
    if (VL && blockIdx.x == 0 && threadIdx.x == 0) *A.since_build += 1u;
    // linked cells rebin every step; lists are rebuilt on schedule or when a
    // particle left its skin (every block reads the same words after the barrier)
    if (!VL)
      for (int64_t c = tid; c < A.ncells; c += nthr) A.cnt[c] = 0u;
    if (!ens_barrier(A, gen)) return;
    const bool rebuild = !VL || *((volatile uint32_t*)A.since_build) >= (uint32_t)A.rebuild_every ||
                         *((volatile uint32_t*)A.skin_flag) != 0u;
    const int64_t ncells = VL ? A.ncells_v : A.ncells;
    if (rebuild) {
    if (VL) {
      for (int64_t c = tid; c < ncells; c += nthr) A.cnt[c] = 0u;
      if (!ens_barrier(A, gen)) return;
    }
    // ---- cell ids and counts
    for (int64_t i = tid; i < n; i += nthr) {
      const EnsBox& B = A.boxes[A.box_of[i]];
      const uint4 p = pos[i];
      const uint32_t nc = (uint32_t)(VL ? B.ncv : B.nc);
      const uint32_t c = (uint32_t)(VL ? B.cell_off_v : B.cell_off) +
                         (cx_of(p.z, nc) * nc + cx_of(p.y, nc)) * nc + cx_of(p.x, nc);
      A.cell_of[i] = c;
      A.slot[i] = atomicAdd(&A.cnt[c], 1u);
    }
    if (!ens_barrier(A, gen)) return;
    // ---- exclusive scan of the counts over all boxes' cells
    const int64_t nscan = (ncells + scan_tile - 1) / scan_tile;
    for (int64_t t = blockIdx.x; t < nscan; t += gridDim.x)
      ens_scan_tile(A.cnt, A.cell_start, ncells, t * scan_tile, &A.scan_tot[t]);
    if (!ens_barrier(A, gen)) return;
    if (blockIdx.x == 0) {
      uint32_t carry = 0;
      for (int64_t t0 = 0; t0 < nscan; t0 += scan_tile) {
        __shared__ uint32_t s_tot;
        ens_scan_tile(A.scan_tot + t0, A.scan_tot + t0, nscan - t0, 0, &s_tot);
        if (carry) {
          for (int64_t k = threadIdx.x; k < scan_tile && t0 + k < nscan; k += blockDim.x) A.scan_tot[t0 + k] += carry;
        }
        __syncthreads();
        carry += s_tot;
        __syncthreads();
      }
      if (threadIdx.x == 0) A.cell_start[ncells] = carry;
    }
    if (!ens_barrier(A, gen)) return;
    for (int64_t c = tid; c < ncells; c += nthr) A.cell_start[c] += A.scan_tot[c / scan_tile];
    if (!ens_barrier(A, gen)) return;
    // ---- scatter, per-cell sort, permutation
    for (int64_t i = tid; i < n; i += nthr)
      A.key[A.cell_start[A.cell_of[i]] + A.slot[i]] = ((unsigned long long)pos[i].w << 32) | (unsigned long long)i;
    if (!ens_barrier(A, gen)) return;
    {
      const int lane = threadIdx.x & 31;
      for (int64_t c = tid >> 5; c < ncells; c += nthr >> 5) {
        const uint32_t b = A.cell_start[c], e = A.cell_start[c + 1], m = e - b;
        if (m == 0) continue;
        if (m <= 32) {
          unsigned long long v = lane < (int)m ? A.key[b + lane] : ~0ull;
#pragma unroll
          for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
              const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
              const bool up = (lane & k) == 0, low = (lane & j) == 0;
              v = (low == up) ? (v < o ? v : o) : (v > o ? v : o);
            }
          if (lane < (int)m) A.key2[b + lane] = v;
        } else {
          for (uint32_t t = lane; t < m; t += 32) {
            const unsigned long long v = A.key[b + t];
            uint32_t r = 0;
            for (uint32_t q = 0; q < m; ++q) r += A.key[b + q] < v ? 1u : 0u;
            A.key2[b + r] = v;
          }
        }
      }
    }
    if (!ens_barrier(A, gen)) return;
    for (int64_t d = tid; d < n; d += nthr) {
      const uint32_t s = (uint32_t)(A.key2[d] & 0xffffffffull);
      pos2[d] = pos[s];
#pragma unroll
      for (int a = 0; a < 3; ++a) vel2[a * n + d] = vel[a * n + s];
    }
    {
      uint4* tp = pos; pos = pos2; pos2 = tp;
      double* tv = vel; vel = vel2; vel2 = tv;
      double* tf = frc; frc = frc2; frc2 = tf;
    }
    if (!ens_barrier(A, gen)) return;
    if (VL) {
      // ---- list build; a list beyond the capacity stops the run
      ens_build_lists(A, pos, A.cell_start);
      if (!ens_barrier(A, gen)) return;
      if (*((volatile uint32_t*)A.status) & ST_CAPACITY) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        *A.since_build = 0u;
        *A.skin_flag = 0u;
      }
    }
    }  // rebuild
    // ---- forces, then the closing kick of this step
    if (VL)
      ens_forces_vl<W>(A, pos, frc);
    else
      ens_forces<W>(A, pos, A.cell_start, frc);
    if (!ens_barrier(A, gen)) return;
    if (move) {
      for (int64_t i = tid; i < n; i += nthr)
#pragma unroll
        for (int a = 0; a < 3; ++a) vel[a * n + i] = __fma_rn(A.hdtm, frc[a * n + i], vel[a * n + i]);
    }
    if (!ens_barrier(A, gen)) return;
  }
  // the state ends in the buffers the pointers now name; record which via status bit 31
  if (blockIdx.x == 0 && threadIdx.x == 0 && pos != A.pos) atomicOr(A.status, 0x80000000u);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Ens {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool graph_failed = false;
  bool last_run_graph = false;  // the last run replayed a captured graph
  int nboxes = 0;
  int64_t ntot = 0, ncells = 0;
  std::vector<EnsBox> hb;
  std::vector<int64_t> counts;
  EnsArgs A{};
  double mass = 1.0, rc = 2.5, eps = 1.0, sigma = 1.0;
  double skin = 0.0;
  int W = 8, block = 256;
  bool forces_valid = false;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_W = 0, graph_block = 0, graph_steps = -1, graph_first = -1;
  double graph_dt = 0.0;
  std::string err;
};

}  // namespace ljgb

using namespace ljgb;

struct lj_ens {
  Ens e;
};

namespace {

uint64_t ens_cut2(double L, double r) {
  // floor((r/u)^2), u = L/2^32, by exact long division of the squared 53-bit mantissas
  int er = 0, eL = 0;
  const double fr = std::frexp(r, &er), fL = std::frexp(L, &eL);
  const unsigned __int128 mr = (uint64_t)std::ldexp(fr, 53), mL = (uint64_t)std::ldexp(fL, 53);
  const unsigned __int128 num = mr * mr, den = mL * mL;
  int k = 2 * (er - eL) + 64;
  unsigned __int128 q = num / den, rem = num - q * den;
  for (; k > 0; --k) {
    rem <<= 1;
    q <<= 1;
    if (rem >= den) {
      rem -= den;
      q |= 1;
    }
    if (q >> 64) return ~0ull;
  }
  if (k < 0) q = (-k >= 128) ? 0 : (q >> -k);
  return (uint64_t)q;
}

template <int W, bool VL>
cudaError_t ens_grid_w(int block, int& grid) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ensemble<W, VL>, block, 0);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  grid = per_sm * sms;
  return cudaSuccess;
}

// Cooperative launch (all blocks resident) through cudaLaunchKernelEx, which
// stream capture records as a cooperative kernel node.
template <int W, bool VL>
cudaError_t ens_launch_w(Ens& E, int grid) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(E.block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = E.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_ensemble<W, VL>, E.A);
}

template <bool VL>
cudaError_t ens_grid_v(Ens& E, int& grid) {
  switch (E.W) {
    case 2: return ens_grid_w<2, VL>(E.block, grid);
    case 4: return ens_grid_w<4, VL>(E.block, grid);
    case 16: return ens_grid_w<16, VL>(E.block, grid);
    case 32: return ens_grid_w<32, VL>(E.block, grid);
    default: return ens_grid_w<8, VL>(E.block, grid);
  }
}

template <bool VL>
cudaError_t ens_launch_v(Ens& E, int grid) {
  switch (E.W) {
    case 2: return ens_launch_w<2, VL>(E, grid);
    case 4: return ens_launch_w<4, VL>(E, grid);
    case 16: return ens_launch_w<16, VL>(E, grid);
    case 32: return ens_launch_w<32, VL>(E, grid);
    default: return ens_launch_w<8, VL>(E, grid);
  }
}

// Linked-cell and Verlet-list batches are separate instantiations, so that the
// linked-cell kernel carries none of the list code (registers, occupancy).
cudaError_t ens_grid(Ens& E, int& grid) { return E.A.vl ? ens_grid_v<true>(E, grid) : ens_grid_v<false>(E, grid); }

cudaError_t ens_launch(Ens& E, int grid) { return E.A.vl ? ens_launch_v<true>(E, grid) : ens_launch_v<false>(E, grid); }

}  // namespace

extern "C" {

lj_status lj_ensemble_create(lj_ens** out, int32_t nboxes, const double* box_L, const int64_t* counts,
                             const uint32_t* pos_fp, const double* vel, double cutoff, double eps, double sigma,
                             double mass, void* cuda_stream) {
  if (!out || nboxes < 1 || nboxes > 65535 || !box_L || !counts || !pos_fp) return LJ_ERR_ARG;
  if (!(cutoff > 0) || !(eps > 0) || !(sigma > 0) || !(mass > 0)) return LJ_ERR_ARG;
  *out = nullptr;
  lj_ens* h = new (std::nothrow) lj_ens();
  if (!h) return LJ_ERR_OOM;
  Ens& E = h->e;
  E.stream = (cudaStream_t)cuda_stream;
  if (!E.stream) {  // the legacy default stream cannot be captured into a graph
    if (cudaStreamCreateWithFlags(&E.stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return LJ_ERR_CUDA;
    }
    E.own_stream = true;
  }
  E.nboxes = nboxes;
  E.mass = mass;
  E.rc = cutoff;
  E.eps = eps;
  E.sigma = sigma;
  int64_t off = 0, coff = 0;
  for (int b = 0; b < nboxes; ++b) {
    const double L = box_L[b];
    if (!(L > 2 * cutoff) || counts[b] < 1) {
      lj_ensemble_destroy(h);
      return LJ_ERR_ARG;
    }
    EnsBox B{};
    B.L = L;
    const double u = std::ldexp(L, -32);
    B.e24u = 24.0 * eps / u;
    B.Rc2 = ens_cut2(L, cutoff);
    coarse_band(B.Rc2, &B.rc2p_lo, &B.rc2p_hi);
    const double S = sigma * sigma / (u * u);
    B.S_hi = (float)S;
    B.S_lo = (float)(S - (double)B.S_hi);
    const int nc = (int)std::floor(L / cutoff);
    B.nc = nc >= 3 ? nc : 1;
    B.n = (int32_t)counts[b];
    B.off = off;
    B.cell_off = coff;
    off += counts[b];
    coff += (int64_t)B.nc * B.nc * B.nc;
    E.hb.push_back(B);
    E.counts.push_back(counts[b]);
  }
  E.ntot = off;
  E.ncells = coff;
  if (E.ntot > 0x7fffffffLL) {
    lj_ensemble_destroy(h);
    return LJ_ERR_ARG;
  }
  const int64_t n = E.ntot;
  EnsArgs& A = E.A;
  A.nboxes = nboxes;
  A.ntot = n;
  A.ncells = E.ncells;
  cudaError_t e = cudaSuccess;
  auto M = [&](auto*& p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc((void**)&p, bytes);
  };
  M(A.boxes, sizeof(EnsBox) * nboxes);
  M(A.box_of, sizeof(uint16_t) * n);
  M(A.pos, sizeof(uint4) * n);
  M(A.pos_alt, sizeof(uint4) * n);
  M(A.vel, sizeof(double) * 3 * n);
  M(A.vel_alt, sizeof(double) * 3 * n);
  M(A.frc, sizeof(double) * 3 * n);
  M(A.frc_alt, sizeof(double) * 3 * n);
  M(A.cnt, sizeof(uint32_t) * (E.ncells + 1));
  M(A.cell_start, sizeof(uint32_t) * (E.ncells + 1));
  M(A.cell_of, sizeof(uint32_t) * n);
  M(A.slot, sizeof(uint32_t) * n);
  M(A.key, sizeof(unsigned long long) * n);
  M(A.key2, sizeof(unsigned long long) * n);
  M(A.scan_tot, sizeof(uint32_t) * (E.ncells / 256 + 64));
  M(A.bar, sizeof(unsigned) * 2);
  M(A.status, sizeof(uint32_t));
  M(A.npairs, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    lj_ensemble_destroy(h);
    return LJ_ERR_OOM;
  }
  // host staging: positions (x, y, z, original index within the box), velocities, box ids
  std::vector<uint4> hp(n);
  std::vector<double> hv(3 * n, 0.0);
  std::vector<uint16_t> hbox(n);
  for (int b = 0; b < nboxes; ++b) {
    const EnsBox& B = E.hb[b];
    const int64_t nb = B.n;
    const uint32_t* pb = pos_fp + 3 * B.off;
    for (int64_t k = 0; k < nb; ++k) {
      hp[B.off + k] = make_uint4(pb[k], pb[nb + k], pb[2 * nb + k], (uint32_t)k);
      hbox[B.off + k] = (uint16_t)b;
      if (vel)
        for (int a = 0; a < 3; ++a) hv[a * n + B.off + k] = vel[3 * B.off + a * nb + k];
    }
  }
  cudaStream_t s = E.stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)A.boxes, E.hb.data(), sizeof(EnsBox) * nboxes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)A.box_of, hbox.data(), sizeof(uint16_t) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.pos, hp.data(), sizeof(uint4) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.vel, hv.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.frc, 0, sizeof(double) * 3 * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.npairs, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    lj_ensemble_destroy(h);
    return LJ_ERR_CUDA;
  }
  A.spin_limit = 20000000u;
  A.skip_block = -1;
  *out = h;
  return LJ_OK;
}

// Runs nsteps velocity-Verlet steps of every box in one persistent launch
// (computing the initial forces first when none are current).  use_graph = 1
// captures the launch in a CUDA graph (re-captured when the step count, dt,
// or the tuned shape changes) and replays it.
lj_status lj_ensemble_run(lj_ens* h, double dt, int32_t nsteps, int32_t use_graph) {
  if (!h || !(dt > 0) || nsteps < 0) return LJ_ERR_ARG;
  Ens& E = h->e;
  EnsArgs& A = E.A;
  A.hdtm = 0.5 * dt / E.mass;
  A.nsteps = nsteps;
  A.first_force = E.forces_valid ? 0 : 1;
  for (auto& B : E.hb) B.dtu = dt * 4294967296.0 / B.L;
  cudaStream_t s = E.stream;
  cudaError_t e = cudaMemcpyAsync((void*)A.boxes, E.hb.data(), sizeof(EnsBox) * E.nboxes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int grid = 0;
  if (e == cudaSuccess) e = ens_grid(E, grid);
  if (e != cudaSuccess) {
    E.err = cudaGetErrorString(e);
    return LJ_ERR_CUDA;
  }
  if (use_graph && !E.graph_failed) {
    const bool stale = !E.gexec || E.graph_W != E.W || E.graph_block != E.block || E.graph_steps != nsteps ||
                       E.graph_first != A.first_force || E.graph_dt != dt;
    if (stale) {
      if (E.gexec) cudaGraphExecDestroy(E.gexec);
      if (E.graph) cudaGraphDestroy(E.graph);
      E.gexec = nullptr;
      E.graph = nullptr;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) e = cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), s);
      if (e == cudaSuccess) e = ens_launch(E, grid);
      cudaError_t e2 = cudaStreamEndCapture(s, &E.graph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&E.gexec, E.graph, 0);
      if (e != cudaSuccess) {
        // capture of the cooperative launch not available: launch directly from now on
        E.err = std::string("graph capture failed, direct launches used: ") + cudaGetErrorString(e);
        cudaGetLastError();
        if (E.gexec) cudaGraphExecDestroy(E.gexec);
        if (E.graph) cudaGraphDestroy(E.graph);
        E.gexec = nullptr;
        E.graph = nullptr;
        E.graph_failed = true;
        return lj_ensemble_run(h, dt, nsteps, 0);
      }
      E.graph_W = E.W;
      E.graph_block = E.block;
      E.graph_steps = nsteps;
      E.graph_first = A.first_force;
      E.graph_dt = dt;
    }
    e = cudaGraphLaunch(E.gexec, s);
    E.last_run_graph = true;
  } else {
    E.last_run_graph = false;
    e = cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = ens_launch(E, grid);
  }
  uint32_t st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, A.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    E.err = cudaGetErrorString(e);
    return LJ_ERR_CUDA;
  }
  if (st & 0x80000000u) {  // the state ended in the alternate buffers
    std::swap(A.pos, A.pos_alt);
    std::swap(A.vel, A.vel_alt);
    std::swap(A.frc, A.frc_alt);
    if (E.gexec) {  // the captured graph names the old buffers
      cudaGraphExecDestroy(E.gexec);
      cudaGraphDestroy(E.graph);
      E.gexec = nullptr;
      E.graph = nullptr;
    }
  }
  if (st) cudaMemsetAsync(A.status, 0, sizeof(uint32_t), s);
  if (st & ST_TIMEOUT) {
    E.err = "an ensemble grid barrier timed out";
    E.forces_valid = false;
    return LJ_ERR_TIMEOUT;
  }
  if (st & ST_NONFINITE) {
    E.err = "non-finite force";
    return LJ_ERR_NONFINITE;
  }
  if (st & ST_OOB) {
    E.err = "device index check failed";
    E.forces_valid = false;
    return LJ_ERR_CUDA;
  }
  if (st & ST_CAPACITY) {
    E.err = "a Verlet list outgrew the capacity (lj_ensemble_set_lists with a larger cap); the run stopped mid-step";
    E.forces_valid = false;
    return LJ_ERR_CAPACITY;
  }
  E.forces_valid = true;
  return LJ_OK;
}

namespace {
// The next step of a list-mode run rebuilds the lists (after a state that the
// lists do not describe was put back).
cudaError_t ens_force_rebuild(Ens& E) {
  if (!E.A.vl) return cudaSuccess;
  const uint32_t big = 0x40000000u;
  return cudaMemcpyAsync(E.A.since_build, &big, sizeof(uint32_t), cudaMemcpyHostToDevice, E.stream);
}
}  // namespace

// Chooses the JSPLIT width and block size of the persistent kernel by timing
// `steps` steps of each candidate on a copy of the state (restored after every
// trial).  Writes the choice to *w_out / *block_out (may be NULL).
lj_status lj_ensemble_tune(lj_ens* h, double dt, int32_t steps, int32_t* w_out, int32_t* block_out) {
  if (!h || steps < 1) return LJ_ERR_ARG;
  Ens& E = h->e;
  EnsArgs& A = E.A;
  const int64_t n = E.ntot;
  cudaStream_t s = E.stream;
  uint4* bp = nullptr;
  double *bv = nullptr, *bf = nullptr;
  cudaError_t e = cudaMalloc(&bp, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&bv, sizeof(double) * 3 * n);
  if (e == cudaSuccess) e = cudaMalloc(&bf, sizeof(double) * 3 * n);
  if (e != cudaSuccess) {
    cudaFree(bp);
    cudaFree(bv);
    cudaFree(bf);
    return LJ_ERR_OOM;
  }
  const bool valid0 = E.forces_valid;
  cudaMemcpyAsync(bp, A.pos, sizeof(uint4) * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(bv, A.vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(bf, A.frc, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int Ws[4] = {2, 4, 8, 16};
  const int Bs[3] = {128, 256, 512};
  float best = 3.0e38f;
  int bw = E.W, bb = E.block;
  lj_status st = LJ_OK;
  for (int w : Ws)
    for (int bk : Bs) {
      E.W = w;
      E.block = bk;
      cudaMemcpyAsync(A.pos, bp, sizeof(uint4) * n, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(A.vel, bv, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(A.frc, bf, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
      ens_force_rebuild(E);   // every trial starts with a list build (list mode)
      E.forces_valid = true;  // time steps only
      cudaEventRecord(e0, s);
      st = lj_ensemble_run(h, dt, steps, 0);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      if (st != LJ_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bw = w;
        bb = bk;
      }
    }
  E.W = bw;
  E.block = bb;
  cudaMemcpyAsync(A.pos, bp, sizeof(uint4) * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(A.vel, bv, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(A.frc, bf, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
  ens_force_rebuild(E);
  cudaStreamSynchronize(s);
  E.forces_valid = valid0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(bp);
  cudaFree(bv);
  cudaFree(bf);
  if (w_out) *w_out = bw;
  if (block_out) *block_out = bb;
  return st;
}

lj_status lj_ensemble_set_lists(lj_ens* h, double skin, int32_t rebuild_every, int32_t cap) {
  if (!h || !(skin >= 0) || rebuild_every < 1 || cap < 0) return LJ_ERR_ARG;
  Ens& E = h->e;
  EnsArgs& A = E.A;
  cudaStream_t s = E.stream;
  if (E.gexec) {  // a captured graph holds the old mode and arguments
    cudaGraphExecDestroy(E.gexec);
    cudaGraphDestroy(E.graph);
    E.gexec = nullptr;
    E.graph = nullptr;
  }
  if (skin == 0.0) {  // back to linked cells
    A.vl = 0;
    E.skin = 0.0;
    E.forces_valid = false;
    return LJ_OK;
  }
  const double rl = E.rc + skin;
  int64_t coff = 0;
  double rho_max = 0.0;
  for (auto& B : E.hb) {
    const int nc = (int)std::floor(B.L / rl);
    B.ncv = nc >= 3 ? nc : 1;
    B.cell_off_v = coff;
    coff += (int64_t)B.ncv * B.ncv * B.ncv;
    B.Rl2 = ens_cut2(B.L, rl);
    coarse_band(B.Rl2, &B.rl2p_lo, &B.rl2p_hi);
    const double hs = 0.5 * skin * 4294967296.0 / B.L;
    B.skin2 = (uint64_t)std::min(hs * hs, 1.8e19);
    rho_max = std::max(rho_max, (double)B.n / (B.L * B.L * B.L));
  }
  const int64_t ncv = coff, n = E.ntot;
  if (cap == 0) {  // the densest box's expected list length, with room for fluctuations
    const double m = 4.18879020478639 * rl * rl * rl * rho_max;
    cap = (int32_t)(std::ceil((1.5 * m + 32.0) / 16.0) * 16.0);
  }
  cudaFree(A.nbr);
  cudaFree(A.nnbr);
  cudaFree(A.xb);
  cudaFree((void*)A.cell_box_v);
  A.nbr = nullptr;
  A.nnbr = nullptr;
  A.xb = nullptr;
  A.cell_box_v = nullptr;
  cudaError_t e = cudaSuccess;
  auto M = [&](auto*& p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc((void**)&p, bytes);
  };
  M(A.nbr, sizeof(int32_t) * (size_t)n * cap);
  M(A.nnbr, sizeof(int32_t) * n);
  M(A.xb, sizeof(uint32_t) * 3 * n);
  uint16_t* cbv = nullptr;
  M(cbv, sizeof(uint16_t) * ncv);
  A.cell_box_v = cbv;
  if (!A.since_build) M(A.since_build, sizeof(uint32_t) * 2);
  A.skin_flag = A.since_build ? A.since_build + 1 : nullptr;
  if (ncv > E.ncells) {  // the cell arrays serve both grids
    cudaFree(A.cnt);
    cudaFree(A.cell_start);
    cudaFree(A.scan_tot);
    A.cnt = A.cell_start = A.scan_tot = nullptr;
    M(A.cnt, sizeof(uint32_t) * (ncv + 1));
    M(A.cell_start, sizeof(uint32_t) * (ncv + 1));
    M(A.scan_tot, sizeof(uint32_t) * (ncv / 256 + 64));
    E.ncells = ncv;
  }
  if (e != cudaSuccess) {
    E.err = "out of device memory for the Verlet lists";
    A.vl = 0;
    return LJ_ERR_OOM;
  }
  std::vector<uint16_t> hcb(ncv);
  for (int b = 0; b < E.nboxes; ++b) {
    const EnsBox& B = E.hb[b];
    const int64_t m = (int64_t)B.ncv * B.ncv * B.ncv;
    for (int64_t c = 0; c < m; ++c) hcb[B.cell_off_v + c] = (uint16_t)b;
  }
  const uint32_t words[2] = {0x40000000u, 0u};  // build at the next step; no skin event
  e = cudaMemcpyAsync(cbv, hcb.data(), sizeof(uint16_t) * ncv, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.since_build, words, sizeof(words), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)A.boxes, E.hb.data(), sizeof(EnsBox) * E.nboxes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    E.err = cudaGetErrorString(e);
    return LJ_ERR_CUDA;
  }
  A.vl = 1;
  A.rebuild_every = rebuild_every;
  A.cap = cap;
  A.ncells_v = ncv;
  E.skin = skin;
  E.forces_valid = false;
  return LJ_OK;
}

// Copies the state out (host arrays, boxes concatenated; within box b the
// caller's original order; layout per box: 3 * n_b SoA at offset 3 * off_b).
lj_status lj_ensemble_get(lj_ens* h, uint32_t* pos_fp, double* vel, double* frc) {
  if (!h) return LJ_ERR_ARG;
  Ens& E = h->e;
  const int64_t n = E.ntot;
  std::vector<uint4> hp(n);
  std::vector<double> hv(3 * n), hf(3 * n);
  cudaStream_t s = E.stream;
  cudaError_t e = cudaMemcpyAsync(hp.data(), E.A.pos, sizeof(uint4) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hv.data(), E.A.vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf.data(), E.A.frc, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LJ_ERR_CUDA;
  for (int b = 0; b < E.nboxes; ++b) {
    const EnsBox& B = E.hb[b];
    const int64_t nb = B.n;
    for (int64_t k = 0; k < nb; ++k) {
      const int64_t src = B.off + k;
      const int64_t o = hp[src].w;
      if (pos_fp) {
        pos_fp[3 * B.off + o] = hp[src].x;
        pos_fp[3 * B.off + nb + o] = hp[src].y;
        pos_fp[3 * B.off + 2 * nb + o] = hp[src].z;
      }
      for (int a = 0; a < 3; ++a) {
        if (vel) vel[3 * B.off + a * nb + o] = hv[a * n + src];
        if (frc) frc[3 * B.off + a * nb + o] = hf[a * n + src];
      }
    }
  }
  return LJ_OK;
}

// Test hook for the failure path: a barrier spin bound (iterations of about
// 0.1 us) and a block that leaves the kernel before its first barrier, so the
// other blocks' waits run out and the run reports LJ_ERR_TIMEOUT.
lj_status lj_ensemble_debug(lj_ens* h, uint32_t spin_limit, int32_t skip_block) {
  if (!h) return LJ_ERR_ARG;
  h->e.A.spin_limit = spin_limit ? spin_limit : 20000000u;
  h->e.A.skip_block = skip_block;
  if (h->e.gexec) {
    cudaGraphExecDestroy(h->e.gexec);
    cudaGraphDestroy(h->e.graph);
    h->e.gexec = nullptr;
    h->e.graph = nullptr;
  }
  return LJ_OK;
}

int64_t lj_ensemble_size(const lj_ens* h) { return h ? h->e.ntot : 0; }

const char* lj_ensemble_last_error(const lj_ens* h) { return h ? h->e.err.c_str() : "null ensemble"; }

// Unique in-cutoff pairs summed over all force evaluations since the last
// call (each pair is evaluated from both sides); resets the count.  Synchronises.
int64_t lj_ensemble_pairs(lj_ens* h) {
  if (!h) return -1;
  unsigned long long v = 0;
  if (cudaMemcpyAsync(&v, h->e.A.npairs, sizeof(v), cudaMemcpyDeviceToHost, h->e.stream) != cudaSuccess) return -1;
  if (cudaMemsetAsync(h->e.A.npairs, 0, sizeof(v), h->e.stream) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(h->e.stream) != cudaSuccess) return -1;
  return (int64_t)(v / 2);
}

int32_t lj_ensemble_uses_graph(const lj_ens* h) { return h && h->e.last_run_graph ? 1 : 0; }

void lj_ensemble_destroy(lj_ens* h) {
  if (!h) return;
  Ens& E = h->e;
  cudaStreamSynchronize(E.stream);
  if (E.gexec) cudaGraphExecDestroy(E.gexec);
  if (E.graph) cudaGraphDestroy(E.graph);
  EnsArgs& A = E.A;
  void* ps[] = {(void*)A.boxes, (void*)A.box_of, A.pos, A.pos_alt, A.vel, A.vel_alt, A.frc, A.frc_alt, A.cnt,
                A.cell_start, A.cell_of, A.slot, A.key, A.key2, A.scan_tot, A.bar, A.status, A.npairs,
                A.nbr, A.nnbr, A.xb, (void*)A.cell_box_v, A.since_build};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (E.own_stream) cudaStreamDestroy(E.stream);
  delete h;
}

}  // extern "C"

// k_force_lc.cuh -- Linked Cells force functors: the GPU interaction orders.
//
// The paper's functor receives two particle lists and runs Algorithm 1 (Sec.
// 4.1): fill i registers, fill j registers, ForceKernel, applyNewton3,
// accumulate, storeForces.  Its register-filling patterns (Sec. 4.1.1, Fig. 4)
// decide how many distinct i and j particles share one vector.  On the GPU the
// "vector" is a warp of 32 lanes, and the orders here are:
//
//   IPT_SMEM  (V/1)  one i per lane; the j list staged in shared memory and
//                    broadcast, so one j load serves 32 pairs.  i lists are
//                    "row tiles" of <= 32 consecutive particles of one cell row.
//   IPT_TMA   (V/1)  as IPT_SMEM with the j chunks brought in by bulk
//                    asynchronous copies on an mbarrier double buffer.
//   KI<k>            k i's per lane (row tiles of <= 32 k particles): one
//                    broadcast j serves 32 k pairs (register blocking).
//   ROT32            one i and one j per lane; the 32 j's rotate through the
//                    warp by shuffles (32 x 32 pairs per tile) and, with
//                    Newton-3, each j's force rotates with it.
//   JSPLIT<w>        w lanes per i, striding over the i's own 27-cell
//                    neighbourhood, with a w-lane shuffle reduction of the i
//                    force (1/V for w = 32, 2/V2 for w = 16, V2/2 for w = 2).
//
// Newton-3 (Sec. 4.1.3): with it the i's visit only the forward half shell
// and the j contribution goes to memory by FP64 atomics: V/1-type orders
// reduce it across the warp first (the ReduceSum of the mirrored 1/V store),
// ROT32 carries it with the rotating j, JSPLIT scatters it per pair.
//
// Forces are accumulated per lane in the pair precision R over one tile (one
// particle's pairs of this evaluation) and folded once into FP64 (f2d_exact,
// one FP64 multiply by 24 eps / u; with Newton-3 the unscaled sums are added
// by atomics and scaled once per particle afterwards); energy and virial
// likewise, then reduced in FP64 per block.
#pragma once
#include "ljgb_internal.cuh"

namespace ljgb {

// A contiguous range of j's in cell order.  kind 0: all lanes; kind 1: own
// row of a Newton-3 half shell, lane uses j only if j > i (j < i in the
// backward shell); kind 2: wrap cell of the own row, used only by lanes whose
// i sits in the last cell of the row (the first cell in the backward shell).
struct Seg {
  uint32_t b, e;
  int kind;
};

__device__ __forceinline__ uint32_t cx_of(uint32_t x, uint32_t nc) {
  return (uint32_t)(((unsigned long long)x * nc) >> 32);
}

// Segments of the x-cell set [lo, hi] (as cells, lo may be -1 and hi may be
// nc; the set is taken modulo nc) in row r.  whole = the set covers the row.
__device__ __forceinline__ int row_segments(const uint32_t* __restrict__ cs, int nc, int r, int lo, int hi,
                                            Seg* out) {
  const int64_t base = (int64_t)r * nc;
  if (hi - lo + 1 >= nc) {
    out[0] = {cs[base], cs[base + nc], 0};
    return 1;
  }
  if (lo < 0) {
    out[0] = {cs[base], cs[base + hi + 1], 0};
    out[1] = {cs[base + nc - 1], cs[base + nc], 0};
    return 2;
  }
  if (hi >= nc) {
    out[0] = {cs[base], cs[base + 1], 0};
    out[1] = {cs[base + lo], cs[base + nc], 0};
    return 2;
  }
  out[0] = {cs[base + lo], cs[base + hi + 1], 0};
  return 1;
}

// The j segments of an i-range in row (cy, cz) spanning cells cf..cl.
// Full shell: the 9 rows (dz, dy) in {-1,0,1}^2 with x-cells cf-1..cl+1.
// Half shell (Newton-3), forward: the own row from the first i up to cell
// min(cl+1, nc-1) with j > i (kind 1), the wrap cell 0 when cl = nc-1 (kind 2,
// for the i's of cell nc-1), and the 4 forward rows (0,+1), (+1,-1), (+1,0),
// (+1,+1) with x-cells cf-1..cl+1.  Backward (BWD) is its mirror, the same
// pairs with the roles of the two cells of every pair swapped (the domain
// traversal dimension of Sec. 5.1): the own row from cell max(cf-1, 0) up to
// the tile's last i with j < i (kind 1), the wrap cell nc-1 when cf = 0 (kind 2,
// for the i's of cell 0), and the 4 rows (0,-1), (-1,+1), (-1,0), (-1,-1).
// end_i is one past the tile's last particle.
template <bool HALF, bool BWD = false>
__device__ __forceinline__ int make_segments(const uint32_t* __restrict__ cs, int nc, int row, int cf, int cl,
                                             uint32_t first_i, uint32_t end_i, Seg* segs) {
  const int cy = row % nc, cz = row / nc;
  int ns = 0;
  if (!HALF) {
#pragma unroll 1
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll 1
      for (int dy = -1; dy <= 1; ++dy) {
        const int r = ((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc;
        ns += row_segments(cs, nc, r, cf - 1, cl + 1, segs + ns);
      }
  } else if (!BWD) {
    const int64_t base = (int64_t)row * nc;
    const int last = min(cl + 1, nc - 1);
    segs[ns++] = {first_i, cs[base + last + 1], 1};
    if (cl == nc - 1) segs[ns++] = {cs[base], cs[base + 1], 2};
    const int fw[4][2] = {{0, 1}, {1, -1}, {1, 0}, {1, 1}};
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const int r = ((cz + fw[q][0] + nc) % nc) * nc + (cy + fw[q][1] + nc) % nc;
      ns += row_segments(cs, nc, r, cf - 1, cl + 1, segs + ns);
    }
  } else {
    const int64_t base = (int64_t)row * nc;
    const int lo = max(cf - 1, 0);
    segs[ns++] = {cs[base + lo], end_i, 1};
    if (cf == 0) segs[ns++] = {cs[base + nc - 1], cs[base + nc], 2};
    const int bw[4][2] = {{0, -1}, {-1, 1}, {-1, 0}, {-1, -1}};
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const int r = ((cz + bw[q][0] + nc) % nc) * nc + (cy + bw[q][1] + nc) % nc;
      ns += row_segments(cs, nc, r, cf - 1, cl + 1, segs + ns);
    }
  }
  return ns;
}

// Segments of one particle i (sorted index i, cell (cx, cy, cz)) on sub-cells of
// edge >= r_c / 2: the 5 x 5 x 5 cells around its own (nc >= 5, so that the
// offsets -2..2 name distinct cells on every axis).  Full shell: the 25 rows
// (dz, dy) in {-2..2}^2 with x-cells cx-2..cx+2.  Forward half (Newton-3): the
// offsets after (0, 0, 0) in (dz, dy, dx) order, which hold every pair once:
// the own cell's j > i and the x-cells cx+1, cx+2 of the own row, the rows
// (0, +1), (0, +2), and the 10 rows with dz = +1, +2.  Backward half: the
// mirror (j < i, x-cells cx-2, cx-1, rows (0, -1), (0, -2), dz = -1, -2).
// All segments are of kind 0: the set is this particle's own.
// Segments of the x-cells lo..hi (any integers with hi - lo < nc, taken modulo
// nc) in row r: one or two contiguous pieces, the wrapped one first.
__device__ __forceinline__ int row_segments_mod(const uint32_t* __restrict__ cs, int nc, int r, int lo, int hi,
                                                Seg* out) {
  const int64_t base = (int64_t)r * nc;
  const int len = hi - lo + 1;
  const int a = ((lo % nc) + nc) % nc;
  if (a + len <= nc) {
    out[0] = {cs[base + a], cs[base + a + len], 0};
    return 1;
  }
  out[0] = {cs[base], cs[base + a + len - nc], 0};
  out[1] = {cs[base + a], cs[base + nc], 0};
  return 2;
}

template <bool HALF, bool BWD = false>
__device__ __forceinline__ int make_segments_sub(const uint32_t* __restrict__ cs, int nc, int cx, int cy, int cz,
                                                 uint32_t i, Seg* segs) {
  int ns = 0;
  auto row_of = [&](int dz, int dy) { return ((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc; };
  if (!HALF) {
#pragma unroll 1
    for (int dz = -2; dz <= 2; ++dz)
#pragma unroll 1
      for (int dy = -2; dy <= 2; ++dy) ns += row_segments_mod(cs, nc, row_of(dz, dy), cx - 2, cx + 2, segs + ns);
    return ns;
  }
  const int own = row_of(0, 0);
  const int64_t base = (int64_t)own * nc;
  const int s = BWD ? -1 : 1;
  if (!BWD) {
    segs[ns++] = {i + 1u, cs[base + cx + 1], 0};                       // own cell, j > i
    ns += row_segments_mod(cs, nc, own, cx + 1, cx + 2, segs + ns);         // x-cells cx+1, cx+2 (wrapping)
  } else {
    segs[ns++] = {cs[base + cx], i, 0};                                 // own cell, j < i
    ns += row_segments_mod(cs, nc, own, cx - 2, cx - 1, segs + ns);         // x-cells cx-2, cx-1 (wrapping)
  }
  ns += row_segments_mod(cs, nc, row_of(0, s), cx - 2, cx + 2, segs + ns);
  ns += row_segments_mod(cs, nc, row_of(0, 2 * s), cx - 2, cx + 2, segs + ns);
#pragma unroll 1
  for (int dz = 1; dz <= 2; ++dz)
#pragma unroll 1
    for (int dy = -2; dy <= 2; ++dy) ns += row_segments_mod(cs, nc, row_of(s * dz, dy), cx - 2, cx + 2, segs + ns);
  return ns;
}

// Checks build: a segment outside [0, n] (a corrupt cell start) is emptied
// and reported; in the default build this does nothing.
__device__ __forceinline__ void check_segs(Seg* segs, int ns, uint32_t n, uint32_t* status) {
#ifdef LJGB_CHECKS
  for (int s = 0; s < ns; ++s)
    if (!LJ_IDX_OK(segs[s].b <= segs[s].e && segs[s].e <= n, status)) segs[s].b = segs[s].e = 0u;
#else
  (void)segs;
  (void)ns;
  (void)n;
  (void)status;
#endif
}

template <bool BWD = false>
__device__ __forceinline__ bool seg_ok(int kind, uint32_t j, uint32_t i, uint32_t cxi, int nc) {
  if (kind == 0) return true;
  if (BWD) return kind == 1 ? (j < i) : (cxi == 0u);
  return kind == 1 ? (j > i) : (cxi == (uint32_t)(nc - 1));
}

struct LCArgs {
  const uint4* pos;
  const uint32_t* cs;
  const uint4* tiles;
  const uint32_t* ntiles;   // device count of tiles
  uint32_t* tile_ctr;       // work counter, zero before launch
};

// ---------------------------------------------------------------------------
// IPT_SMEM (K = 1) and KI<K>: warp per row tile of <= 32 K particles, j
// chunks of 32 staged in the warp's shared-memory slot.
// ---------------------------------------------------------------------------
template <typename R, int K, bool N3, bool EV, bool BWD = false>
__global__ void __launch_bounds__(256) k_lc_ipt(LJParams P, LCArgs A, ForceOut out) {
  __shared__ uint4 s_j[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nc = P.nc;
  const uint32_t ntiles = *A.ntiles;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(A.tile_ctr, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntiles) break;
    const uint4 tile = A.tiles[t];
    const int cf = (int)(tile.w & 0xffffu), cl = (int)(tile.w >> 16);
    uint4 pi[K];
    uint32_t ii[K], cxi[K];
    bool vi[K];
    R fx[K], fy[K], fz[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      ii[k] = tile.x + lane + 32 * k;
      vi[k] = ii[k] < tile.y;
      pi[k] = vi[k] ? A.pos[ii[k]] : make_uint4(0, 0, 0, 0);
      cxi[k] = cx_of(pi[k].x, nc);
      fx[k] = fy[k] = fz[k] = (R)0;
    }
    R eu = 0, ew = 0;
    Seg segs[18];
    const int ns = make_segments<N3, BWD>(A.cs, nc, (int)tile.z, cf, cl, tile.x, tile.y, segs);
    check_segs(segs, ns, (uint32_t)P.n, out.status);
#pragma unroll 1
    for (int s = 0; s < ns; ++s) {
      const Seg sg = segs[s];
#pragma unroll 1
      for (uint32_t jb = sg.b; jb < sg.e; jb += 32) {
        const uint32_t m = min(32u, sg.e - jb);
        if (lane < (int)m) s_j[wib][lane] = A.pos[jb + lane];
        __syncwarp();
        R gx = 0, gy = 0, gz = 0;    // Newton-3: this lane's j (index jb + lane)
#pragma unroll 1
        for (uint32_t q = 0; q < m; ++q) {
          const uint4 pj = s_j[wib][q];
          const uint32_t jidx = jb + q;
          R hx = 0, hy = 0, hz = 0;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            if (vi[k] && seg_ok<BWD>(sg.kind, jidx, ii[k], cxi[k], nc)) {
              R af, bf, cf_;
              const R fac = Prec<R>::template pair<EV, true>(mimg(pi[k].x, pj.x), mimg(pi[k].y, pj.y),
                                                       mimg(pi[k].z, pj.z), P, af, bf, cf_, eu, ew, cnt);
              fx[k] += fac * af;
              fy[k] += fac * bf;
              fz[k] += fac * cf_;
              if (N3) {
                hx += fac * af;
                hy += fac * bf;
                hz += fac * cf_;
              }
            }
          }
          if (N3) {
            if (__any_sync(0xffffffffu, (hx != (R)0) | (hy != (R)0) | (hz != (R)0))) {
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                hx += __shfl_xor_sync(0xffffffffu, hx, o);
                hy += __shfl_xor_sync(0xffffffffu, hy, o);
                hz += __shfl_xor_sync(0xffffffffu, hz, o);
              }
              if (lane == (int)q) {
                gx = hx;
                gy = hy;
                gz = hz;
              }
            }
          }
        }
        if (N3 && lane < (int)m) {
          n3_add<R>(out, jb + lane, gx, gy, gz);
        }
        __syncwarp();
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!vi[k]) continue;
      if (N3) {
        n3_add<R>(out, ii[k], -fx[k], -fy[k], -fz[k]);
      } else {
        out.fx[ii[k]] = -P.e24u * Prec<R>::to_d(fx[k]);
        out.fy[ii[k]] = -P.e24u * Prec<R>::to_d(fy[k]);
        out.fz[ii[k]] = -P.e24u * Prec<R>::to_d(fz[k]);
      }
    }
    if (EV) {
      eu_d += Prec<R>::to_d(eu);
      ew_d += Prec<R>::to_d(ew);
    }
  }
  block_flush<R>(eu_d, ew_d, cnt, out, EV);
}

// ---------------------------------------------------------------------------
// IPT_TMA: as IPT_SMEM (K = 1) but each j chunk of up to 64 particles is
// brought into the warp's shared-memory slot by one cp.async.bulk, double
// buffered on two mbarriers.  Waits are bounded: a wait that gives up sets
// ST_TIMEOUT, waits (bounded) for its copy and leaves the tile loop.
// ---------------------------------------------------------------------------
constexpr int TMA_CH = 64;
constexpr int TMA_WARPS = 4;
constexpr uint32_t TMA_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for the phase with the given parity; true when it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < TMA_SPIN_LIMIT; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename R, bool N3, bool EV, bool BWD = false>
__global__ void __launch_bounds__(TMA_WARPS * 32) k_lc_tma(LJParams P, LCArgs A, ForceOut out) {
  __shared__ __align__(128) uint4 s_j[TMA_WARPS][2][TMA_CH];
  __shared__ __align__(8) uint64_t s_bar[TMA_WARPS][2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nc = P.nc;
  if (lane == 0) {
    mbar_init(&s_bar[wib][0], 1);
    mbar_init(&s_bar[wib][1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t phase[2] = {0u, 0u};
  const uint32_t ntiles = *A.ntiles;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  bool failed = false;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(A.tile_ctr, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntiles || failed) break;
    const uint4 tile = A.tiles[t];
    const int cf = (int)(tile.w & 0xffffu), cl = (int)(tile.w >> 16);
    const uint32_t ii = tile.x + lane;
    const bool vi = ii < tile.y;
    const uint4 pi = vi ? A.pos[ii] : make_uint4(0, 0, 0, 0);
    const uint32_t cxi = cx_of(pi.x, nc);
    R fx = 0, fy = 0, fz = 0, eu = 0, ew = 0;
    Seg segs[18];
    const int ns = make_segments<N3, BWD>(A.cs, nc, (int)tile.z, cf, cl, tile.x, tile.y, segs);
    check_segs(segs, ns, (uint32_t)P.n, out.status);
    // flatten (segment, offset) into chunks; issue chunk c+1 while computing c
    int s_cur = 0;
    uint32_t o_cur = 0;
    while (s_cur < ns && segs[s_cur].b >= segs[s_cur].e) ++s_cur;
    auto issue = [&](int s, uint32_t o, int buf) {
      const uint32_t m = min((uint32_t)TMA_CH, segs[s].e - segs[s].b - o);
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&s_bar[wib][buf], m * 16u);
        bulk_g2s(&s_j[wib][buf][0], A.pos + segs[s].b + o, m * 16u, &s_bar[wib][buf]);
      }
    };
    int buf = 0;
    if (s_cur < ns) issue(s_cur, 0, 0);
    while (s_cur < ns) {
      const Seg sg = segs[s_cur];
      const uint32_t m = min((uint32_t)TMA_CH, sg.e - sg.b - o_cur);
      const uint32_t jb = sg.b + o_cur;
      // next chunk
      int s_nx = s_cur;
      uint32_t o_nx = o_cur + m;
      if (o_nx >= sg.e - sg.b) {
        ++s_nx;
        o_nx = 0;
        while (s_nx < ns && segs[s_nx].b >= segs[s_nx].e) ++s_nx;
      }
      if (s_nx < ns) issue(s_nx, o_nx, buf ^ 1);
      const bool ok_wait = mbar_wait(&s_bar[wib][buf], phase[buf]);
      phase[buf] ^= 1u;
      if (!__all_sync(0xffffffffu, ok_wait)) {
        if (lane == 0) atomicOr(out.status, ST_TIMEOUT);
        // bounded wait for the copy still in flight on the other buffer
        if (s_nx < ns) mbar_wait(&s_bar[wib][buf ^ 1], phase[buf ^ 1]);
        failed = true;
        break;
      }
      R gx = 0, gy = 0, gz = 0;
#pragma unroll 1
      for (uint32_t q = 0; q < m; ++q) {
        const uint4 pj = s_j[wib][buf][q];
        const uint32_t jidx = jb + q;
        R hx = 0, hy = 0, hz = 0;
        if (vi && seg_ok<BWD>(sg.kind, jidx, ii, cxi, nc)) {
          R af, bf, cf_;
          const R fac = Prec<R>::template pair<EV, true>(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), P, af,
                                                   bf, cf_, eu, ew, cnt);
          fx += fac * af;
          fy += fac * bf;
          fz += fac * cf_;
          hx = fac * af;
          hy = fac * bf;
          hz = fac * cf_;
        }
        if (N3) {
          if (__any_sync(0xffffffffu, (hx != (R)0) | (hy != (R)0) | (hz != (R)0))) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              hx += __shfl_xor_sync(0xffffffffu, hx, o);
              hy += __shfl_xor_sync(0xffffffffu, hy, o);
              hz += __shfl_xor_sync(0xffffffffu, hz, o);
            }
            if (lane == (int)(q & 31u)) {
              gx += hx;
              gy += hy;
              gz += hz;
            }
          }
          if ((q & 31u) == 31u || q + 1 == m) {
            const uint32_t qb = q & ~31u;
            if (lane <= (int)(q - qb)) {
              n3_add<R>(out, jb + qb + lane, gx, gy, gz);
            }
            gx = gy = gz = 0;
          }
        }
      }
      __syncwarp();
      s_cur = s_nx;
      o_cur = o_nx;
      buf ^= 1;
    }
    if (failed) break;
    if (vi) {
      if (N3) {
        n3_add<R>(out, ii, -fx, -fy, -fz);
      } else {
        out.fx[ii] = -P.e24u * Prec<R>::to_d(fx);
        out.fy[ii] = -P.e24u * Prec<R>::to_d(fy);
        out.fz[ii] = -P.e24u * Prec<R>::to_d(fz);
      }
    }
    if (EV) {
      eu_d += Prec<R>::to_d(eu);
      ew_d += Prec<R>::to_d(ew);
    }
  }
  block_flush<R>(eu_d, ew_d, cnt, out, EV);
}

// ---------------------------------------------------------------------------
// ROT32: warp per row tile of <= 32 i's; each j chunk of <= 32 sits one per
// lane and rotates by one lane per step (32 steps = the full 32 x 32 tile).
// ---------------------------------------------------------------------------
template <typename R, bool N3, bool EV, bool BWD = false>
__global__ void __launch_bounds__(256) k_lc_rot(LJParams P, LCArgs A, ForceOut out) {
  const int lane = threadIdx.x & 31;
  const int nc = P.nc;
  const uint32_t ntiles = *A.ntiles;
  const int nxt = (lane + 1) & 31;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(A.tile_ctr, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntiles) break;
    const uint4 tile = A.tiles[t];
    const int cf = (int)(tile.w & 0xffffu), cl = (int)(tile.w >> 16);
    const uint32_t ii = tile.x + lane;
    const bool vi = ii < tile.y;
    const uint4 pi = vi ? A.pos[ii] : make_uint4(0, 0, 0, 0);
    const uint32_t cxi = cx_of(pi.x, nc);
    R fx = 0, fy = 0, fz = 0, eu = 0, ew = 0;
    Seg segs[18];
    const int ns = make_segments<N3, BWD>(A.cs, nc, (int)tile.z, cf, cl, tile.x, tile.y, segs);
    check_segs(segs, ns, (uint32_t)P.n, out.status);
#pragma unroll 1
    for (int s = 0; s < ns; ++s) {
      const Seg sg = segs[s];
#pragma unroll 1
      for (uint32_t jb = sg.b; jb < sg.e; jb += 32) {
        const uint32_t m = min(32u, sg.e - jb);
        uint4 pj = (lane < (int)m) ? A.pos[jb + lane] : make_uint4(0, 0, 0, 0);
        R gx = 0, gy = 0, gz = 0;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const uint32_t src = (uint32_t)((lane + r) & 31);
          if (vi && src < m && seg_ok<BWD>(sg.kind, jb + src, ii, cxi, nc)) {
            R af, bf, cf_;
            const R fac = Prec<R>::template pair<EV, true>(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), P,
                                                     af, bf, cf_, eu, ew, cnt);
            fx += fac * af;
            fy += fac * bf;
            fz += fac * cf_;
            if (N3) {
              gx += fac * af;
              gy += fac * bf;
              gz += fac * cf_;
            }
          }
          pj.x = __shfl_sync(0xffffffffu, pj.x, nxt);
          pj.y = __shfl_sync(0xffffffffu, pj.y, nxt);
          pj.z = __shfl_sync(0xffffffffu, pj.z, nxt);
          if (N3) {
            gx = __shfl_sync(0xffffffffu, gx, nxt);
            gy = __shfl_sync(0xffffffffu, gy, nxt);
            gz = __shfl_sync(0xffffffffu, gz, nxt);
          }
        }
        if (N3 && lane < (int)m) {
          n3_add<R>(out, jb + lane, gx, gy, gz);
        }
      }
    }
    if (vi) {
      if (N3) {
        n3_add<R>(out, ii, -fx, -fy, -fz);
      } else {
        out.fx[ii] = -P.e24u * Prec<R>::to_d(fx);
        out.fy[ii] = -P.e24u * Prec<R>::to_d(fy);
        out.fz[ii] = -P.e24u * Prec<R>::to_d(fz);
      }
    }
    if (EV) {
      eu_d += Prec<R>::to_d(eu);
      ew_d += Prec<R>::to_d(ew);
    }
  }
  block_flush<R>(eu_d, ew_d, cnt, out, EV);
}

// ---------------------------------------------------------------------------
// JSPLIT<W>: groups of W lanes per i (32/W i's per warp, consecutive in cell
// order); every group walks its own i's 27-cell (or half-shell) segments.
// ---------------------------------------------------------------------------
// REACH = 2: sub-cells of edge >= r_c / 2, each i walking its own 5 x 5 x 5
// cells (make_segments_sub).
template <typename R, int W, bool N3, bool EV, bool BWD = false, int REACH = 1>
__global__ void __launch_bounds__(256) k_lc_jsplit(LJParams P, const uint4* __restrict__ pos,
                                                   const uint32_t* __restrict__ cs, ForceOut out) {
  constexpr int G = 32 / W;
  const int lane = threadIdx.x & 31, g = lane / W, sub = lane % W;
  const int nc = P.nc;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  for (; w * G < P.n; w += nwarps) {
    const uint32_t ii = (uint32_t)(w * G + g);
    const bool vi = ii < (uint32_t)P.n;
    const uint4 pi = vi ? pos[ii] : make_uint4(0, 0, 0, 0);
    const int cx = (int)cx_of(pi.x, nc), cy = (int)cx_of(pi.y, nc), cz = (int)cx_of(pi.z, nc);
    Seg segs[REACH == 2 ? 52 : 18];
    int ns = 0;
    if (vi) {
      if (REACH == 2) ns = make_segments_sub<N3, BWD>(cs, nc, cx, cy, cz, ii, segs);
      else ns = make_segments<N3, BWD>(cs, nc, cz * nc + cy, cx, cx, ii, ii, segs);
    }
    check_segs(segs, ns, (uint32_t)P.n, out.status);
    R fx = 0, fy = 0, fz = 0, eu = 0, ew = 0;
    if (REACH == 2) {
      // the 25-50 short segments (about 7 particles each) as one packed
      // stream: lane sub takes positions sub, sub + W, ... with a running
      // segment pointer, so lanes do not idle at every segment's end
      uint32_t total = 0;
      for (int s = 0; s < ns; ++s) total += segs[s].e - segs[s].b;
      const uint32_t tmax = __reduce_max_sync(0xffffffffu, (total + W - 1) / W);
      int sl = 0;
      uint32_t base = 0;
#pragma unroll 1
      for (uint32_t q = 0; q < tmax; ++q) {
        const uint32_t p = q * W + sub;
        while (sl < ns && p >= base + (segs[sl].e - segs[sl].b)) {
          base += segs[sl].e - segs[sl].b;
          ++sl;
        }
        if (p < total) {
          const uint32_t j = segs[sl].b + (p - base);
          const uint4 pj = pos[j];
          R af, bf, cf_;
          const R fac = Prec<R>::template pair<EV, true>(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), P, af,
                                                   bf, cf_, eu, ew, cnt);
          fx += fac * af;
          fy += fac * bf;
          fz += fac * cf_;
          if (N3) {
            n3_add<R>(out, j, fac * af, fac * bf, fac * cf_);
          }
        }
      }
    }
    const int nsmax = REACH == 2 ? 0 : (int)__reduce_max_sync(0xffffffffu, (unsigned)ns);
#pragma unroll 1
    for (int s = 0; s < nsmax; ++s) {
      const Seg sg = (s < ns) ? segs[s] : Seg{0u, 0u, 0};
      const uint32_t len = sg.e - sg.b;
      const uint32_t trips = (len + W - 1) / W;
      const uint32_t tmax = __reduce_max_sync(0xffffffffu, trips);
#pragma unroll 1
      for (uint32_t q = 0; q < tmax; ++q) {
        const uint32_t j = sg.b + q * W + sub;
        if (j < sg.e && seg_ok<BWD>(sg.kind, j, ii, (uint32_t)cx, nc)) {
          const uint4 pj = pos[j];
          R af, bf, cf_;
          const R fac = Prec<R>::template pair<EV, true>(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), P, af,
                                                   bf, cf_, eu, ew, cnt);
          fx += fac * af;
          fy += fac * bf;
          fz += fac * cf_;
          if (N3) {
            n3_add<R>(out, j, fac * af, fac * bf, fac * cf_);
          }
        }
      }
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
      fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (vi && sub == 0) {
      if (N3) {
        n3_add<R>(out, ii, -fx, -fy, -fz);
      } else {
        out.fx[ii] = -P.e24u * Prec<R>::to_d(fx);
        out.fy[ii] = -P.e24u * Prec<R>::to_d(fy);
        out.fz[ii] = -P.e24u * Prec<R>::to_d(fz);
      }
    }
    if (EV) {
      eu_d += Prec<R>::to_d(eu);
      ew_d += Prec<R>::to_d(ew);
    }
  }
  block_flush<R>(eu_d, ew_d, cnt, out, EV);
}

}  // namespace ljgb

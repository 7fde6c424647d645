// k_build.cuh -- the per-tile scan of the Verlet-list builder (Sec. 2.1.1),
// shared by the single-box builder (k_verlet.cu) and the batched ensemble
// (k_ensemble.cu).
//
// A tile is <= 32 consecutive particles of one cell, so its candidates are
// exactly the 27 cells around it (or, in a box of fewer than 3 cells per axis,
// the whole box).  The warp holds 32 j's, one per lane, and takes the tile's
// i's in turn; survivors of the exact integer rule 0 < R^2 <= floor((r_l/u)^2)
// (half lists: j > i) are compacted with a warp ballot, so every i receives its
// j's in the scan order of rows (dz, dy) and ascending index.  A coarse float
// screen settles every candidate except those in a thin band around r_l,
// which get the exact 64-bit test: each particle's coordinates floor(x / 512)
// are exact floats, the segment's periodic image is one addition per loaded j,
// and a test is three exact subtractions and an FMA sum (the bound of
// coarse_r2, since floor(x_j/512) - floor(x_i/512) is within 1 of
// (x_j - x_i)/512).
#pragma once
#include "ljgb_internal.cuh"

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

// Membership of lane j in particle i's list (the coarse screen, and the
// exact integer test in the band around r_l).
template <bool HALF>
__device__ __forceinline__ bool bv_in(const float4& ci, const uint4* s_iq, float jx, float jy, float jz,
                                      const uint4& pj, int j, uint32_t i, uint64_t Rl2, float rl2p_lo,
                                      float rl2p_hi) {
  const float dx = jx - ci.x, dy = jy - ci.y, dz = jz - ci.z;  // exact (integers < 2^24)
  const float r2p = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  bool in = (HALF ? j > (int)i : j != (int)i) && r2p <= rl2p_hi;
  if (in && r2p >= rl2p_lo) {
    const uint4 pi = *s_iq;
    in = in_cut_exact(mimg(pi.x, pj.x), mimg(pi.y, pj.y), mimg(pi.z, pj.z), Rl2);
  }
  return in;
}

// The scan of one tile: particles first .. first + ni - 1 (ni <= 32), whose
// positions and coarse coordinates this warp has put in s_i / s_c, against the
// segments.  Chunks of 32 j's are packed across segment boundaries (each lane
// carries its own periodic shift), so a tile's ~27 cells take ceil(total / 32)
// chunks; lanes past the end sit at coarse -1e30 with j = -1 and are never
// accepted.  A tile whose neighbourhood has a whole-row segment (n_c = 3, or a
// whole box) takes the per-segment path with the integer test for those rows.
// Returns, in lane q, the list length of particle first + q (entries beyond
// cap are counted, not stored).
template <bool HALF, bool COLMAJOR>
__device__ __forceinline__ uint32_t bv_tile(const uint4* __restrict__ pos, const BSeg* segs, int ns, uint32_t first,
                                            int ni, const uint4* s_i, const float4* s_c, int n, int cap,
                                            uint64_t Rl2, float rl2p_lo, float rl2p_hi, int32_t* __restrict__ nbr) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t my_cnt = 0;  // lane q counts the list of the tile's q-th particle
  __syncwarp();
  bool mixed = false;
  uint32_t total = 0;
  for (int s = 0; s < ns; ++s) {
    mixed |= segs[s].mixed != 0;
    total += segs[s].e - segs[s].b;
  }
  if (!mixed) {
    // Chunks of 32 JPL: each lane holds JPL j's (positions c0 + 32 u + lane of
    // the packed neighbourhood), so that an i's running count and store
    // address serve 32 JPL tests.  The u-th 32 j's survivors are stored before
    // the (u+1)-th's: the order is that of 32-wide chunks.
    int sl = 0;
    uint32_t off = lane;  // this lane's position within segment sl
    auto load_j = [&](int& j, uint4& pj, float& jx, float& jy, float& jz) {
      while (sl < ns && off >= segs[sl].e - segs[sl].b) {
        off -= segs[sl].e - segs[sl].b;
        ++sl;
      }
      j = -1;
      pj = make_uint4(0, 0, 0, 0);
      jx = jy = jz = -1e30f;
      if (sl < ns) {
        const BSeg& sg = segs[sl];
        j = (int)(sg.b + off);
        pj = pos[j];
        jx = coarse_coord(pj.x) + sg.sx;
        jy = coarse_coord(pj.y) + sg.sy;
        jz = coarse_coord(pj.z) + sg.sz;
      }
      off += 32;
    };
    constexpr int JPL = 4;  // j's per lane
#pragma unroll 1
    for (uint32_t c0 = 0; c0 < total; c0 += 32 * JPL) {
      int jv[JPL];
      uint4 pv[JPL];
      float xv[JPL], yv[JPL], zv[JPL];
#pragma unroll
      for (int u = 0; u < JPL; ++u) load_j(jv[u], pv[u], xv[u], yv[u], zv[u]);
#pragma unroll 2
      for (int q = 0; q < ni; ++q) {
        const float4 ci = s_c[q];
        const uint32_t i = first + q;
        unsigned m[JPL];
#pragma unroll
        for (int u = 0; u < JPL; ++u)
          m[u] = __ballot_sync(0xffffffffu, bv_in<HALF>(ci, s_i + q, xv[u], yv[u], zv[u], pv[u], jv[u], i, Rl2,
                                                          rl2p_lo, rl2p_hi));
        uint32_t k = __shfl_sync(0xffffffffu, my_cnt, q);
#pragma unroll
        for (int u = 0; u < JPL; ++u) {
          if ((m[u] >> lane) & 1u) {
            const uint32_t kk = k + __popc(m[u] & lt);
            if (kk < (uint32_t)cap) {
              if (COLMAJOR) nbr[(int64_t)kk * n + i] = jv[u];
              else nbr[(int64_t)i * cap + kk] = jv[u];
            }
          }
          k += (uint32_t)__popc(m[u]);
        }
        if (lane == q) my_cnt = k;
      }
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
            bv_test<HALF, COLMAJOR, true>(s_c[q], s_i[q], jx, jy, jz, pj, j, first + q, q, lane, lt,
                                          n, cap, Rl2, rl2p_lo, rl2p_hi, nbr, my_cnt);
          else
            bv_test<HALF, COLMAJOR, false>(s_c[q], s_i[q], jx, jy, jz, pj, j, first + q, q, lane, lt,
                                           n, cap, Rl2, rl2p_lo, rl2p_hi, nbr, my_cnt);
        }
      }
    }
  }
  return my_cnt;
}

}  // namespace ljgb

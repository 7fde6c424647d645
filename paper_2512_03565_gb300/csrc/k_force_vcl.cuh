// k_force_vcl.cuh -- force kernels over Verlet cluster lists.
//
// The functor of the cluster container takes the base (i) cluster as its
// first list and the neighbour (j) clusters as its second (Sec. 2.3), and
// the paper finds that the interaction order should be aligned to the
// cluster size (Sec. 5.1).  On a 32-lane warp the two GPU orders are:
//
//   CL_TILE   lane = (i, j-slot): the M i's of the base cluster across lanes,
//             32/M j-slots (so several neighbour clusters per pass for M = 4,
//             half a cluster for M = 8; 30 lanes for M = 6).  The base
//             cluster is loaded once; each pass loads one packed list word
//             and one j position per lane (both broadcast within the lane's
//             j-slot group).  The i force is reduced over the j-slots at the
//             end of the list; with Newton-3 the j force of each pass is
//             reduced over the M i lanes and added by one FP64 atomic (the
//             unscaled sum; the factor 24 eps / u follows per particle).
//   CL_JLANE  lane = j-slot (32 j's per pass, from 32/M neighbour clusters);
//             the M i's are held in every lane's registers and visited in
//             turn.  The j force stays in its lane (Newton-3: one atomic per j
//             and pass, no shuffle); each of the M i forces is reduced over
//             the warp at the end of the list.
//
// The pair arithmetic is the same exact-cutoff kernel as the other
// containers, evaluated branch-free (most candidates of a cluster pair are
// outside the cutoff, and the warp would take the branch anyway).  A lane's
// pair enters only when its bit of the entry's member mask is set (the pair
// lies within r_l; the mask also leaves out slots beyond a cluster's size and
// the pairs of the base cluster with itself that a list does not own); the
// others enter as a zero difference, which the rule 0 < R^2 excludes.
#pragma once
#include "ljgb_internal.cuh"

namespace ljgb {

struct VclArgs {
  const uint4* pos;
  const uint32_t* cl_start;
  const uint32_t* nbr;  // [ncl][cap], (begin << 3) | (size - 1)
  const uint64_t* mask; // [ncl][cap], member pairs within r_l: bit a * M + b
  const int32_t* nn;
  int64_t ncl;
  int cap;
};

// Without Newton-3 a particle's force is stored once, scaled by -24 eps / u.
// With it, the unscaled sums are added through n3_add (+ for a j, - for an
// i) and scaled once per particle afterwards.
template <typename R>
__device__ __forceinline__ void store_force(const ForceOut& out, uint32_t i, R fx, R fy, R fz, double s) {
  out.fx[i] = s * Prec<R>::to_d(fx);
  out.fy[i] = s * Prec<R>::to_d(fy);
  out.fz[i] = s * Prec<R>::to_d(fz);
}

template <typename R, int M, bool N3, bool EV>
__global__ void __launch_bounds__(256) k_vcl_tile(LJParams P, VclArgs A, ForceOut out) {
  constexpr int JP = 32 / M;  // j-slots per pass
  constexpr int USED = JP * M;
  const int lane = threadIdx.x & 31;
  const int ii = lane % M, js = lane / M;
  const bool act = lane < USED;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < A.ncl; I += nwarps) {
    const uint32_t ib = A.cl_start[I], ie = A.cl_start[I + 1];
    const uint32_t i = ib + (uint32_t)ii;
    const bool vi = act && i < ie;
    const uint4 pi = A.pos[vi ? i : ib];
    const uint32_t slots = (uint32_t)A.nn[I] * (uint32_t)M;
    const uint32_t* __restrict__ row = A.nbr + I * A.cap;
    const uint64_t* __restrict__ mrow = A.mask + I * A.cap;
    R fx = 0, fy = 0, fz = 0, eu = 0, ew = 0;
#pragma unroll 2
    for (uint32_t q0 = 0; q0 < slots; q0 += JP) {
      const uint32_t q = q0 + (uint32_t)js;
      const bool vq = act && q < slots;
      uint32_t ent = vq ? row[q / M] : ib << 3;  // a slot past the list reads the base cluster
      const uint64_t mk = vq ? mrow[q / M] : 0ull;
      if (!LJ_IDX_OK((ent >> 3) + (ent & 7u) < (uint32_t)P.n, out.status)) ent = ib << 3;
      const uint32_t jb = ent >> 3, jj = q % M;
      const bool vj = vq && jj <= (ent & 7u);
      const uint32_t j = jb + jj;
      const uint4 pj = A.pos[vj ? j : jb];
      const bool ok = vi && vj && ((mk >> ((uint32_t)ii * M + jj)) & 1ull);
      const int a = ok ? mimg(pi.x, pj.x) : 0, b = ok ? mimg(pi.y, pj.y) : 0, c = ok ? mimg(pi.z, pj.z) : 0;
      R af, bf, cf;
      const R fac = Prec<R>::template pair<EV, false, true>(a, b, c, P, af, bf, cf, eu, ew, cnt);
      const R gx = fac * af, gy = fac * bf, gz = fac * cf;
      fx += gx;
      fy += gy;
      fz += gz;
      if (N3) {  // the j force: sum over the M i lanes of this j-slot
        R hx = gx, hy = gy, hz = gz;
#pragma unroll
        for (int o = 1; o < M; o <<= 1) {
          const R tx = __shfl_down_sync(0xffffffffu, hx, o);
          const R ty = __shfl_down_sync(0xffffffffu, hy, o);
          const R tz = __shfl_down_sync(0xffffffffu, hz, o);
          if (ii + o < M) {
            hx += tx;
            hy += ty;
            hz += tz;
          }
        }
        if (ii == 0 && vj) n3_add<R>(out, j, hx, hy, hz);
      }
    }
    // the i force: sum over the j-slots
    if ((M & (M - 1)) == 0) {
#pragma unroll
      for (int o = M; o < 32; o <<= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
      }
    } else {
      R sx = 0, sy = 0, sz = 0;
#pragma unroll
      for (int s = 0; s < JP; ++s) {
        sx += __shfl_sync(0xffffffffu, fx, ii + s * M);
        sy += __shfl_sync(0xffffffffu, fy, ii + s * M);
        sz += __shfl_sync(0xffffffffu, fz, ii + s * M);
      }
      fx = sx;
      fy = sy;
      fz = sz;
    }
    if (vi && js == 0) {
      if (N3) n3_add<R>(out, i, -fx, -fy, -fz);
      else store_force<R>(out, i, fx, fy, fz, -P.e24u);
    }
    if (EV) {
      eu_d += Prec<R>::to_d(eu);
      ew_d += Prec<R>::to_d(ew);
    }
  }
  block_flush<R>(eu_d, ew_d, cnt, out, EV);
}

template <typename R, int M, bool N3, bool EV>
__global__ void __launch_bounds__(256) k_vcl_jlane(LJParams P, VclArgs A, ForceOut out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < A.ncl; I += nwarps) {
    const uint32_t ib = A.cl_start[I], ie = A.cl_start[I + 1];
    const uint32_t ni = ie - ib;
    uint4 pi[M];
#pragma unroll
    for (int k = 0; k < M; ++k) pi[k] = A.pos[ib + ((uint32_t)k < ni ? (uint32_t)k : 0u)];
    R fi[M][3];
#pragma unroll
    for (int k = 0; k < M; ++k) fi[k][0] = fi[k][1] = fi[k][2] = (R)0;
    const uint32_t slots = (uint32_t)A.nn[I] * (uint32_t)M;
    const uint32_t* __restrict__ row = A.nbr + I * A.cap;
    const uint64_t* __restrict__ mrow = A.mask + I * A.cap;
    R eu = 0, ew = 0;
#pragma unroll 1
    for (uint32_t q0 = 0; q0 < slots; q0 += 32) {
      const uint32_t q = q0 + (uint32_t)lane;
      const bool vq = q < slots;
      uint32_t ent = vq ? row[q / M] : ib << 3;  // a slot past the list reads the base cluster
      const uint64_t mk = vq ? mrow[q / M] : 0ull;
      if (!LJ_IDX_OK((ent >> 3) + (ent & 7u) < (uint32_t)P.n, out.status)) ent = ib << 3;
      const uint32_t jb = ent >> 3, jj = q % M;
      const bool vj = vq && jj <= (ent & 7u);
      const uint32_t j = jb + jj;
      const uint4 pj = A.pos[vj ? j : jb];
      const uint64_t mj = vj ? mk >> jj : 0ull;  // bit k * M: this lane's pair with the k-th i
      R gx = 0, gy = 0, gz = 0;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const bool ok = (uint32_t)k < ni && ((mj >> (k * M)) & 1ull);
        const int a = ok ? mimg(pi[k].x, pj.x) : 0, b = ok ? mimg(pi[k].y, pj.y) : 0,
                  c = ok ? mimg(pi[k].z, pj.z) : 0;
        R af, bf, cf;
        const R fac = Prec<R>::template pair<EV, false, true>(a, b, c, P, af, bf, cf, eu, ew, cnt);
        fi[k][0] += fac * af;
        fi[k][1] += fac * bf;
        fi[k][2] += fac * cf;
        if (N3) {
          gx += fac * af;
          gy += fac * bf;
          gz += fac * cf;
        }
      }
      if (N3 && vj) n3_add<R>(out, j, gx, gy, gz);
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
      R sx = fi[k][0], sy = fi[k][1], sz = fi[k][2];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
      }
      if (lane == 0 && (uint32_t)k < ni) {
        if (N3) n3_add<R>(out, ib + k, -sx, -sy, -sz);
        else store_force<R>(out, ib + k, sx, sy, sz, -P.e24u);
      }
    }
    if (EV) {
      eu_d += Prec<R>::to_d(eu);
      ew_d += Prec<R>::to_d(ew);
    }
  }
  block_flush<R>(eu_d, ew_d, cnt, out, EV);
}

template <typename R, bool N3, bool EV>
cudaError_t vcl_launch(Ctx& c, const lj_config& cfg, ForceOut out) {
  VclArgs A{c.pos, c.cl_start, c.vcl_nbr, c.vcl_mask, c.vcl_nn, c.vcl_ncl, c.vcl_cap};
  const int64_t threads = std::max<int64_t>(32, c.vcl_ncl * 32);
  const unsigned g = (unsigned)std::min<int64_t>((threads + 255) / 256, 152 * 16);
  const bool tile = cfg.order == LJ_ORD_CL_TILE;
  switch (cfg.param) {
    case 4:
      if (tile) k_vcl_tile<R, 4, N3, EV><<<g, 256, 0, c.stream>>>(c.P, A, out);
      else k_vcl_jlane<R, 4, N3, EV><<<g, 256, 0, c.stream>>>(c.P, A, out);
      break;
    case 6:
      if (tile) k_vcl_tile<R, 6, N3, EV><<<g, 256, 0, c.stream>>>(c.P, A, out);
      else k_vcl_jlane<R, 6, N3, EV><<<g, 256, 0, c.stream>>>(c.P, A, out);
      break;
    case 8:
      if (tile) k_vcl_tile<R, 8, N3, EV><<<g, 256, 0, c.stream>>>(c.P, A, out);
      else k_vcl_jlane<R, 8, N3, EV><<<g, 256, 0, c.stream>>>(c.P, A, out);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t force_vcl_t(Ctx& c, const lj_config& cfg, bool ev) {
  ForceOut out{c.frc, c.frc + c.n, c.frc + 2 * c.n, c.ev, c.npairs, c.status};
  if (cfg.newton3 == LJ_N3_ATOMIC) {
    cudaError_t e = n3_begin(c, out, sizeof(R) == 4);
    if (e != cudaSuccess) return e;
    return ev ? vcl_launch<R, true, true>(c, cfg, out) : vcl_launch<R, true, false>(c, cfg, out);
  }
  return ev ? vcl_launch<R, false, true>(c, cfg, out) : vcl_launch<R, false, false>(c, cfg, out);
}

}  // namespace ljgb

// k_force_vl.cuh -- Verlet-list force functors (Sec. 2.1.1, Verlet lists).
//
// The paper leaves Verlet lists out of its pattern study because gathering
// j's from a list defeats CPU SIMD loads (Sec. 2.1.1); on the GPU a gather
// per lane is the natural access, and two orders apply:
//   VL_IPT     one i per lane (V/1 over the list): column-major lists
//              nbr[k * n + i], so the k-th entries of 32 i's are one
//              coalesced load.
//   JSPLIT<w>  w lanes per i striding over its row-major list nbr[i * cap + k]
//              with a w-lane shuffle reduction (1/V for w = 32, V2/2 for w = 2);
//              for w = 2 each lane takes two adjacent entries per load.
// With Newton-3 the lists are half lists (j after i in cell order) and every
// pair's j contribution is scattered with FP64 atomics; the two-pass variant
// writes each pair's contribution to its list slot and a second kernel sums a
// particle's slots through the reverse index (see k_verlet.cu) in a fixed order.
#pragma once
#include "ljgb_internal.cuh"

namespace ljgb {

struct VLArgs {
  const uint4* pos;
  const int32_t* nbr;
  const int16_t* nbr16;  // 16-bit entries (j - i wrapped modulo n), same layout; used when non-null
  const int32_t* nnbr;
  int cap;
  void* slot;      // two-pass: per-entry j contributions, R[3][cap * n] (column-major slots)
  uint32_t* status;
};

// Entry k of a list: the 32-bit index, or i plus the 16-bit wrapped
// difference.  List entries are read once per evaluation: streaming loads keep
// them from displacing the positions in L2.
template <bool I16>
__device__ __forceinline__ int vl_entry(const VLArgs& A, int64_t e, int64_t i, int64_t n) {
  if (I16) {
    int64_t j = i + (int64_t)__ldcs(A.nbr16 + e);
    j += (j < 0) ? n : 0;
    j -= (j >= n) ? n : 0;
    return (int)j;
  }
  const int j = __ldcs(A.nbr + e);
  return LJ_IDX_OK((unsigned)j < (unsigned)n, A.status) ? j : (int)i;  // checks build: self, no pair
}

// Stores the FP64 force of particle i; a non-finite component sets
// ST_NONFINITE (tested on the exponent bits, off GB300's narrow FP64 pipe).
__device__ __forceinline__ void vl_store(const ForceOut& out, uint32_t* status, int64_t i, double f0, double f1,
                                         double f2) {
  out.fx[i] = f0;
  out.fy[i] = f1;
  out.fz[i] = f2;
  const uint32_t E = 0x7ff00000u;
  const bool bad = ((uint32_t)__double2hiint(f0) & E) == E || ((uint32_t)__double2hiint(f1) & E) == E ||
                   ((uint32_t)__double2hiint(f2) & E) == E;
  if (bad) atomicOr(status, ST_NONFINITE);
}

// Entries are processed in batches of VL_BATCH: the batch's list entries are
// loaded, then its positions gathered, then its pairs computed, so that every
// lane keeps several independent gathers in flight.  A short last batch is
// padded with j = i, which the exact R^2 = 0 rule rejects.
constexpr int VL_BATCH = 4;

// N3: 0 = off, 1 = atomic, 2 = two-pass (pass 1)
template <typename R, int N3, bool EV, bool I16>
__global__ void __launch_bounds__(256) k_vl_ipt(LJParams P, VLArgs A, ForceOut out) {
  const int64_t n = P.n;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool vi = i < n;
    R fx = 0, fy = 0, fz = 0, eu = 0, ew = 0;
    if (vi) {
      const uint4 pi = A.pos[i];
      const int m = min(A.nnbr[i], A.cap);
      // software pipeline: the next batch's list entries load while the
      // current batch's positions are gathered and its pairs computed
      int jc[VL_BATCH];
#pragma unroll
      for (int t = 0; t < VL_BATCH; ++t) jc[t] = (t < m) ? vl_entry<I16>(A, (int64_t)t * n + i, i, n) : (int)i;
      for (int k0 = 0; k0 < m; k0 += VL_BATCH) {
        uint4 pj[VL_BATCH];
#pragma unroll
        for (int t = 0; t < VL_BATCH; ++t) pj[t] = __ldg(A.pos + jc[t]);
        int jn[VL_BATCH];
#pragma unroll
        for (int t = 0; t < VL_BATCH; ++t) {
          const int k = k0 + VL_BATCH + t;
          jn[t] = (k < m) ? vl_entry<I16>(A, (int64_t)k * n + i, i, n) : (int)i;
        }
#pragma unroll
        for (int t = 0; t < VL_BATCH; ++t) {
          R af, bf, cf;
          const R fac = Prec<R>::template pair<EV>(mimg(pi.x, pj[t].x), mimg(pi.y, pj[t].y), mimg(pi.z, pj[t].z), P,
                                                   af, bf, cf, eu, ew, cnt);
          fx += fac * af;
          fy += fac * bf;
          fz += fac * cf;
          if (N3 == 1) {
            n3_add<R>(out, jc[t], fac * af, fac * bf, fac * cf);
          } else if (N3 == 2) {
            if (k0 + t < m) {
              const int64_t e = (int64_t)(k0 + t) * n + i;
              const int64_t ne = (int64_t)A.cap * n;
              R* sl = (R*)A.slot;
              sl[e] = fac * af;
              sl[ne + e] = fac * bf;
              sl[2 * ne + e] = fac * cf;
            }
          }
        }
#pragma unroll
        for (int t = 0; t < VL_BATCH; ++t) jc[t] = jn[t];
      }
      if (N3 == 1) {
        n3_add<R>(out, i, -fx, -fy, -fz);
      } else {
        vl_store(out, A.status, i, -P.e24u * Prec<R>::to_d(fx), -P.e24u * Prec<R>::to_d(fy),
                 -P.e24u * Prec<R>::to_d(fz));
      }
    }
    if (EV) {
      eu_d += Prec<R>::to_d(eu);
      ew_d += Prec<R>::to_d(ew);
    }
  }
  block_flush<R>(eu_d, ew_d, cnt, out, EV);
}

// Six blocks of 256 per SM (40 registers) without Newton-3.  The Newton-3
// variants hold more live values (the j-side contributions and their vector
// reductions) and get four blocks (64 registers): at five (48) they spilled
// 8-40 bytes and JSPLIT-2/4 ran 11 % / 8 % slower (1,048,576-particle fluid).
template <typename R, int W, int N3, bool EV, bool I16>
__global__ void __launch_bounds__(256, N3 == 1 ? 4 : 6) k_vl_jsplit(LJParams P, VLArgs A, ForceOut out) {
  constexpr int G = 32 / W;
  // Two-lane groups read their list entries in pairs: lane sub takes
  // entries 2 sub and 2 sub + 1 of every 4-entry chunk with one 8-byte load,
  // so a warp's list load serves 4 entries of each of its 16 rows.  (Rows
  // start on 32-byte boundaries: the capacity is a multiple of 8.)  Measured
  // on the 1,048,576-particle fluid: w = 2 gains 6 %; w = 4 and 8 lose 1.5 %
  // and 4 %, their gathers spreading over more lines than the loads save.
  constexpr bool PAIRED = !I16 && W == 2;
  static_assert(VL_BATCH % 2 == 0, "paired entries fill a batch");
  const int lane = threadIdx.x & 31, g = lane / W, sub = lane % W;
  const int64_t n = P.n;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double eu_d = 0.0, ew_d = 0.0;
  int cnt = 0;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * G < n; w += nwarps) {
    const int64_t i = w * G + g;
    const bool vi = i < n;
    R fx = 0, fy = 0, fz = 0, eu = 0, ew = 0;
    if (vi) {
      const uint4 pi = A.pos[i];
      const int m = min(A.nnbr[i], A.cap);
      // running pointer to this lane's next entries of row i (entries k0 + t W,
      // or k0 + 2 W c + {0, 1} when paired)
      const int32_t* rp = A.nbr + i * A.cap + (PAIRED ? 2 * sub : sub);
      const int16_t* rp16 = I16 ? A.nbr16 + i * A.cap + sub : nullptr;
      auto entry = [&](int off) -> int {
        if (I16) {
          int64_t j = i + (int64_t)__ldcs(rp16 + off);
          j += (j < 0) ? n : 0;
          j -= (j >= n) ? n : 0;
          return (int)j;
        }
        const int j = __ldcs(rp + off);
        return LJ_IDX_OK((unsigned)j < (unsigned)n, A.status) ? j : (int)i;  // checks build: self, no pair
      };
      // the lane's VL_BATCH entries from rp on, k0 being the first one's index;
      // entries past the row's end are i itself (R^2 = 0: no pair)
      auto batch = [&](int k0, int (&jj)[VL_BATCH]) {
        if constexpr (PAIRED) {
#pragma unroll
          for (int c = 0; c < VL_BATCH / 2; ++c) {
            const int k = k0 + c * 2 * W;  // even, so k < m <= cap keeps k + 1 inside the row
            int2 v = make_int2((int)i, (int)i);
            if (k < m) v = __ldcs(reinterpret_cast<const int2*>(rp + c * 2 * W));
            jj[2 * c] = LJ_IDX_OK((unsigned)v.x < (unsigned)n, A.status) ? v.x : (int)i;
            jj[2 * c + 1] = (k + 1 < m && LJ_IDX_OK((unsigned)v.y < (unsigned)n, A.status)) ? v.y : (int)i;
          }
        } else {
#pragma unroll
          for (int t = 0; t < VL_BATCH; ++t) jj[t] = (k0 + t * W < m) ? entry(t * W) : (int)i;
        }
      };
      int jc[VL_BATCH];
      batch(PAIRED ? 2 * sub : sub, jc);
      for (int k0 = PAIRED ? 2 * sub : sub; k0 < m; k0 += W * VL_BATCH) {
        uint4 pj[VL_BATCH];
#pragma unroll
        for (int t = 0; t < VL_BATCH; ++t) pj[t] = __ldg(A.pos + jc[t]);
        int jn[VL_BATCH];
        rp += W * VL_BATCH;
        if (I16) rp16 += W * VL_BATCH;
        batch(k0 + W * VL_BATCH, jn);
#pragma unroll
        for (int t = 0; t < VL_BATCH; ++t) {
          R af, bf, cf;
          const R fac = Prec<R>::template pair<EV, false, true>(mimg(pi.x, pj[t].x), mimg(pi.y, pj[t].y),
                                                                mimg(pi.z, pj[t].z), P, af, bf, cf, eu, ew, cnt);
          fx += fac * af;
          fy += fac * bf;
          fz += fac * cf;
          if (N3 == 1) {
            n3_add<R>(out, jc[t], fac * af, fac * bf, fac * cf);
          }
        }
#pragma unroll
        for (int t = 0; t < VL_BATCH; ++t) jc[t] = jn[t];
      }
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
      fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (vi && sub == 0) {
      if (N3 == 1) {
        n3_add<R>(out, i, -fx, -fy, -fz);
      } else {
        vl_store(out, A.status, i, -P.e24u * Prec<R>::to_d(fx), -P.e24u * Prec<R>::to_d(fy),
                 -P.e24u * Prec<R>::to_d(fz));
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

// k_force_dispatch.cuh -- selects the force kernel instantiation for a
// configuration (order x parameter x Newton-3 x energy/virial) and launches it
// on the context's stream.  Included by one translation unit per
// (container, precision) so that the instantiations compile in parallel.
#pragma once
#include "k_force_lc.cuh"
#include "k_force_vl.cuh"

namespace ljgb {

constexpr int kSMs = 152;

inline unsigned grid_for(int64_t threads, int tpb, int per_sm) {
  int64_t b = (threads + tpb - 1) / tpb;
  if (b > (int64_t)kSMs * per_sm) b = (int64_t)kSMs * per_sm;
  return (unsigned)(b < 1 ? 1 : b);
}

template <typename R, bool N3, bool EV, bool BWD>
cudaError_t lc_launch(Ctx& c, const lj_config& cfg, ForceOut out) {
  LCArgs A{c.pos, c.cell_start, c.tiles, c.ntiles_dev, c.tile_ctr};
  cudaError_t e;
  const int64_t n = c.n;
  auto prep = [&](int T) -> cudaError_t {
    cudaError_t r = build_tiles(c, T);
    if (r != cudaSuccess) return r;
    A.tiles = c.tiles;
    A.ntiles = c.ntiles_dev;
    return cudaMemsetAsync(c.tile_ctr, 0, sizeof(uint32_t), c.stream);
  };
  switch (cfg.order) {
    case LJ_ORD_IPT_SMEM:
      if ((e = prep(32)) != cudaSuccess) return e;
      k_lc_ipt<R, 1, N3, EV, BWD><<<grid_for(n, 256, 8), 256, 0, c.stream>>>(c.P, A, out);
      break;
    case LJ_ORD_KI:
      if (cfg.param == 2) {
        if ((e = prep(64)) != cudaSuccess) return e;
        k_lc_ipt<R, 2, N3, EV, BWD><<<grid_for(n / 2 + 32, 256, 8), 256, 0, c.stream>>>(c.P, A, out);
      } else {
        if ((e = prep(128)) != cudaSuccess) return e;
        k_lc_ipt<R, 4, N3, EV, BWD><<<grid_for(n / 4 + 32, 256, 8), 256, 0, c.stream>>>(c.P, A, out);
      }
      break;
    case LJ_ORD_IPT_TMA:
      if ((e = prep(32)) != cudaSuccess) return e;
      k_lc_tma<R, N3, EV, BWD><<<grid_for(n, TMA_WARPS * 32, 16), TMA_WARPS * 32, 0, c.stream>>>(c.P, A, out);
      break;
    case LJ_ORD_ROT32:
      if ((e = prep(32)) != cudaSuccess) return e;
      k_lc_rot<R, N3, EV, BWD><<<grid_for(n, 256, 8), 256, 0, c.stream>>>(c.P, A, out);
      break;
    case LJ_ORD_JSPLIT: {
      const int w = cfg.param;
      const int64_t thr = n * w;
      if (cfg.container == LJ_LCS) {  // sub-cells: the 5 x 5 x 5 stencil
        switch (w) {
          case 8: k_lc_jsplit<R, 8, N3, EV, BWD, 2><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
          case 4: k_lc_jsplit<R, 4, N3, EV, BWD, 2><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
          default: k_lc_jsplit<R, 2, N3, EV, BWD, 2><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
        }
        break;
      }
      switch (w) {
        case 32: k_lc_jsplit<R, 32, N3, EV, BWD><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
        case 16: k_lc_jsplit<R, 16, N3, EV, BWD><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
        case 8: k_lc_jsplit<R, 8, N3, EV, BWD><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
        case 4: k_lc_jsplit<R, 4, N3, EV, BWD><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
        default: k_lc_jsplit<R, 2, N3, EV, BWD><<<grid_for(thr, 256, 16), 256, 0, c.stream>>>(c.P, c.pos, c.cell_start, out); break;
      }
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t force_lc_t(Ctx& c, const lj_config& cfg, bool ev) {
  ForceOut out{c.frc, c.frc + c.n, c.frc + 2 * c.n, c.ev, c.npairs, c.status};
  const bool bwd = cfg.newton3 == LJ_N3_ATOMIC_BWD;
  const bool n3 = cfg.newton3 == LJ_N3_ATOMIC || bwd;
  if (n3) {
    cudaError_t e = n3_begin(c, out, sizeof(R) == 4);
    if (e != cudaSuccess) return e;
  }
  if (bwd) return ev ? lc_launch<R, true, true, true>(c, cfg, out) : lc_launch<R, true, false, true>(c, cfg, out);
  if (n3) return ev ? lc_launch<R, true, true, false>(c, cfg, out) : lc_launch<R, true, false, false>(c, cfg, out);
  return ev ? lc_launch<R, false, true, false>(c, cfg, out) : lc_launch<R, false, false, false>(c, cfg, out);
}

// Launch of a Verlet-list kernel with an L2 access-policy window over the
// position array: the positions (16 B per particle, gathered ~70 times each)
// persist in L2 while the list entries (read once) stream past them.
template <typename... KArgs, typename... Args>
cudaError_t vl_launch_ex(const Ctx& c, void (*k)(KArgs...), unsigned grid, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.stream = c.stream;
  cudaLaunchAttribute attr[1];
  unsigned na = 0;
  if (c.l2_window_bytes > 0) {
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = (void*)c.pos;
    attr[0].val.accessPolicyWindow.num_bytes = std::min(c.l2_window_bytes, (size_t)c.n * sizeof(uint4));
    attr[0].val.accessPolicyWindow.hitRatio = 1.0f;
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    na = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename R, int N3, bool EV, bool I16>
cudaError_t vl_launch_i(Ctx& c, const lj_config& cfg, ForceOut out) {
  VLArgs A{c.pos, c.nbr, I16 ? c.nbr16 : nullptr, c.nnbr, c.vl_cap, c.twopass, c.status};
  const int64_t n = c.n;
  if (cfg.order == LJ_ORD_VL_IPT) {
    return vl_launch_ex(c, k_vl_ipt<R, N3, EV, I16>, grid_for(n, 256, 8), c.P, A, out);
  } else if (N3 != 2) {
    const unsigned g = grid_for(n * cfg.param, 256, 16);
    switch (cfg.param) {
      case 32: return vl_launch_ex(c, k_vl_jsplit<R, 32, N3, EV, I16>, g, c.P, A, out);
      case 16: return vl_launch_ex(c, k_vl_jsplit<R, 16, N3, EV, I16>, g, c.P, A, out);
      case 8: return vl_launch_ex(c, k_vl_jsplit<R, 8, N3, EV, I16>, g, c.P, A, out);
      case 4: return vl_launch_ex(c, k_vl_jsplit<R, 4, N3, EV, I16>, g, c.P, A, out);
      default: return vl_launch_ex(c, k_vl_jsplit<R, 2, N3, EV, I16>, g, c.P, A, out);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename R, int N3, bool EV>
cudaError_t vl_launch(Ctx& c, const lj_config& cfg, ForceOut out) {
  return c.vl_idx16 ? vl_launch_i<R, N3, EV, true>(c, cfg, out) : vl_launch_i<R, N3, EV, false>(c, cfg, out);
}

template <typename R>
cudaError_t force_vl_t(Ctx& c, const lj_config& cfg, bool ev) {
  ForceOut out{c.frc, c.frc + c.n, c.frc + 2 * c.n, c.ev, c.npairs, c.status};
  cudaError_t e;
  if (cfg.newton3 == LJ_N3_ATOMIC) {
    if ((e = n3_begin(c, out, sizeof(R) == 4)) != cudaSuccess) return e;
    return ev ? vl_launch<R, 1, true>(c, cfg, out) : vl_launch<R, 1, false>(c, cfg, out);
  }
  if (cfg.newton3 == LJ_N3_TWOPASS) {
    e = ev ? vl_launch<R, 2, true>(c, cfg, out) : vl_launch<R, 2, false>(c, cfg, out);
    if (e != cudaSuccess) return e;
    return launch_twopass_gather(c);
  }
  return ev ? vl_launch<R, 0, true>(c, cfg, out) : vl_launch<R, 0, false>(c, cfg, out);
}

}  // namespace ljgb

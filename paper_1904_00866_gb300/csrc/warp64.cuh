// FP64 FORMULA of one node computed by a whole warp (FP32 / FP16 storage
// fixups): lane i < Q holds population i, so each lane evaluates one
// population's equilibrium factor, division and logarithms, and the sums
// over i are warp reductions.
//
// GB300 issues one FP64 warp instruction per ~64 cycles on each SM
// sub-partition.  A node collided on one lane (node64_prepare +
// alpha_formula64: ~2,400 FP64 instructions for D3Q27, most of them the 27
// divisions and logarithms) therefore holds its warp for ~75 us, and a
// fixup with a few thousand such nodes ends ~0.2 ms after its last node
// started, however they are spread.  Spread over the lanes the node takes
// ~460 FP64 warp instructions (divisions, logarithms and the reductions)
// and so ends ~6x sooner; in bulk, one node per lane costs fewer FP64
// instructions per node (~75), which the fixups use on long queues.
//
// The arithmetic is that of node64_prepare and alpha_formula64 (Eq. (8),
// the acceptance test after it, Eq. (9)), population by population; only
// the order of the sums over i differs (pairwise over the lanes), which
// moves Delta H by rounding only.
#pragma once
#include "node_fp64.cuh"

namespace elbm {

// Velocity, weight and binary16 scale of the population a lane holds.
struct LanePop {
  int c[3];
  double w;
  float hscale, hscale_inv;
  bool on;   // lane < Q
};

template <class L>
__device__ __forceinline__ LanePop lane_pop(int lane) {
  LanePop r{{0, 0, 0}, 0.0, 1.0f, 1.0f, lane < L::Q};
#pragma unroll
  for (int q = 0; q < L::Q; ++q)
    if (q == lane) {
      r.c[0] = L::c(q, 0);
      r.c[1] = L::c(q, 1);
      r.c[2] = L::c(q, 2);
      r.w = L::w(q);
      r.hscale = L::hscale(q);
      r.hscale_inv = L::hscale_inv(q);
    }
  return r;
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_min64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Result of formula64_warp (the same on every lane).
struct Warp64 {
  double rho, j[3], alpha;
  unsigned flags;   // NF_ACCEPT_* / NF_FORMULA, or NF_BAD_* (state invalid)
};

// All 32 lanes call this with f = f_i on lane i < Q (anything on the other
// lanes).  Writes the post-collision population of the lane through
// store(value) (lanes < Q only): f + alpha beta (f^eq - f), alpha rounded
// down to FP32 (the FP32 storage paths' convention), or f unchanged when
// the state is invalid.
template <class L, class Store>
__device__ __forceinline__ Warp64 formula64_warp(const LanePop& lp, double f,
                                                 double beta, Store store) {
  Warp64 r;
  r.flags = 0;
  const double fi = lp.on ? f : 0.0;
  if (__any_sync(0xffffffffu, lp.on && !(f > 0.0))) r.flags |= NF_BAD_NEG;
  r.rho = warp_sum64(fi);
  double u[3] = {0.0, 0.0, 0.0}, dp[3], dm[3], d0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r.j[a] = a < L::D ? warp_sum64((double)lp.c[a] * fi) : 0.0;
    if (a >= L::D) continue;
    u[a] = r.j[a] / r.rho;
    if (!(fabs(u[a]) < 1.0)) r.flags |= NF_BAD_NONFINITE;
    const double sg = 3.0 * u[a] * u[a] / (1.0 + sqrt(1.0 + 3.0 * u[a] * u[a]));
    dp[a] = 3.0 * u[a] + 2.0 * sg;
    dm[a] = -3.0 * u[a] + 2.0 * sg;
    d0[a] = -sg;
  }
  if (!(r.rho > 0.0) || !isfinite(r.rho)) r.flags |= NF_BAD_NONFINITE;
  r.alpha = 1.0;
  if (r.flags) {
    if (lp.on) store(f);
    return r;
  }
  double P = r.rho * lp.w;
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const int ca = lp.c[a];
    P *= 1.0 + (ca == 1 ? dp[a] : (ca == -1 ? dm[a] : d0[a]));
  }
  const double x = lp.on ? (P - f) / f : 0.0;
  const double amax = warp_min64(x < 0.0 ? -1.0 / x : INFINITY);
  const double astar = fmin(2.0, amax);
  const double Li = log1p(x);
  const double B = warp_sum64(fi * x * Li);
  const double D1 = warp_sum64(fi * (Li - x));
  const double Dstar = warp_sum64(fi * phi64(astar * x)) - astar * B;
  double alpha;
  if (Dstar <= 0.0) {
    r.flags |= NF_ACCEPT_STAR;
    if (astar == 2.0) r.flags |= NF_ACCEPT_TWO;
    alpha = astar;
  } else {
    r.flags |= NF_FORMULA;
    alpha = Dstar - D1 > 0.0 ? astar + Dstar / (Dstar - D1) * (1.0 - astar)
                             : 1.0;
  }
  alpha = (double)__double2float_rd(alpha);
  r.alpha = alpha;
  if (lp.on) store(fma(alpha * beta, f * x, f));
  return r;
}

}  // namespace elbm

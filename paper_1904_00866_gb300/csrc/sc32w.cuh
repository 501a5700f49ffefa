// FP32-shifted FORMULA stream-collide with wide (16-byte) gathers, for
// lattices whose x extent is a multiple of 64.
//
// A warp owns 64-node row segments [x0, x0 + 64) of one (y, z) row and walks
// them with a grid stride.  For every population i the pull sources of the
// segment are the 64 (+1 at the shifted edge) consecutive elements of one
// row of array i, so a single cp.async instruction per population moves
// them: lanes 0..15 copy the 16 aligned 16-byte chunks of [x0, x0 + 64) and,
// for the 18 (or 6) populations shifted by +-1 in x, lane 16 copies the
// aligned 16-byte chunk holding x0 - 1 or x0 + 64 (wrapped periodically).
// Each load instruction then moves 256-272 bytes instead of the 128 of one
// element per lane; on GB300 the memory system serves these at a markedly
// higher rate (copying 27 population arrays with 256- versus 128-byte load
// instructions: 6.0 vs 5.2 TB/s).
// Lane l collides nodes x0 + l and x0 + 32 + l from the warp's own
// shared-memory rows (warp-level synchronisation only); stores stay plain
// coalesced 4-byte writes.  Two stages per warp: the next segment is in
// flight while one is computed.  The shared-memory rows (58 KB per
// 4-warp block) and 155 registers allow 12 warps per SM against the
// default kernel's 16, so the full step gains nothing on GB300 (the node
// arithmetic hides the narrower loads there); the variant is opt-in
// (ELBM_SC32_VARIANT=wide).
#pragma once
#include <stdint.h>

#include "sc32.cuh"

namespace elbm {

constexpr int kWideWarps = 4;                 // warps per block
constexpr int kWideThreads = 32 * kWideWarps;
constexpr int kWideSeg = 64;                  // nodes per warp segment

__device__ __forceinline__ void cp_async16(float* smem_dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s),
               "l"(src)
               : "memory");
}

// Shared-memory row of population i within a warp stage: 64 floats, plus a
// 4-float halo chunk on the left (c_ix = +1, source x - 1) or on the right
// (c_ix = -1, source x + 1).
template <class L>
__host__ __device__ constexpr int wide_len(int i) {
  return L::c(i, 0) == 0 ? kWideSeg : kWideSeg + 4;
}
template <class L>
__host__ __device__ constexpr int wide_base(int i) {
  int b = 0;
  for (int j = 0; j < i; ++j) b += wide_len<L>(j);
  return b;
}
template <class L>
__host__ __device__ constexpr int wide_stage_floats() {
  return wide_base<L>(L::Q);
}
// offset within the row of the source of segment position t: t + shift
template <class L>
__host__ __device__ constexpr int wide_shift(int i) {
  return L::c(i, 0) == 1 ? 3 : (L::c(i, 0) == -1 ? 1 : 0);
}

template <class L>
__device__ __forceinline__ void issue_wide(const StepParams& p, float* st,
                                           unsigned seg, int lane) {
  const unsigned node0 = seg * kWideSeg;
  const unsigned row = p.div_nx.div(node0);
  const int x0 = (int)(node0 - row * (unsigned)p.nx);
  const unsigned zq = p.div_ny.div(row);
  const int y = (int)(row - zq * (unsigned)p.ny), z = (int)zq;
  const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
  // lanes 0..15: main chunks; lane 16: halo chunk (shifted populations)
  const int xl = x0 == 0 ? p.nx - 4 : x0 - 4;
  const int xr = x0 + kWideSeg == p.nx ? 0 : x0 + kWideSeg;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    if (lane > 16 || (lane == 16 && cx == 0)) continue;
    const int ys = cy == 1 ? ym : (cy == -1 ? yp : y);
    const int zs = cz == 1 ? zm : (cz == -1 ? zp : z);
    const float* src_row =
        p.in_pop[i] + ((size_t)zs * (size_t)p.ny + (size_t)ys) * (size_t)p.nx;
    float* dst = st + wide_base<L>(i);
    if (lane < 16)
      cp_async16(dst + (cx == 1 ? 4 : 0) + 4 * lane, src_row + x0 + 4 * lane);
    else
      cp_async16(dst + (cx == 1 ? 0 : kWideSeg),
                 src_row + (cx == 1 ? xl : xr));
  }
}

template <class L, int DIAG, int CHECK>
__global__ void __launch_bounds__(kWideThreads, 3)
    k_sc32w(const StepParams p) {
  constexpr int S = wide_stage_floats<L>();
  extern __shared__ __align__(16) float smem_wide[];   // [warps][2][S]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* my = smem_wide + w * 2 * S;
  const unsigned nseg = (unsigned)(p.n / kWideSeg);
  const unsigned nwarps = gridDim.x * kWideWarps;
  const float rho0f = p.rho0f;
  const float beta = p.betaf;
  Acc32 acc;
  if (DIAG) acc.init();
  __shared__ unsigned s_refine;     // this block's undecided-node entries
  refine_block_begin(&s_refine);

  unsigned seg = blockIdx.x * kWideWarps + w;
  int stage = 0;
  if (seg < nseg) issue_wide<L>(p, my, seg, lane);
  cp_async_commit();
  for (; seg < nseg; seg += nwarps) {
    // every lane has finished reading the stage refilled here
    __syncwarp();
    const unsigned next = seg + nwarps;
    if (next < nseg) issue_wide<L>(p, my + (stage ^ 1) * S, next, lane);
    cp_async_commit();
    cp_async_wait<1>();   // this lane's copies of `seg` have landed ...
    __syncwarp();         // ... and so have the other lanes'
    const float* st = my + stage * S;
    stage ^= 1;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int t = 32 * h + lane;
      const unsigned node = seg * kWideSeg + t;
      auto in = [&](int i) { return st[wide_base<L>(i) + wide_shift<L>(i) + t]; };
      float ap = 0.0f;
      const unsigned res = sc32_node_in<L, true, DIAG, CHECK>(
          in, rho0f, p.rho0, beta, 0.0f, nullptr,
          p.alpha_map ? p.alpha_map + node : nullptr, acc,
          [&](int i, float v) { p.out_pop[i][node] = v; },
          p.exact ? &ap : nullptr);
      if (p.exact)
        defer_undecided<L>(p, &s_refine, res == kNodeRefine, in, node, ap);
      defer_nodes(&p.far_count[p.parity], p.far_queue, p.far_cap,
                  p.err_flags, node, res == kNodeFar ? kNodeFar : kNodeDone);
    }
  }
  cp_async_wait<0>();
  refine_block_end(p, &s_refine);
  if (DIAG) store_acc32(acc, p.partials);
}

}  // namespace elbm

// Pipelined FP32-storage FORMULA stream-collide kernel (Eq. (5b) pull gather
// + Eq. (5a) relax), the hot path for FP32 / FP32-shifted storage.
//
// A block owns tiles of 256 consecutive nodes (flat index, so ragged
// lattices keep every lane busy) and walks them with a grid stride.  The 27
// (or 9) pull gathers of the NEXT tile are issued as asynchronous
// global->shared copies (cp.async, 4 B per thread and population) while the
// current tile is computed from shared memory: every thread keeps one
// tile's worth of loads in flight without holding them in registers.
// Stores of the post-collision populations are plain coalesced writes.
// Shared memory: 2 stages x Q x 256 floats (55 KB for D3Q27).
#pragma once
#include <stdint.h>

#include "node_fp32.cuh"
#include "stream_collide.cuh"

namespace elbm {

constexpr int kSc32Threads = 256;

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Compensated FP32 sum (Kahan) for the per-thread diagnostics.
struct KSum {
  float s, c;
  __device__ __forceinline__ void init() { s = c = 0.0f; }
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const {
    return (double)s - (double)c;
  }
};

struct Acc32 {
  KSum drho, j0, j1, j2, ke, asum;
  float amin, amax;
  unsigned nodes, acc2, formula, band, degen;
  double h, adev;
  unsigned viol, mismatch;
  __device__ __forceinline__ void init() {
    drho.init(); j0.init(); j1.init(); j2.init(); ke.init(); asum.init();
    amin = INFINITY;
    amax = -INFINITY;
    nodes = acc2 = formula = band = degen = 0u;
    h = adev = 0.0;
    viol = mismatch = 0u;
  }
};

// Block reduction of the per-thread FP32 accumulators into one partials
// row (FP64 slots).
__device__ __forceinline__ void store_acc32(const Acc32& acc,
                                            double* partials) {
  Acc a;
  a.init();
  a.drho = acc.drho.value();
  a.j0 = acc.j0.value();
  a.j1 = acc.j1.value();
  a.j2 = acc.j2.value();
  a.ke = acc.ke.value();
  a.asum = acc.asum.value();
  a.h = acc.h;
  a.amin = acc.amin;
  a.amax = acc.amax;
  a.adev = acc.adev;
  a.nodes = acc.nodes;
  a.acc2 = acc.acc2;
  a.accstar = acc.acc2;
  a.formula = acc.formula;
  a.band = acc.band;
  a.degen = acc.degen;
  a.viol = acc.viol;
  a.mismatch = acc.mismatch;
  a.block_reduce_store(partials);
}

template <class L>
__device__ __forceinline__ void node_xyz(const StepParams& p, unsigned node,
                                         int& x, int& y, int& z) {
  const unsigned q1 = p.div_nx.div(node);
  x = (int)(node - q1 * (unsigned)p.nx);
  const unsigned q2 = p.div_ny.div(q1);
  y = (int)(q1 - q2 * (unsigned)p.ny);
  z = (int)q2;
}

template <class L>
__device__ __forceinline__ void issue_tile(const StepParams& p, float* sm,
                                           unsigned tile) {
  const unsigned node = tile * kSc32Threads + threadIdx.x;
  if (node >= (unsigned)p.n) return;
  int x, y, z;
  node_xyz<L>(p, node, x, y, z);
  const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    // pull source x - c_i
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int xs = cx == 1 ? xm : (cx == -1 ? xp : x);
    const int ys = cy == 1 ? ym : (cy == -1 ? yp : y);
    const int zs = cz == 1 ? zm : (cz == -1 ? zp : z);
    const unsigned off = ((unsigned)zs * (unsigned)p.ny + (unsigned)ys) *
                             (unsigned)p.nx + (unsigned)xs;
    cp_async4(sm + i * kSc32Threads + threadIdx.x, p.in_pop[i] + off);
  }
}

// Collision of one node whose Q gathered values are returned by in(i)
// (shared memory).  Writes the Q post-collision values through
// out(i, value) and the alpha through amap (nullable).  Returns false when
// the node must go to the FP64 fixup (nothing written).
template <class L, bool SHIFTED, int DIAG, int CHECK, class In, class Out>
__device__ __forceinline__ bool sc32_node_in(In in, float rho0f, double rho0,
                                             float beta, float corr_rho,
                                             const float* __restrict__ corr,
                                             float* amap, Acc32& acc,
                                             Out out) {
  constexpr int Q = L::Q;
  constexpr int P = npairs<L>();
  float d0;
  float2 dd[P];
  {
    const float v = in(0);
    d0 = SHIFTED ? v : v - L::wf(0) * rho0f;
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const float2 v = make_float2(in(2 * k + 1), in(2 * k + 2));
    dd[k] = SHIFTED ? v : sub2(v, f2(L::wf(2 * k + 1) * rho0f));
  }
  float a_extra = 0.0f;
  if (!SHIFTED) {
    // delta_i = v_i - s_i is exact unless v_i leaves [s_i/2, 2 s_i]
    float A = fabsf(d0);
#pragma unroll
    for (int k = 0; k < P; ++k) A += fabsf(dd[k].x) + fabsf(dd[k].y);
    a_extra = 2.0f * 5.9604645e-8f * A / rho0f;
  }
  N32<L> r;
  node32_formula<L, SHIFTED>(d0, dd, rho0f, corr_rho, corr, a_extra, r);
  if (r.flags & NF_FAR) return false;
  // relax with the conservation-projected n:  f~ = f + alpha beta n
  const float ab = r.alpha * beta;
  projection<L>(
      r,
      [&](float wt) {
        const float nv = fmaf(ab, r.n0 - wt, d0);
        out(0, SHIFTED ? nv : nv + L::wf(0) * rho0f);
      },
      [&](int k, float2 wt) {
        float2 nv = fma2(f2(ab), sub2(r.n2[k], wt), dd[k]);
        if (!SHIFTED) nv = add2(nv, f2(L::wf(2 * k + 1) * rho0f));
        out(2 * k + 1, nv.x);
        out(2 * k + 2, nv.y);
      });
  if (amap) *amap = r.alpha;
  if (DIAG) {
    acc.nodes += 1;
    acc.drho.add(r.drho);
    acc.j0.add(r.j[0]);
    acc.j1.add(r.j[1]);
    acc.j2.add(r.j[2]);
    acc.ke.add(0.5f * (r.j[0] * r.j[0] + r.j[1] * r.j[1] + r.j[2] * r.j[2]) /
               r.rho);
    acc.asum.add(r.alpha);
    acc.amin = fminf(acc.amin, r.alpha);
    acc.amax = fmaxf(acc.amax, r.alpha);
    acc.acc2 += (r.flags & NF_ACCEPT_TWO) != 0;
    acc.formula += (r.flags & NF_FORMULA) != 0;
    acc.band += (r.flags & NF_BAND) != 0;
    acc.degen += (r.flags & NF_DEGENERATE) != 0;
    if (CHECK) {
      Node64<L> nd;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double v = (double)in(i);
        nd.f[i] = SHIFTED ? L::w(i) * rho0 + v : v;
      }
      node64_prepare(nd);
      Check64 ck = node64_check(nd, (double)r.alpha);
      acc.h += ck.h;
      acc.viol += ck.violation;
      acc.mismatch += ((r.flags & NF_ACCEPT_STAR) != 0) != ck.accept_ref;
      acc.adev = fmax(acc.adev, fabs((double)r.alpha - ck.alpha_ref));
    }
  }
  return true;
}

// Same, with the values in a shared-memory column of stride TB.
template <class L, bool SHIFTED, int DIAG, int CHECK, int TB, class Out>
__device__ __forceinline__ bool sc32_node(const float* sm, float rho0f,
                                          double rho0, float beta,
                                          float corr_rho,
                                          const float* __restrict__ corr,
                                          float* amap, Acc32& acc, Out out) {
  return sc32_node_in<L, SHIFTED, DIAG, CHECK>(
      [&](int i) { return sm[i * TB]; }, rho0f, rho0, beta, corr_rho, corr,
      amap, acc, out);
}

template <class L, bool SHIFTED, int DIAG, int CHECK>
__global__ void __launch_bounds__(kSc32Threads, 2)
    k_sc32(const StepParams p) {
  constexpr int Q = L::Q;
  extern __shared__ float smem[];   // [2][Q][256]
  const unsigned ntiles = (unsigned)((p.n + kSc32Threads - 1) / kSc32Threads);
  const float rho0f = (float)p.rho0;
  const float beta = (float)p.beta;
  Acc32 acc;
  if (DIAG) acc.init();

  unsigned tile = blockIdx.x;
  int stage = 0;
  if (tile < ntiles) issue_tile<L>(p, smem, tile);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const unsigned next = tile + gridDim.x;
    if (next < ntiles)
      issue_tile<L>(p, smem + (stage ^ 1) * Q * kSc32Threads, next);
    cp_async_commit();
    cp_async_wait<1>();   // this thread's copies of `tile` have landed

    const unsigned node = tile * kSc32Threads + threadIdx.x;
    const float* sm = smem + stage * Q * kSc32Threads + threadIdx.x;
    stage ^= 1;
    if (node >= (unsigned)p.n) continue;
    const bool done = sc32_node<L, SHIFTED, DIAG, CHECK, kSc32Threads>(
        sm, rho0f, p.rho0, beta, p.corr_rho, p.corr,
        p.alpha_map ? p.alpha_map + node : nullptr, acc,
        [&](int i, float v) { p.out_pop[i][node] = v; });
    if (!done) {
      // far from (or invalid, or within FP32 noise of) equilibrium: the FP64
      // fixup collides this node from f_in
      const unsigned slot = atomicAdd(&p.far_count[p.parity], 1u);
      if (slot < p.far_cap)
        p.far_queue[slot] = node;
      else
        atomicOr(p.err_flags, NF_BAD_NONFINITE);   // cannot happen: cap = n
    }
  }
  cp_async_wait<0>();
  if (DIAG) store_acc32(acc, p.partials);
}

}  // namespace elbm

// Fixup kernels of the FP32 / FP16 FORMULA step, after the stream-collide
// kernel; both read f_in (unchanged during the step) and write f_out.
//   k_refine_stage: the second stage of the nodes whose FP32 entropy
//     decision was not certified (the stream-collide kernel wrote them with
//     the certified alpha and put their stored values in a buffer): f^eq - f
//     recomputed in double-float arithmetic, the decision retaken with its
//     much smaller error bound (node32_refine), and the populations the
//     decided alpha changes rewritten.
//   k_far_fixup: the FP64 FORMULA (Eqs. (8)-(9) with logarithms, alpha
//     rounded down to FP32; one node per warp) for nodes far from
//     equilibrium (max |x_i| > 1/8, a velocity component >= 1/4), invalid
//     states and the rare node the second stage left undecided.  It also
//     resets the other parity's counter for the next step (stream order
//     makes that counter idle here).
#pragma once
#include <type_traits>
#include "sc32.cuh"
#include "warp64.cuh"

namespace elbm {

// Second stage of one deferred node from its stored values v[] (FP32
// storage: the stored value; FP16: the decoded deviation); the kernel wrote
// it with the provisional alpha ap (NaN: unknown, recomputed).  Returns
// the second stage's status (kStageDone, kStageRetry: run again with DFS,
// kStageFP64: left to the FP64 path).
template <class L, bool SHIFTED, int DIAG, int CHECK, bool DFS, class Out>
__device__ __forceinline__ int refine_deferred(const StepParams& p,
                                               const float (&v)[L::Q],
                                               long long node, float ap,
                                               Acc& acc, Out out) {
  auto in = [&](int i) { return v[i]; };
  return second_stage32<L, SHIFTED, DIAG, CHECK, DFS>(
      in, p.rho0f, p.betaf, p.corr_rho, p.corr,
      p.alpha_map ? p.alpha_map + node : nullptr, ap, out,
      [&](const N32<L>& r) {
        if (!DIAG) return;
        const double j[3] = {r.j[0], r.j[1], r.j[2]};
        acc.add_moments((double)r.drho, j, (double)r.rho);
        acc.add_alpha((double)r.alpha, r.flags, 0);
        if (CHECK) {
          Node64<L> nd;
          const Check64 ck = check32<L, SHIFTED>(in, p.rho0, r.alpha, nd);
          acc.add_check(ck.h, ck.violation,
                        decision_mismatch(r.flags, ck.accept_ref),
                        fabs((double)r.alpha - ck.alpha_ref));
        }
      });
}

// Second stage of the undecided nodes in the buffer (S: the storage type,
// float or half_t).  Block b of the stream-collide launch (`blocks`
// blocks) wrote refine_counts[b] entries from b (refine_cap / blocks) on;
// every block of this kernel forms their prefix sums in shared memory and
// takes entries k with a grid stride.  The double-float stage decides (and
// rewrites the populations its alpha changes); the few nodes its FP32
// series leaves open join the deferred-node queue tagged, so that the
// fixup (whose register budget holds it) runs them again with the leading
// terms of the series in double-float and collides the rest in FP64 with
// a whole warp.
template <class L, class S, int DIAG, int CHECK>
__global__ void __launch_bounds__(256, 2) k_refine_stage(const StepParams p,
                                                         int blocks) {
  constexpr int Q = L::Q;
  __shared__ unsigned pre[kMaxRefineBlocks + 1];
  block_prefix(p.refine_counts, blocks, pre);
  const unsigned total = pre[blocks];
  const unsigned seg = p.refine_cap / (unsigned)blocks;
  const bool shifted = sizeof(S) == 2 || !p.unshifted;
  Acc acc;
  acc.init();
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += gridDim.x * blockDim.x) {
    int lo = 0, hi = blocks;   // pre[lo] <= k < pre[lo + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pre[mid] <= k)
        lo = mid;
      else
        hi = mid;
    }
    constexpr int R = refine_record<L>();
    const float4* rec = reinterpret_cast<const float4*>(
        p.refine_buf + ((size_t)lo * seg + (k - pre[lo])) * (size_t)R);
    float w[R];
#pragma unroll
    for (int j = 0; j < R / 4; ++j) {
      const float4 t = rec[j];
      w[4 * j] = t.x;
      w[4 * j + 1] = t.y;
      w[4 * j + 2] = t.z;
      w[4 * j + 3] = t.w;
    }
    float v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = w[i];
    const long long node = __float_as_uint(w[Q]);
    const float ap = w[Q + 1];
    int st;
    if constexpr (sizeof(S) == 2) {
      st = refine_deferred<L, true, DIAG, CHECK, false>(
          p, v, node, ap, acc, [&](int i, float val) {
            reinterpret_cast<unsigned short*>(p.out_pop[i])[node] =
                h16_bits<L>(val, i);
          });
    } else {
      auto out = [&](int i, float val) { p.out_pop[i][node] = val; };
      st = shifted
               ? refine_deferred<L, true, DIAG, CHECK, false>(p, v, node, ap,
                                                              acc, out)
               : refine_deferred<L, false, DIAG, CHECK, false>(p, v, node, ap,
                                                               acc, out);
    }
    if (st != kStageDone) {
      // kStageRetry: tagged, so that the fixup runs the double-float
      // series pass (in its larger register budget) before any FP64
      const unsigned q = atomicAdd(&p.far_count[p.parity], 1u);
      if (q < p.far_cap)
        p.far_queue[q] =
            (unsigned)node | (st == kStageRetry ? kTagRefine : 0u);
      else
        atomicOr(p.err_flags, NF_BAD_NONFINITE);   // cannot happen: cap = n
    }
  }
  if (DIAG) acc.block_reduce_store(p.partials);
}

// FP64 fixup (S: the storage type, float or half_t): the deferred-node
// queue, with values gathered from f_in.  Entries tagged kTagRefine (a
// full buffer segment, or no buffer) take the second stage here first, one
// entry per thread; the nodes that need the FP64 FORMULA are then collided
// one at a time by their whole warp (formula64_warp, one population per
// lane).  Lane l of warp w takes entry w + l W of each round of 32 W
// entries (W warps in the grid), so a short queue leaves at most a few
// FP64 nodes to each warp and a long one (the first step after
// initialisation) still gives every lane its own entry; a warp with more
// than 16 FP64 nodes in a round runs them one per lane.  On steps with the
// FP64 entropy check (CHECK) the FP64 nodes run on their own lanes, as the
// check's statistics need each node's populations in one thread.
template <class L, class S, int DIAG, int CHECK>
__global__ void __launch_bounds__(256) k_far_fixup(const StepParams p) {
  constexpr int Q = L::Q;
  const unsigned count = min(p.far_count[p.parity], p.far_cap);
  const bool shifted = sizeof(S) == 2 || !p.unshifted;
  const int lane = threadIdx.x & 31;
  const unsigned W = gridDim.x * (blockDim.x >> 5);
  const unsigned wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const LanePop lp = lane_pop<L>(lane);
  const bool bulk = count > gridDim.x * blockDim.x;
  Acc acc;
  acc.init();
  auto coords = [&](long long node, int& x, int& y, int& z) {
    x = (int)(node % p.nx);
    y = (int)((node / p.nx) % p.ny);
    z = (int)(node / ((long long)p.nx * p.ny));
  };
  auto out_s = [&](long long node, int i, float val) {
    if constexpr (sizeof(S) == 2)
      reinterpret_cast<unsigned short*>(p.out_pop[i])[node] =
          h16_bits<L>(val, i);
    else
      p.out_pop[i][node] = val;
  };
  // FP64 FORMULA of one node in this thread
  auto fp64_lane = [&](long long node) {
    int x, y, z;
    coords(node, x, y, z);
    Node64<L> nd;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const long long src = src_index<L>(p, i, x, y, z);
      double vi;
      if constexpr (sizeof(S) == 2)
        vi = h16_dev<L>(reinterpret_cast<const unsigned short*>(
                            p.in_pop[i])[src],
                        i);
      else
        vi = p.in_pop[i][src];
      nd.f[i] = shifted ? L::w(i) * p.rho0 + vi : vi;
    }
    auto store_s = [&](int i, double val) {
      if (i < 0) {
        p.alpha_map[node] = (float)val;
      } else if constexpr (sizeof(S) == 2) {
        reinterpret_cast<half_t*>(p.out_pop[i])[node] =
            h16_from_dev<L>(val - L::w(i) * p.rho0, i);
      } else {
        p.out_pop[i][node] =
            (float)(p.unshifted ? val : val - L::w(i) * p.rho0);
      }
    };
    if (DIAG) acc.far += 1;
    collide64<L, MODE_FORMULA, CHECK>(nd, p, true, acc, DIAG != 0, store_s);
  };
  // FP64 FORMULA of node nd by the whole warp (every lane calls)
  auto fp64_warp = [&](long long nd) {
    int x, y, z;
    coords(nd, x, y, z);
    double f = 0.0;
    if (lp.on) {
      int xs = x - lp.c[0], ys = y - lp.c[1], zs = z - lp.c[2];
      xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
      ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
      zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
      const long long src = ((long long)zs * p.ny + ys) * p.nx + xs;
      if constexpr (sizeof(S) == 2) {
        const unsigned short b =
            reinterpret_cast<const unsigned short*>(p.in_pop[lane])[src];
        f = (double)(__half2float(__ushort_as_half(b)) * lp.hscale_inv);
      } else {
        f = (double)p.in_pop[lane][src];
      }
      if (shifted) f += lp.w * p.rho0;
    }
    const Warp64 r = formula64_warp<L>(lp, f, p.beta, [&](double val) {
      if constexpr (sizeof(S) == 2)
        reinterpret_cast<half_t*>(p.out_pop[lane])[nd] =
            __double2half((val - lp.w * p.rho0) * (double)lp.hscale);
      else
        p.out_pop[lane][nd] = (float)(p.unshifted ? val : val - lp.w * p.rho0);
    });
    if (lane == 0) {
      if (DIAG) acc.far += 1;
      if (r.flags & (NF_BAD_NEG | NF_BAD_NONFINITE)) {
        atomicOr(p.err_flags, r.flags);
      } else {
        if (p.alpha_map) p.alpha_map[nd] = (float)r.alpha;
        if (DIAG) {
          acc.add_moments(r.rho - p.rho0, r.j, r.rho);
          acc.add_alpha(r.alpha, r.flags, 0);
        }
      }
    }
  };
  // bulk queues: this warp's pending FP64 nodes (warp-uniform count)
  __shared__ unsigned pend_s[8][32];   // 256 threads: 8 warps
  unsigned* pend = pend_s[threadIdx.x >> 5];
  int npend = 0;
  auto flush = [&]() {   // every lane calls
    __syncwarp();
    if (lane < npend) fp64_lane((long long)pend[lane]);
    __syncwarp();
    npend = 0;
  };
  for (unsigned base = 0; base < count; base += 32u * W) {
    const unsigned k = base + (unsigned)lane * W + wid;
    bool need64 = false;
    long long node = 0;
    if (k < count) {
      const unsigned e = p.far_queue[k];
      node = e & ~kTagRefine;
      need64 = true;
      if (e & kTagRefine) {
        int x, y, z;
        coords(node, x, y, z);
        float v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const long long src = src_index<L>(p, i, x, y, z);
          if constexpr (sizeof(S) == 2)
            v[i] = h16_dev<L>(reinterpret_cast<const unsigned short*>(
                                  p.in_pop[i])[src],
                              i);
          else
            v[i] = p.in_pop[i][src];
        }
        const float ap = __int_as_float(0x7fc00000);   // NaN: recomputed
        auto out = [&](int i, float val) { out_s(node, i, val); };
        auto run = [&](auto dfs) {
          constexpr bool DFS = decltype(dfs)::value;
          return shifted ? refine_deferred<L, true, DIAG, CHECK, DFS>(
                               p, v, node, ap, acc, out)
                         : refine_deferred<L, false, DIAG, CHECK, DFS>(
                               p, v, node, ap, acc, out);
        };
        int st = run(std::false_type{});
        // the series pass pays off on the few nodes of a developed flow; on
        // a queue longer than the grid (the first step after
        // initialisation, where n is rounding noise and the pass decides
        // few nodes) they go to the FP64 path directly
        if (st == kStageRetry && !bulk) st = run(std::true_type{});
        need64 = st != kStageDone;
      }
    }
    // FP64 nodes of this round.  Per lane a node costs ~75 FP64 warp
    // instructions of its warp (2,400 shared by 32 lanes), per warp ~460:
    // one per warp ends sooner when a warp has few such nodes (developed
    // flows), one per lane costs less FP64 issue in bulk.  On a queue
    // longer than the grid (the first step after initialisation, ~1 % of
    // the nodes in FP64) each warp collects its FP64 nodes in shared memory
    // and runs them 32 at a time, one per lane.  The check's statistics
    // need each node in one thread.
    const unsigned m64 = __ballot_sync(0xffffffffu, need64);
    if (CHECK != 0 || (!bulk && __popc(m64) > 16)) {
      if (need64) fp64_lane(node);
    } else if (bulk) {
      const int nk = __popc(m64);
      if (npend + nk > 32) flush();
      if (need64) pend[npend + __popc(m64 & ((1u << lane) - 1u))] =
          (unsigned)node;
      npend += nk;
    } else {
      unsigned m = m64;
      while (m) {
        const int src_lane = __ffs(m) - 1;
        m &= m - 1;
        fp64_warp(__shfl_sync(0xffffffffu, node, src_lane));
      }
    }
  }
  if (npend > 0) {   // bulk remainder: few nodes run one per warp
    __syncwarp();
    if (npend > 5) {
      flush();
    } else {
      for (int j = 0; j < npend; ++j) fp64_warp((long long)pend[j]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) p.far_count[p.parity ^ 1] = 0u;
  if (DIAG) acc.block_reduce_store(p.partials);
}

}  // namespace elbm

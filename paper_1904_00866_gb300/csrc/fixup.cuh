// Fixup kernel of the FP32 / FP16 FORMULA step: collides the nodes the
// stream-collide kernel deferred, reading f_in (unchanged during the step)
// and writing f_out.
//
// Entries come from the undecided-node buffer (coalesced) and from the
// deferred-node queue; two kinds of entries:
//   * nodes whose FP32 entropy decision was not certified (tagged
//     kTagRefine; the kernel wrote them with a provisional alpha): the
//     second stage recomputes f^eq - f in double-float arithmetic, decides
//     with its much smaller error bound (node32_refine) and rewrites the
//     populations the decided alpha changes; the rare node still undecided
//     falls through to
//   * FP64: nodes far from equilibrium (max |x_i| > 1/8, |u| >= 1/2),
//     invalid states, and the undecided rest, collided by the FP64 FORMULA
//     (Eqs. (8)-(9) with logarithms), alpha rounded down to FP32.
// Resets the other parity's counter for the next step (stream order makes
// that counter idle here).
#pragma once
#include "sc32.cuh"

namespace elbm {

// Second stage of one deferred node from its stored values v[] (FP32
// storage: the stored value; FP16: the decoded deviation); the kernel wrote
// it with the provisional alpha ap (NaN: unknown, recomputed).  Returns
// false when the node is still undecided (left to the FP64 path).
template <class L, bool SHIFTED, int DIAG, int CHECK, class Out>
__device__ __forceinline__ bool refine_deferred(const StepParams& p,
                                                const float (&v)[L::Q],
                                                long long node, float ap,
                                                Acc& acc, Out out) {
  auto in = [&](int i) { return v[i]; };
  return second_stage32<L, SHIFTED, DIAG, CHECK>(
      in, (float)p.rho0, (float)p.beta, p.corr_rho, p.corr,
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
                        ((r.flags & NF_ACCEPT_STAR) != 0) != ck.accept_ref,
                        fabs((double)r.alpha - ck.alpha_ref));
        }
      });
}

// S: the storage type (float or half_t).  Entries [0, rcount) come from the
// undecided-node buffer (values stored there, read coalesced), the rest
// from the deferred-node queue (values gathered from f_in).
template <class L, class S, int DIAG, int CHECK>
__global__ void __launch_bounds__(256) k_far_fixup(const StepParams p) {
  constexpr int Q = L::Q;
  const unsigned rcount =
      p.refine_cap ? min(p.refine_count[p.parity], p.refine_cap) : 0u;
  const unsigned fcount = min(p.far_count[p.parity], p.far_cap);
  const bool shifted = sizeof(S) == 2 || !p.unshifted;
  Acc acc;
  acc.init();
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < rcount + fcount;
       k += gridDim.x * blockDim.x) {
    float v[Q];
    long long node;
    bool refine;
    float ap = __int_as_float(0x7fc00000);   // NaN: provisional alpha unknown
    if (k < rcount) {
      const float* b = p.refine_buf + k;
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = b[(size_t)i * p.refine_cap];
      node = __float_as_uint(b[(size_t)Q * p.refine_cap]);
      ap = b[(size_t)(Q + 1) * p.refine_cap];
      refine = true;
    } else {
      const unsigned e = p.far_queue[k - rcount];
      node = e & ~kTagRefine;
      refine = (e & kTagRefine) != 0u;
      const int x = (int)(node % p.nx);
      const int y = (int)((node / p.nx) % p.ny);
      const int z = (int)(node / ((long long)p.nx * p.ny));
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
    }
    if (refine) {
      bool done;
      if constexpr (sizeof(S) == 2) {
        done = refine_deferred<L, true, DIAG, CHECK>(
            p, v, node, ap, acc, [&](int i, float val) {
              reinterpret_cast<unsigned short*>(p.out_pop[i])[node] =
                  h16_bits<L>(val, i);
            });
      } else {
        auto out = [&](int i, float val) { p.out_pop[i][node] = val; };
        done = shifted ? refine_deferred<L, true, DIAG, CHECK>(p, v, node, ap,
                                                               acc, out)
                       : refine_deferred<L, false, DIAG, CHECK>(p, v, node, ap,
                                                                acc, out);
      }
      if (done) continue;
    }
    // FP64 FORMULA from the stored values
    Node64<L> nd;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double vi = (double)v[i];
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
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.far_count[p.parity ^ 1] = 0u;
    if (p.refine_count) p.refine_count[p.parity ^ 1] = 0u;
  }
  if (DIAG) acc.block_reduce_store(p.partials);
}

}  // namespace elbm

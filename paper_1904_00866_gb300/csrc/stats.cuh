// Fused per-step diagnostics: per-thread accumulation, warp-shuffle and
// shared-memory block reduction into one row of partials per block, then a
// single-block finish kernel that sums the rows in a fixed order (the result
// does not depend on scheduling).
#pragma once
#include <math.h>

#include "node_fp64.cuh"

namespace elbm {

// Partial slots.  Slots [0, S_NSUM) are sums, the rest min / max.
enum {
  S_DRHO = 0,   // sum (rho - rho0)
  S_J0, S_J1, S_J2,
  S_KE,         // 1/2 sum |j|^2 / rho
  S_ASUM,
  S_H,          // sum H(f)      (CHECK)
  S_NODES,
  S_ACC2, S_ACCSTAR, S_FORMULA, S_BAND, S_FAR, S_DEGEN,
  S_ITERS, S_CAP, S_NOROOT,
  S_VIOL, S_MISMATCH,  // (CHECK)
  S_NSUM,
  S_AMIN = S_NSUM,
  S_AMAX,
  S_ADEV,       // max |alpha - alpha_FP64|   (CHECK)
  NSTAT
};

struct Acc {
  double drho, j0, j1, j2, ke, asum, h;
  double amin, amax, adev;
  unsigned nodes, acc2, accstar, formula, band, far, degen, iters, cap,
      noroot, viol, mismatch;

  __device__ __forceinline__ void init() {
    drho = j0 = j1 = j2 = ke = asum = h = 0.0;
    amin = INFINITY;
    amax = -INFINITY;
    adev = 0.0;
    nodes = acc2 = accstar = formula = band = far = degen = iters = cap =
        noroot = viol = mismatch = 0u;
  }
  __device__ __forceinline__ void add_moments(double dr, const double* j,
                                              double rho) {
    drho += dr;
    j0 += j[0];
    j1 += j[1];
    j2 += j[2];
    ke += 0.5 * (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / rho;
  }
  __device__ __forceinline__ void add_alpha(double a, unsigned flags, int it) {
    nodes += 1;
    asum += a;
    amin = fmin(amin, a);
    amax = fmax(amax, a);
    acc2 += (flags & NF_ACCEPT_TWO) != 0;
    accstar += (flags & NF_ACCEPT_STAR) != 0;
    formula += (flags & NF_FORMULA) != 0;
    band += (flags & NF_BAND) != 0;
    degen += (flags & NF_DEGENERATE) != 0;
    cap += (flags & NF_ROOT_CAP) != 0;
    noroot += (flags & NF_NO_ROOT) != 0;
    iters += (unsigned)it;
  }
  __device__ __forceinline__ void add_check(double hf, bool v, bool mis,
                                            double dev) {
    h += hf;
    viol += v;
    mismatch += mis;
    adev = fmax(adev, dev);
  }

  __device__ __forceinline__ double slot(int k) const {
    switch (k) {
      case S_DRHO: return drho;
      case S_J0: return j0;
      case S_J1: return j1;
      case S_J2: return j2;
      case S_KE: return ke;
      case S_ASUM: return asum;
      case S_H: return h;
      case S_NODES: return nodes;
      case S_ACC2: return acc2;
      case S_ACCSTAR: return accstar;
      case S_FORMULA: return formula;
      case S_BAND: return band;
      case S_FAR: return far;
      case S_DEGEN: return degen;
      case S_ITERS: return iters;
      case S_CAP: return cap;
      case S_NOROOT: return noroot;
      case S_VIOL: return viol;
      case S_MISMATCH: return mismatch;
      case S_AMIN: return amin;
      case S_AMAX: return amax;
      default: return adev;
    }
  }

  // Reduce over the block and write partials[blockIdx.x * NSTAT + k].
  // Must be reached by every thread of the block.
  __device__ __forceinline__ void block_reduce_store(double* partials) {
    __shared__ double sm[32][NSTAT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NSTAT; ++k) {
      double v = slot(k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = k < S_NSUM ? v + w : (k == S_AMIN ? fmin(v, w) : fmax(v, w));
      }
      if (lane == 0) sm[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NSTAT) {
      const int k = threadIdx.x;
      double v = sm[0][k];
      for (int w = 1; w < nw; ++w) {
        const double x = sm[w][k];
        v = k < S_NSUM ? v + x : (k == S_AMIN ? fmin(v, x) : fmax(v, x));
      }
      partials[(long long)blockIdx.x * NSTAT + k] = v;
    }
  }
};

}  // namespace elbm

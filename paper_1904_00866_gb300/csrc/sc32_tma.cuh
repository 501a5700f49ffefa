// FP32-shifted FORMULA stream-collide with bulk-copy (TMA) row staging, for
// lattices whose x extent is a multiple of 256.
//
// A tile is 256 consecutive x-nodes of one (y, z) row.  For every population
// i the pull source x - c_i of the whole tile lies in one row of array i:
// one elected thread copies the aligned 1 KB segment [x0, x0 + 256) of that
// row into shared memory with cp.async.bulk, plus -- for the 18 (or 6)
// populations shifted by +-1 in x -- a 16-byte halo block holding x0 - 1
// or x0 + 256 (wrapped periodically).  Thread t then reads its value at
// offset 4 + t - c_ix of the population's shared row.  Compared with per-
// thread gathers this issues 45 copy instructions per 256 nodes instead of
// 6,912 and never fetches a row's edge sector twice.
//
// Completion is tracked by one mbarrier per stage of a 3-stage ring; the
// last warp to release a stage refills it, so there is no block-wide barrier
// in the loop.  On GB300 this variant reads exactly the algorithmic bytes
// but runs at about three quarters of the per-thread cp.async gather's
// throughput (its warps stall on the row copies' completion), so it is an
// opt-in alternative rather than the default.  Every wait is bounded: after kWaitLimit polls the warp
// records NF_TIMEOUT in the error word, waits (bounded again) for the copies
// in flight and leaves.
#pragma once
#include <stdint.h>

#include "sc32.cuh"

namespace elbm {

constexpr int kTmaRow = 4 + 256 + 4;   // halo | tile | halo (floats)
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_addr(m)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(float* dst, const float* src,
                                         unsigned bytes, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(m))
      : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait for one phase of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m,
                                                  unsigned parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

template <class L>
__host__ __device__ constexpr unsigned tma_tile_bytes() {
  unsigned shifted = 0;
  for (int i = 0; i < L::Q; ++i) shifted += L::c(i, 0) != 0;
  return L::Q * 256u * 4u + shifted * 16u;
}

template <class L>
__device__ __forceinline__ void tma_produce(const StepParams& p, float* stage,
                                            uint64_t* mbar, unsigned tile) {
  const unsigned chunks = (unsigned)p.nx / 256u;
  const unsigned row = tile / chunks;
  const int x0 = (int)(tile - row * chunks) * 256;
  const int y = (int)(row % (unsigned)p.ny);
  const int z = (int)(row / (unsigned)p.ny);
  const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
  const int xl = x0 == 0 ? p.nx - 4 : x0 - 4;            // left halo block
  const int xr = x0 + 256 == p.nx ? 0 : x0 + 256;         // right halo block
  mbar_expect_tx(mbar, tma_tile_bytes<L>());
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int ys = cy == 1 ? ym : (cy == -1 ? yp : y);
    const int zs = cz == 1 ? zm : (cz == -1 ? zp : z);
    const float* src =
        p.in_pop[i] + ((size_t)zs * (size_t)p.ny + (size_t)ys) * (size_t)p.nx;
    float* dst = stage + i * kTmaRow;
    bulk_g2s(dst + 4, src + x0, 1024u, mbar);
    if (cx == 1) bulk_g2s(dst, src + xl, 16u, mbar);        // holds x0 - 1
    if (cx == -1) bulk_g2s(dst + 260, src + xr, 16u, mbar); // holds x0 + 256
  }
}

// Stages of the shared-memory ring.  A stage is refilled by the last warp
// that finishes reading it (a per-stage release counter), so warps never
// meet at a block-wide barrier inside the loop.
constexpr int kTmaStages = 3;

template <class L, int DIAG, int CHECK>
__global__ void __launch_bounds__(256, 2) k_sc32_tma(const StepParams p) {
  constexpr int Q = L::Q;
  constexpr int S = kTmaStages;
  constexpr int kWarps = 256 / 32;
  extern __shared__ __align__(128) float smem[];   // [S][Q][kTmaRow]
  __shared__ __align__(8) uint64_t full[S];
  __shared__ unsigned released[S];
  const unsigned chunks = (unsigned)p.nx / 256u;
  const unsigned ntiles = chunks * (unsigned)p.ny * (unsigned)p.nz;
  const float rho0f = p.rho0f;
  const float beta = p.betaf;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      released[st] = 0u;
    }
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < S; ++k) {
      const unsigned t = blockIdx.x + (unsigned)k * gridDim.x;
      if (t < ntiles) tma_produce<L>(p, smem + k * Q * kTmaRow, &full[k], t);
    }
  }
  Acc32 acc;
  if (DIAG) acc.init();
  bool timed_out = false;
  unsigned k = 0;
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int st = (int)(k % S);
    const unsigned parity = (k / S) & 1u;
    if (!mbar_wait_bounded(&full[st], parity)) {
      if (lane == 0) atomicOr(p.err_flags, NF_TIMEOUT);
      timed_out = true;
      break;
    }
    const float* sm = smem + st * Q * kTmaRow + 4 + threadIdx.x;
    const unsigned row = tile / chunks;
    const unsigned node = row * (unsigned)p.nx +
                          (tile - row * chunks) * 256u + threadIdx.x;
    // gather this node's inputs before releasing the stage
    float v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = sm[i * kTmaRow - L::c(i, 0)];
    __syncwarp();
    if (lane == 0) {
      // release: this warp's shared reads precede the count; acquire: the
      // last warp's refill follows every other warp's reads
      __threadfence_block();
      const unsigned done = atomicAdd(&released[st], 1u) + 1u;
      if (done == kWarps) {
        // last reader of this stage: refill it with tile k + S
        released[st] = 0u;
        __threadfence_block();
        const unsigned t = tile + (unsigned)S * gridDim.x;
        if (t < ntiles) {
          fence_proxy_async();
          tma_produce<L>(p, smem + st * Q * kTmaRow, &full[st], t);
        }
      }
    }
    float ap = 0.0f;   // this variant sends undecided nodes to the queue
    const unsigned res = sc32_node_in<L, true, DIAG, CHECK>(
        [&](int i) { return v[i]; }, rho0f, p.rho0, beta, 0.0f, nullptr,
        p.alpha_map ? p.alpha_map + node : nullptr, acc,
        [&](int i, float val) { p.out_pop[i][node] = val; },
        p.exact ? &ap : nullptr);
    if (res != kNodeDone) {
      // one atomic per node: a warp whose bounded wait ran out may leave
      // the loop lane by lane, so no warp-wide vote here
      const unsigned slot = atomicAdd(&p.far_count[p.parity], 1u);
      if (slot < p.far_cap)
        p.far_queue[slot] = node | (res == kNodeRefine ? kTagRefine : 0u);
      else
        atomicOr(p.err_flags, NF_BAD_NONFINITE);   // cannot happen: cap = n
    }
  }
  if (timed_out) {
    // drain: bounded waits for the copies still in flight; every warp still
    // reaches the block reduction below (the other warps' waits are bounded
    // too, so they get there as well)
    for (int st = 0; st < S; ++st) mbar_wait_bounded(&full[st], 0u);
  }
  if (threadIdx.x == 0 && p.refine_counts) p.refine_counts[blockIdx.x] = 0u;
  if (DIAG) store_acc32(acc, p.partials);
}

}  // namespace elbm

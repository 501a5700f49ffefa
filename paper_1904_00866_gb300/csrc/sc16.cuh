// Pipelined FP16-shifted FORMULA stream-collide kernel: the k_sc32 scheme
// (Eq. (5b) pull gather, Eq. (5a) relax, certified FP32 entropy decision,
// FP64 fixup queue for far nodes) on binary16 storage of the scaled
// deviations (f_i - W_i rho0) 2^k_i.
//
// cp.async moves at least 4 bytes, so each gather copies the aligned 4-byte
// word that holds the source element into shared memory; the thread keeps a
// 27-bit mask of which half of each word is its element.  Neighbouring
// lanes fetch the same words, which the coalescer merges, so the DRAM
// traffic is the binary16 array itself: Q x 2 bytes read and written per
// node.  Stores are 2-byte coalesced writes.
#pragma once
#include "fp16_storage.cuh"
#include "sc32.cuh"

namespace elbm {

// Issue the word gathers of one tile; returns the upper-half mask.
template <class L>
__device__ __forceinline__ unsigned issue_tile16(const StepParams& p,
                                                 unsigned* sm, unsigned tile) {
  const unsigned node = tile * kSc32Threads + threadIdx.x;
  if (node >= (unsigned)p.n) return 0u;
  int x, y, z;
  node_xyz<L>(p, node, x, y, z);
  const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
  unsigned upper = 0u;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int xs = cx == 1 ? xm : (cx == -1 ? xp : x);
    const int ys = cy == 1 ? ym : (cy == -1 ? yp : y);
    const int zs = cz == 1 ? zm : (cz == -1 ? zp : z);
    const unsigned off = ((unsigned)zs * (unsigned)p.ny + (unsigned)ys) *
                             (unsigned)p.nx + (unsigned)xs;
    const unsigned* words = reinterpret_cast<const unsigned*>(p.in_pop[i]);
    cp_async4(reinterpret_cast<float*>(sm + i * kSc32Threads + threadIdx.x),
              reinterpret_cast<const float*>(words + (off >> 1)));
    upper |= (off & 1u) << i;
  }
  return upper;
}

template <class L, int DIAG, int CHECK>
__global__ void __launch_bounds__(kSc32Threads, 2)
    k_sc16(const StepParams p) {
  constexpr int Q = L::Q;
  extern __shared__ unsigned smem_w[];   // [2][Q][256] words
  const unsigned ntiles = (unsigned)((p.n + kSc32Threads - 1) / kSc32Threads);
  const float rho0f = p.rho0f;
  const float beta = p.betaf;
  Acc32 acc;
  if (DIAG) acc.init();
  __shared__ unsigned s_refine;     // this block's undecided-node entries
  refine_block_begin(&s_refine);

  unsigned tile = blockIdx.x;
  int stage = 0;
  unsigned upper_cur = 0u;
  if (tile < ntiles) upper_cur = issue_tile16<L>(p, smem_w, tile);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const unsigned next = tile + gridDim.x;
    unsigned upper_next = 0u;
    if (next < ntiles)
      upper_next =
          issue_tile16<L>(p, smem_w + (stage ^ 1) * Q * kSc32Threads, next);
    cp_async_commit();
    cp_async_wait<1>();   // this thread's copies of `tile` have landed

    const unsigned node = tile * kSc32Threads + threadIdx.x;
    const unsigned* sm = smem_w + stage * Q * kSc32Threads + threadIdx.x;
    const unsigned upper = upper_cur;
    upper_cur = upper_next;
    stage ^= 1;
    // stored values: the decoded deviations
    auto in = [&](int i) {
      const unsigned w = sm[i * kSc32Threads];
      const unsigned sh = ((upper >> i) & 1u) << 4;
      return h16_dev<L>((unsigned short)(w >> sh), i);
    };
    unsigned st = kNodeDone;
    float ap = 0.0f;
    if (node < (unsigned)p.n)
      st = sc32_node_in<L, true, DIAG, CHECK>(
          in, rho0f, p.rho0, beta, 0.0f, nullptr,
          p.alpha_map ? p.alpha_map + node : nullptr, acc,
          [&](int i, float v) {
            reinterpret_cast<unsigned short*>(p.out_pop[i])[node] =
                h16_bits<L>(v, i);
          },
          p.exact ? &ap : nullptr);
    if (p.exact)
      defer_undecided<L>(p, &s_refine, st == kNodeRefine, in, node, ap);
    defer_nodes(&p.far_count[p.parity], p.far_queue, p.far_cap, p.err_flags,
                node, st == kNodeFar ? kNodeFar : kNodeDone);
  }
  cp_async_wait<0>();
  refine_block_end(p, &s_refine);
  if (DIAG) store_acc32(acc, p.partials);
}

}  // namespace elbm

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

// Outcome of the FP32 stage of one node in the stream-collide kernels.
enum : unsigned {
  kNodeDone = 0u,     // collided and stored
  kNodeFar = 1u,      // far from equilibrium or invalid: FP64 fixup
  kNodeRefine = 2u    // FP32 decision not certified: second stage in the
                      // fixup kernel (double-float, FP64 as a last resort)
};
// Deferred-node queue entries carry the node index; this bit marks the
// entries due for the second stage.  Node indices stay below 2^31.
constexpr unsigned kTagRefine = 0x80000000u;

// Deviations delta_i of a node from its stored values in(i): the values
// themselves for shifted storage, v_i - fl(W_i rho0) for plain FP32
// storage (exact unless v_i leaves [s_i / 2, 2 s_i]; a_extra bounds the
// resulting error of x_i).
template <class L, bool SHIFTED, class In>
__device__ __forceinline__ void load_deviations(In in, float rho0f, float& d0,
                                                float2 (&dd)[npairs<L>()],
                                                float& a_extra) {
  constexpr int P = npairs<L>();
  {
    const float v = in(0);
    d0 = SHIFTED ? v : v - L::wf(0) * rho0f;
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const float2 v = make_float2(in(2 * k + 1), in(2 * k + 2));
    dd[k] = SHIFTED ? v : sub2(v, f2(L::wf(2 * k + 1) * rho0f));
  }
  a_extra = 0.0f;
  if (!SHIFTED) {
    float A = fabsf(d0);
#pragma unroll
    for (int k = 0; k < P; ++k) A += fabsf(dd[k].x) + fabsf(dd[k].y);
    a_extra = 2.0f * 5.9604645e-8f * A / rho0f;
  }
}

// Relaxation with the conservation-projected n, f~ = f + alpha beta n
// (Eq. (1)), stored through out(i, value) as the storage's value.
template <class L, bool SHIFTED, class Out>
__device__ __forceinline__ void relax_store32(const N32<L>& r, float d0,
                                              const float2 (&dd)[npairs<L>()],
                                              float rho0f, float beta,
                                              Out out) {
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
}

// The second stage's correction of a node written with the provisional
// alpha ap: the populations relaxed with the decided alpha ae (same n, same
// operations), stored through out(i, value) only where they differ from
// the provisional ones (most differ by less than the storage rounding).
template <class L, bool SHIFTED, class Out>
__device__ __forceinline__ void relax_update32(const N32<L>& r, float ap,
                                               float ae, float d0,
                                               const float2 (&dd)[npairs<L>()],
                                               float rho0f, float beta,
                                               Out out) {
  const float abp = ap * beta, abe = ae * beta;
  projection<L>(
      r,
      [&](float wt) {
        const float m = r.n0 - wt;
        float vp = fmaf(abp, m, d0), ve = fmaf(abe, m, d0);
        if (!SHIFTED) {
          vp += L::wf(0) * rho0f;
          ve += L::wf(0) * rho0f;
        }
        if (ve != vp) out(0, ve);
      },
      [&](int k, float2 wt) {
        const float2 m = sub2(r.n2[k], wt);
        float2 vp = fma2(f2(abp), m, dd[k]), ve = fma2(f2(abe), m, dd[k]);
        if (!SHIFTED) {
          vp = add2(vp, f2(L::wf(2 * k + 1) * rho0f));
          ve = add2(ve, f2(L::wf(2 * k + 1) * rho0f));
        }
        if (ve.x != vp.x) out(2 * k + 1, ve.x);
        if (ve.y != vp.y) out(2 * k + 2, ve.y);
      });
}

// FP64 entropy check (Eq. (7)) of a node given its stored values in(i), at
// the alpha used.
template <class L, bool SHIFTED, class In>
__device__ __forceinline__ Check64 check32(In in, double rho0, float alpha,
                                           Node64<L>& nd) {
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double v = (double)in(i);
    nd.f[i] = SHIFTED ? L::w(i) * rho0 + v : v;
  }
  node64_prepare(nd);
  return node64_check(nd, (double)alpha);
}

// Statistics of one collided node (FP32 accumulators).
template <class L, bool SHIFTED, int CHECK, class In>
__device__ __forceinline__ void diag32(const N32<L>& r, In in, double rho0,
                                       Acc32& acc) {
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
    const Check64 ck = check32<L, SHIFTED>(in, rho0, r.alpha, nd);
    acc.h += ck.h;
    acc.viol += ck.violation;
    acc.mismatch += decision_mismatch(r.flags, ck.accept_ref);
    acc.adev = fmax(acc.adev, fabs((double)r.alpha - ck.alpha_ref));
  }
}

// Collision of one node whose Q gathered values are returned by in(i)
// (shared memory).  Writes the Q post-collision values through
// out(i, value) and the alpha through amap (nullable).  Returns kNodeDone;
// kNodeRefine for a node whose FP32 decision is undecided when the caller
// runs the second stage (aprov non-null: populations written with the
// certified alpha, stored in *aprov; no statistics or alpha map -- the
// second stage completes the node); or kNodeFar (nothing written: the FP64
// fixup collides it).  With aprov null an undecided node keeps its
// certified alpha.
template <class L, bool SHIFTED, int DIAG, int CHECK, class In, class Out>
__device__ __forceinline__ unsigned sc32_node_in(
    In in, float rho0f, double rho0, float beta, float corr_rho,
    const float* __restrict__ corr, float* amap, Acc32& acc, Out out,
    float* aprov = nullptr) {
  constexpr int P = npairs<L>();
  float d0, a_extra;
  float2 dd[P];
  load_deviations<L, SHIFTED>(in, rho0f, d0, dd, a_extra);
  N32<L> r;
  node32_formula<L, SHIFTED>(d0, dd, rho0f, corr_rho, corr, a_extra, r,
                             aprov != nullptr);
  if (r.flags & NF_FAR) return kNodeFar;
  // every other node writes all its populations now (whole write sectors)
  relax_store32<L, SHIFTED>(r, d0, dd, rho0f, beta, out);
  if (r.flags & NF_REFINE) {
    if (aprov) {   // the second stage completes the node
      *aprov = r.alpha;
      return kNodeRefine;
    }
    // without a second stage the certified alpha is final
    r.flags = (r.flags & NF_DEGENERATE) ? NF_DEGENERATE : NF_FORMULA | NF_BAND;
  }
  if (amap) *amap = r.alpha;
  if (DIAG) diag32<L, SHIFTED, CHECK>(r, in, rho0, acc);
  return kNodeDone;
}

// Second stage of one undecided node from its stored values in(i), after
// the stream-collide kernel wrote it with the provisional alpha ap (NaN when
// unknown: then the FP32 stage is run again to recover it): the
// double-float decision (node32_refine), then the populations relaxed with
// the decided alpha where they differ from the provisional ones, the alpha
// map and the statistics.  Both relaxations use the double-float n, so a
// population the decided alpha does not change at storage precision keeps
// the provisional value, which differs from it by at most the rounding of
// the FP32 n.  Returns kStageDone, kStageRetry (still undecided by the FP32
// series on the double-float n: the DFS pass, which also evaluates the
// leading terms in double-float, may decide it) or kStageFP64 (left to the
// FP64 path, which rewrites all of it).  Nothing is written unless done.
enum { kStageDone = 0, kStageRetry = 1, kStageFP64 = 2 };
template <class L, bool SHIFTED, int DIAG, int CHECK, bool DFS, class In,
          class Out, class Stat>
__device__ __forceinline__ int second_stage32(In in, float rho0f, float beta,
                                              float corr_rho,
                                              const float* __restrict__ corr,
                                              float* amap, float ap, Out out,
                                              Stat stat) {
  constexpr int P = npairs<L>();
  float d0, a_extra;
  float2 dd[P];
  load_deviations<L, SHIFTED>(in, rho0f, d0, dd, a_extra);
  if (!(ap == ap)) {
    N32<L> r;
    node32_formula<L, SHIFTED>(d0, dd, rho0f, corr_rho, corr, a_extra, r,
                               true);
    ap = r.alpha;
  }
  N32<L> t;
  t.flags = 0u;
  t.alpha = 1.0f;
  node32_refine<L, SHIFTED, DFS>(d0, dd, rho0f, corr_rho, corr, a_extra, t);
  if (t.flags & NF_FAR)
    return (t.flags & NF_REFINE) ? kStageRetry : kStageFP64;
  if (t.alpha != ap)
    relax_update32<L, SHIFTED>(t, ap, t.alpha, d0, dd, rho0f, beta, out);
  if (amap) *amap = t.alpha;
  stat(t);
  return kStageDone;
}

// Buffer of undecided nodes for the second stage: one record of
// refine_record<L>() floats per node (its Q stored values, its key and its
// provisional alpha, padded to 16 bytes: 128 bytes for D3Q27), written by
// the stream-collide kernels as whole 16-byte vectors and read by the
// second-stage kernel; a node that finds its block's segment full goes to
// the deferred-node queue tagged kTagRefine (the fixup then gathers it
// from f_in).  Every lane of the warp calls; `mine` marks an undecided
// node, in(i) its stored values, ap its provisional alpha.


// Append the deferred nodes of a warp to the fixup queue with one atomic
// per warp (every lane of the warp must call; st = kNodeDone for lanes
// with nothing to defer).  The warp's entries are contiguous, so the
// fixup's neighbouring threads gather neighbouring nodes.
__device__ __forceinline__ void defer_nodes(unsigned* count, unsigned* queue,
                                            unsigned cap, unsigned* err,
                                            unsigned node, unsigned st) {
  const unsigned mask = __ballot_sync(0xffffffffu, st != kNodeDone);
  if (mask == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned base = 0u;
  if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (st != kNodeDone) {
    const unsigned slot = base + (unsigned)__popc(mask & ((1u << lane) - 1u));
    if (slot < cap)
      queue[slot] = node | (st == kNodeRefine ? kTagRefine : 0u);
    else
      atomicOr(err, NF_BAD_NONFINITE);   // cannot happen: cap = n
  }
}

// Same, with the values in a shared-memory column of stride TB.
template <class L, bool SHIFTED, int DIAG, int CHECK, int TB, class Out>
__device__ __forceinline__ unsigned sc32_node(const float* sm, float rho0f,
                                          double rho0, float beta,
                                          float corr_rho,
                                          const float* __restrict__ corr,
                                          float* amap, Acc32& acc, Out out,
                                          float* aprov = nullptr) {
  return sc32_node_in<L, SHIFTED, DIAG, CHECK>(
      [&](int i) { return sm[i * TB]; }, rho0f, rho0, beta, corr_rho, corr,
      amap, acc, out, aprov);
}

template <class L, class In>
__device__ __forceinline__ void defer_undecided(const StepParams& p,
                                                unsigned* block_count,
                                                bool mine, In in,
                                                unsigned node, float ap) {
  const unsigned seg = p.refine_cap / gridDim.x;   // this block's segment
  if (seg == 0u) {   // no buffer: the tagged queue and a gather
    defer_nodes(&p.far_count[p.parity], p.far_queue, p.far_cap, p.err_flags,
                node, mine ? kNodeRefine : kNodeDone);
    return;
  }
  const unsigned m = __ballot_sync(0xffffffffu, mine);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0u;
  if (lane == leader) base = atomicAdd(block_count, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  bool over = false;
  if (mine) {
    const unsigned slot = base + (unsigned)__popc(m & ((1u << lane) - 1u));
    if (slot < seg) {
      // one record of refine_record<L>() floats, written as 16-byte vectors
      float4* rec = reinterpret_cast<float4*>(
          p.refine_buf +
          ((size_t)blockIdx.x * seg + slot) * (size_t)refine_record<L>());
      auto val = [&](int k) {
        return k < L::Q ? in(k)
                        : (k == L::Q ? __uint_as_float(node)
                                     : (k == L::Q + 1 ? ap : 0.0f));
      };
#pragma unroll
      for (int j = 0; j < refine_record<L>() / 4; ++j)
        rec[j] = make_float4(val(4 * j), val(4 * j + 1), val(4 * j + 2),
                             val(4 * j + 3));
    } else {
      over = true;
    }
  }
  // a full segment: the tagged queue (one atomic per warp; after
  // initialisation nearly every node of the first step lands here)
  defer_nodes(&p.far_count[p.parity], p.far_queue, p.far_cap, p.err_flags,
              node, over ? kNodeRefine : kNodeDone);
}

// Exclusive prefix sums pre[0..n] of counts[0..n-1] (n <= kMaxRefineBlocks)
// in shared memory, computed by the whole block (blockDim.x a multiple of
// 32, at most 1024): each thread sums a run of consecutive counts, the run
// totals are scanned with warp shuffles and once more across the warps.
// Every thread of the block must call; ends with a block barrier.
__device__ __forceinline__ void block_prefix(const unsigned* counts, int n,
                                             unsigned* pre) {
  __shared__ unsigned warp_tot[32];
  const int T = blockDim.x, t = threadIdx.x;
  const int run = (n + T - 1) / T;   // <= 8 for n <= 2048, T = 256
  const int b0 = t * run;
  unsigned sum = 0u;
  for (int k = 0; k < run; ++k)
    if (b0 + k < n) sum += counts[b0 + k];
  // inclusive scan of the run totals within the warp
  const int lane = t & 31, w = t >> 5;
  unsigned inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int nw = T >> 5;
    unsigned v = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) warp_tot[lane] = v;   // inclusive over the warps
  }
  __syncthreads();
  unsigned acc = inc - sum + (w > 0 ? warp_tot[w - 1] : 0u);
  for (int k = 0; k < run; ++k)
    if (b0 + k < n) {
      pre[b0 + k] = acc;
      acc += counts[b0 + k];
    }
  if (t == T - 1) pre[n] = warp_tot[(T >> 5) - 1];
  __syncthreads();
}

// Block prologue / epilogue of the buffer: the block's entry counter in
// shared memory starts at zero; at the end the number of entries the block
// wrote goes to refine_counts[blockIdx.x] (0 when unused).
__device__ __forceinline__ void refine_block_begin(unsigned* block_count) {
  if (threadIdx.x == 0) *block_count = 0u;
  __syncthreads();
}
__device__ __forceinline__ void refine_block_end(const StepParams& p,
                                                 const unsigned* block_count) {
  __syncthreads();
  if (threadIdx.x == 0 && p.refine_counts)
    p.refine_counts[blockIdx.x] = min(*block_count, p.refine_cap / gridDim.x);
}

// D2Q9 nodes need about half the registers of D3Q27 nodes: more resident
// blocks keep more gathers in flight (4 per SM, 3 with the statistics)
template <class L, bool SHIFTED, int DIAG, int CHECK>
__global__ void __launch_bounds__(kSc32Threads,
                                  L::Q == 9 ? (DIAG ? 3 : 4) : 2)
    k_sc32(const StepParams p) {
  constexpr int Q = L::Q;
  extern __shared__ float smem[];   // [2][Q][256]
  __shared__ unsigned s_refine;     // this block's undecided-node entries
  const unsigned ntiles = (unsigned)((p.n + kSc32Threads - 1) / kSc32Threads);
  const float rho0f = p.rho0f;
  const float beta = p.betaf;
  Acc32 acc;
  if (DIAG) acc.init();
  refine_block_begin(&s_refine);

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
    unsigned st = kNodeDone;
    float ap = 0.0f;
    if (node < (unsigned)p.n)
      st = sc32_node<L, SHIFTED, DIAG, CHECK, kSc32Threads>(
          sm, rho0f, p.rho0, beta, p.corr_rho, p.corr,
          p.alpha_map ? p.alpha_map + node : nullptr, acc,
          [&](int i, float v) { p.out_pop[i][node] = v; },
          p.exact ? &ap : nullptr);
    // undecided (written with the certified alpha): the second stage
    // decides
    if (p.exact)
      defer_undecided<L>(p, &s_refine, st == kNodeRefine,
                         [&](int i) { return sm[i * kSc32Threads]; }, node,
                         ap);
    // far from equilibrium or invalid: the FP64 fixup collides these nodes
    // from f_in
    defer_nodes(&p.far_count[p.parity], p.far_queue, p.far_cap, p.err_flags,
                node, st == kNodeFar ? kNodeFar : kNodeDone);
  }
  cp_async_wait<0>();
  refine_block_end(p, &s_refine);
  if (DIAG) store_acc32(acc, p.partials);
}

}  // namespace elbm

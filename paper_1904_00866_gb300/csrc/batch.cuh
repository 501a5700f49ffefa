// Batched stream-collide over many independent periodic lattices in one
// persistent launch (FP32-shifted storage, FORMULA).
//
// Members may differ in lattice type (D2Q9 / D3Q27), size and viscosity.
// Each member's lattice is cut into tiles of TB consecutive nodes; the tiles
// of all stepping members form one flat list whose prefix offsets and
// per-tile member index live in device memory, so a launch (or a captured
// CUDA graph of launches) reads the current membership at run time.  The
// per-tile index replaces a per-thread binary search over the prefix (a
// chain of dependent shared-memory loads on every node).  Blocks walk the list with a grid
// stride and the same cp.async double-buffered gather / shared-memory
// compute as the single-lattice kernel; a tile's block switches on its
// member's lattice type (uniform per block).
//
// A burst is a sequence of steps s = 0, 1, ...; member m takes part in
// steps s < steps_left(m) and reads buf[(parity0 + s) & 1], writes the other
// buffer; its tiles are skipped in later steps of the burst.  Members with
// no steps left are left out of the tile list.
#pragma once
#include <stdint.h>

#include "fixup.cuh"

namespace elbm {

constexpr int kBatchMaxMembers = 256;

struct __align__(16) MemberDesc {
  float* buf[2];        // FP32-shifted pull-layout populations (select with
                        // pick(): a runtime index would force local memory)
  float* alpha_map;     // nullable
  unsigned n;           // nodes
  int nx, ny, nz;
  FastDiv div_nx, div_ny;
  float beta;
  float rho0f;
  double rho0;
  double beta64;        // beta of Eq. (2) in FP64 (far-node fixup)
  int lattice;          // 0: D2Q9, 1: D3Q27
  int parity0;          // buffer holding f^n at burst step 0
  int steps_left;       // steps of this burst the member takes
  int diag;             // accumulate statistics on its last burst step
};

// Per-member statistics of one step (atomically accumulated).
struct MemberStats {
  double drho, j0, j1, j2, ke, asum;
  unsigned long long nodes, acc2, formula, band, degen, far;
  unsigned amin_bits, amax_bits;   // positive floats: integer order
};

struct BatchParams {
  const MemberDesc* members;
  const unsigned* tile_begin;   // [count + 1] tile prefix of the members
  const unsigned char* tile_member;   // [tiles] member of each tile
  int desc_cap;                 // member descriptors staged in shared memory
                                // (>= count; fixes the launch's smem size)
  const int* count;             // members in the tile list
  MemberStats* stats;           // [kBatchMaxMembers]
  unsigned long long* far_queue;   // (member << 32) | node
  unsigned far_cap;
  unsigned* far_count;          // [2]
  unsigned* err_flags;
  int step;                     // step index within the burst
  // undecided nodes for the second stage: records of kBatchRecord floats
  // (the member's Q stored values from float 0, then node and member index
  // as bits and the provisional alpha at floats 28, 29, 30); block b of a
  // launch of G blocks owns the segment of refine_cap / G records from
  // b (refine_cap / G) on and writes how many it used to refine_counts[b]
  float* refine_buf;
  unsigned refine_cap;
  unsigned* refine_counts;
  int exact;                    // 0: undecided nodes keep the certified alpha
};
constexpr int kBatchRecord = 32;   // floats per undecided-node record

__device__ __forceinline__ float* pick(const MemberDesc& m, int parity) {
  return (parity & 1) ? m.buf[1] : m.buf[0];
}

template <class L, int TB>
__device__ __forceinline__ void batch_issue(const MemberDesc& m, int step,
                                            float* sm, unsigned local) {
  const unsigned node = local * TB + threadIdx.x;
  if (node >= m.n) return;
  const unsigned q1 = m.div_nx.div(node);
  const int x = (int)(node - q1 * (unsigned)m.nx);
  const unsigned q2 = m.div_ny.div(q1);
  const int y = (int)(q1 - q2 * (unsigned)m.ny), z = (int)q2;
  const int xm = x == 0 ? m.nx - 1 : x - 1, xp = x == m.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? m.ny - 1 : y - 1, yp = y == m.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? m.nz - 1 : z - 1, zp = z == m.nz - 1 ? 0 : z + 1;
  const float* in = pick(m, m.parity0 + step);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int xs = cx == 1 ? xm : (cx == -1 ? xp : x);
    const int ys = cy == 1 ? ym : (cy == -1 ? yp : y);
    const int zs = cz == 1 ? zm : (cz == -1 ? zp : z);
    const unsigned off =
        ((unsigned)zs * (unsigned)m.ny + (unsigned)ys) * (unsigned)m.nx +
        (unsigned)xs;
    cp_async4(sm + i * TB + threadIdx.x, in + off);
    in += m.n;   // next population array
  }
}

// Block reduction of one tile's statistics into the member's record.
template <int TB>
__device__ __forceinline__ void batch_tile_stats(const Acc32& a,
                                                 MemberStats* st) {
  __shared__ double red[TB / 32][6];
  __shared__ unsigned long long redc[TB / 32][5];
  __shared__ float redm[TB / 32][2];
  double v[6] = {a.drho.value(), a.j0.value(), a.j1.value(), a.j2.value(),
                 a.ke.value(), a.asum.value()};
  unsigned long long c[5] = {a.nodes, a.acc2, a.formula, a.band, a.degen};
  float mn = a.amin, mx = a.amax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
#pragma unroll
    for (int k = 0; k < 5; ++k) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) red[w][k] = v[k];
#pragma unroll
    for (int k = 0; k < 5; ++k) redc[w][k] = c[k];
    redm[w][0] = mn;
    redm[w][1] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int ww = 1; ww < TB / 32; ++ww) {
      for (int k = 0; k < 6; ++k) red[0][k] += red[ww][k];
      for (int k = 0; k < 5; ++k) redc[0][k] += redc[ww][k];
      redm[0][0] = fminf(redm[0][0], redm[ww][0]);
      redm[0][1] = fmaxf(redm[0][1], redm[ww][1]);
    }
    if (redc[0][0] > 0) {
      atomicAdd(&st->drho, red[0][0]);
      atomicAdd(&st->j0, red[0][1]);
      atomicAdd(&st->j1, red[0][2]);
      atomicAdd(&st->j2, red[0][3]);
      atomicAdd(&st->ke, red[0][4]);
      atomicAdd(&st->asum, red[0][5]);
      atomicAdd(&st->nodes, redc[0][0]);
      atomicAdd(&st->acc2, redc[0][1]);
      atomicAdd(&st->formula, redc[0][2]);
      atomicAdd(&st->band, redc[0][3]);
      atomicAdd(&st->degen, redc[0][4]);
      atomicMin(&st->amin_bits, __float_as_uint(redm[0][0]));
      atomicMax(&st->amax_bits, __float_as_uint(redm[0][1]));
    }
  }
  __syncthreads();
}

template <int TB, int DIAG>
__global__ void __launch_bounds__(TB, 2048 / TB / 4)
    k_batch(const BatchParams bp) {
  extern __shared__ __align__(16) float smem[];   // [2][27][TB], descs
  __shared__ unsigned s_begin[kBatchMaxMembers + 1];
  // the member descriptors are read on every tile: stage them in shared
  // memory once (word copy; MemberDesc is trivially copyable)
  MemberDesc* s_desc = reinterpret_cast<MemberDesc*>(smem + 2 * 27 * TB);
  __shared__ unsigned s_refine;   // this block's undecided-node entries
  if (threadIdx.x == 0) s_refine = 0u;
  const unsigned seg = bp.refine_cap / gridDim.x;
  const int count = *bp.count;
  for (int k = threadIdx.x; k <= count; k += TB) s_begin[k] = bp.tile_begin[k];
  {
    constexpr int W = (int)(sizeof(MemberDesc) / sizeof(unsigned));
    const unsigned* src = reinterpret_cast<const unsigned*>(bp.members);
    unsigned* dst = reinterpret_cast<unsigned*>(s_desc);
    const int words = min(count, bp.desc_cap) * W;
    for (int k = threadIdx.x; k < words; k += TB) dst[k] = src[k];
  }
  __syncthreads();
  const unsigned total = s_begin[count];
  constexpr int kStage = 27 * TB;

  unsigned tile = blockIdx.x;
  int stage = 0;
  auto issue = [&](unsigned t, int mi, float* sm) {
    const MemberDesc m = s_desc[mi];   // by value: no reloads after stores
    if (bp.step >= m.steps_left) return;   // member finished in this burst
    const unsigned local = t - s_begin[mi];
    if (m.lattice == 1)
      batch_issue<D3Q27, TB>(m, bp.step, sm, local);
    else
      batch_issue<D2Q9, TB>(m, bp.step, sm, local);
  };
  // member indices of this tile and the next are carried in registers; the
  // one after is loaded an iteration ahead (the table streams from L2)
  int mi_cur = tile < total ? bp.tile_member[tile] : 0;
  int mi_next = tile + gridDim.x < total ? bp.tile_member[tile + gridDim.x] : 0;
  if (tile < total) issue(tile, mi_cur, smem);
  cp_async_commit();
  for (; tile < total; tile += gridDim.x) {
    const unsigned next = tile + gridDim.x, after = next + gridDim.x;
    const int mi_after = after < total ? bp.tile_member[after] : 0;
    if (next < total) issue(next, mi_next, smem + (stage ^ 1) * kStage);
    cp_async_commit();
    cp_async_wait<1>();
    const float* sm = smem + stage * kStage + threadIdx.x;
    stage ^= 1;

    const int mi = mi_cur;
    mi_cur = mi_next;
    mi_next = mi_after;
    const MemberDesc m = s_desc[mi];   // by value: no reloads after stores
    if (bp.step >= m.steps_left) continue;   // uniform per block
    const unsigned node = (tile - s_begin[mi]) * TB + threadIdx.x;
    const bool stats_step = DIAG && m.diag && bp.step == m.steps_left - 1;
    Acc32 acc;
    if (DIAG) acc.init();
    unsigned res = kNodeDone;
    float ap = 0.0f;
    if (node < m.n) {
      float* out = pick(m, m.parity0 + bp.step + 1);
      float* amap = m.alpha_map ? m.alpha_map + node : nullptr;
      auto store = [&](int i, float v) { out[(size_t)i * m.n + node] = v; };
      if (m.lattice == 1)
        res = sc32_node<D3Q27, true, DIAG, 0, TB>(sm, m.rho0f, m.rho0, m.beta,
                                                  0.0f, nullptr, amap, acc,
                                                  store,
                                                  bp.exact ? &ap : nullptr);
      else
        res = sc32_node<D2Q9, true, DIAG, 0, TB>(sm, m.rho0f, m.rho0, m.beta,
                                                 0.0f, nullptr, amap, acc,
                                                 store,
                                                 bp.exact ? &ap : nullptr);
    }
    {
      // undecided nodes (written provisionally) into the second-stage
      // buffer, one atomic per warp (every lane gets here: the member is
      // uniform per block); a full buffer sends them to the tagged queue
      const unsigned um = __ballot_sync(0xffffffffu, res == kNodeRefine);
      if (um != 0u) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(um) - 1;
        unsigned base = 0u;
        if (lane == leader) base = atomicAdd(&s_refine, (unsigned)__popc(um));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (res == kNodeRefine) {
          const unsigned slot =
              base + (unsigned)__popc(um & ((1u << lane) - 1u));
          if (slot < seg) {
            float4* rec = reinterpret_cast<float4*>(
                bp.refine_buf +
                ((size_t)blockIdx.x * seg + slot) * (size_t)kBatchRecord);
            const int q = m.lattice == 1 ? 27 : 9;
            auto val = [&](int k) { return k < q ? sm[k * TB] : 0.0f; };
            for (int j = 0; j < (q + 3) / 4; ++j)
              rec[j] = make_float4(val(4 * j), val(4 * j + 1), val(4 * j + 2),
                                   val(4 * j + 3));
            rec[7] = make_float4(__uint_as_float(node),
                                 __uint_as_float((unsigned)mi), ap, 0.0f);
            res = kNodeDone;
          }
        }
      }
    }
    {
      // deferred nodes, one atomic per warp
      const unsigned mask = __ballot_sync(0xffffffffu, res != kNodeDone);
      if (mask != 0u) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(mask) - 1;
        unsigned base = 0u;
        if (lane == leader)
          base = atomicAdd(&bp.far_count[bp.step & 1], (unsigned)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (res != kNodeDone) {
          const unsigned slot =
              base + (unsigned)__popc(mask & ((1u << lane) - 1u));
          if (slot < bp.far_cap)
            bp.far_queue[slot] =
                ((unsigned long long)mi << 32) |
                (node | (res == kNodeRefine ? kTagRefine : 0u));
          else
            atomicOr(bp.err_flags, NF_BAD_NONFINITE);   // cannot happen
        }
      }
    }
    if (DIAG) {
      // uniform per block: the whole tile belongs to member mi
      if (stats_step) batch_tile_stats<TB>(acc, bp.stats + mi);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  if (threadIdx.x == 0) bp.refine_counts[blockIdx.x] = min(s_refine, seg);
}

// Statistics of one node collided by a fixup kernel, added to its member's
// record (on the member's statistics step).
__device__ __forceinline__ void member_stats_add(const BatchParams& bp, int mi,
                                                 const MemberDesc& m,
                                                 const Acc& acc, bool fp64) {
  if (!(m.diag && bp.step == m.steps_left - 1 && acc.nodes > 0)) return;
  MemberStats* st = bp.stats + mi;
  atomicAdd(&st->drho, acc.drho);
  atomicAdd(&st->j0, acc.j0);
  atomicAdd(&st->j1, acc.j1);
  atomicAdd(&st->j2, acc.j2);
  atomicAdd(&st->ke, acc.ke);
  atomicAdd(&st->asum, acc.asum);
  atomicAdd(&st->nodes, 1ull);
  if (fp64) atomicAdd(&st->far, 1ull);
  atomicAdd(&st->acc2, (unsigned long long)acc.acc2);
  atomicAdd(&st->formula, (unsigned long long)acc.formula);
  atomicAdd(&st->band, (unsigned long long)acc.band);
  atomicAdd(&st->degen, (unsigned long long)acc.degen);
  const float a = (float)acc.asum;
  atomicMin(&st->amin_bits, __float_as_uint(a));
  atomicMax(&st->amax_bits, __float_as_uint(a));
}

// Second stage of the undecided nodes the batch kernel (`blocks` blocks)
// buffered, two blocks per SM; a node it leaves undecided joins the
// deferred-node queue for the fixup that follows (tagged when the
// double-float series pass may still decide it).
template <int DIAG>
__global__ void __launch_bounds__(256, 2) k_batch_refine(const BatchParams bp,
                                                         int blocks) {
  __shared__ unsigned pre[kMaxRefineBlocks + 1];
  block_prefix(bp.refine_counts, blocks, pre);
  const unsigned total = pre[blocks];
  const unsigned seg = bp.refine_cap / (unsigned)blocks;
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
    const float4* rec = reinterpret_cast<const float4*>(
        bp.refine_buf + ((size_t)lo * seg + (k - pre[lo])) * (size_t)kBatchRecord);
    const float4 tail = rec[7];
    const unsigned node = __float_as_uint(tail.x);
    const int mi = (int)__float_as_uint(tail.y);
    const float ap = tail.z;
    const MemberDesc& m = bp.members[mi];
    float* out = pick(m, m.parity0 + bp.step + 1);
    StepParams pp;
    pp.beta = m.beta64;
    pp.rho0 = m.rho0;
    pp.betaf = m.beta;
    pp.rho0f = m.rho0f;
    pp.alpha_map = m.alpha_map;
    pp.unshifted = 0;
    pp.corr_rho = 0.0f;
    Acc acc;
    acc.init();
    auto run = [&](auto lat) {
      using L = decltype(lat);
      float v[L::Q + 3];
#pragma unroll
      for (int j = 0; j < (L::Q + 3) / 4; ++j) {
        const float4 t = rec[j];
        v[4 * j] = t.x;
        if (4 * j + 1 < L::Q + 3) v[4 * j + 1] = t.y;
        if (4 * j + 2 < L::Q + 3) v[4 * j + 2] = t.z;
        if (4 * j + 3 < L::Q + 3) v[4 * j + 3] = t.w;
      }
      float (&vq)[L::Q] = *reinterpret_cast<float (*)[L::Q]>(v);
      auto out32 = [&](int i, float val) { out[(size_t)i * m.n + node] = val; };
      return refine_deferred<L, true, DIAG, 0, false>(pp, vq, node, ap, acc,
                                                      out32);
    };
    const int st = m.lattice == 1 ? run(D3Q27{}) : run(D2Q9{});
    if (st != kStageDone) {
      // kStageRetry: tagged, so that the fixup (whose register budget
      // holds it) runs the double-float series pass before any FP64
      const unsigned q = atomicAdd(&bp.far_count[bp.step & 1], 1u);
      if (q < bp.far_cap)
        bp.far_queue[q] = ((unsigned long long)mi << 32) |
                          (node | (st == kStageRetry ? kTagRefine : 0u));
      else
        atomicOr(bp.err_flags, NF_BAD_NONFINITE);   // cannot happen
    } else if (DIAG) {
      member_stats_add(bp, mi, m, acc, false);
    }
  }
}

// FP64 fixup of the batch kernel's deferred-node queue (values gathered
// from the member's buffer): the second stage for entries tagged
// kTagRefine (a full buffer segment), one entry per thread, then the FP64
// FORMULA for the nodes that need it, one node per warp
// (formula64_warp); entries are dealt as in k_far_fixup.  Clears the other
// parity's counter for the next step.
template <int DIAG>
__global__ void __launch_bounds__(256) k_batch_fixup(const BatchParams bp) {
  const unsigned count = min(bp.far_count[bp.step & 1], bp.far_cap);
  const int lane = threadIdx.x & 31;
  const unsigned W = gridDim.x * (blockDim.x >> 5);
  const unsigned wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const LanePop lp27 = lane_pop<D3Q27>(lane), lp9 = lane_pop<D2Q9>(lane);
  const bool bulk = count > gridDim.x * blockDim.x;
  auto coords = [](const MemberDesc& m, unsigned node, int& x, int& y,
                   int& z) {
    x = (int)(node % (unsigned)m.nx);
    y = (int)((node / (unsigned)m.nx) % (unsigned)m.ny);
    z = (int)(node / ((unsigned)m.nx * (unsigned)m.ny));
  };
  auto params = [&](const MemberDesc& m) {
    StepParams pp;
    pp.beta = m.beta64;
    pp.rho0 = m.rho0;
    pp.betaf = m.beta;
    pp.rho0f = m.rho0f;
    pp.err_flags = bp.err_flags;
    pp.secant_iters = 1;
    pp.alpha_map = m.alpha_map;
    pp.unshifted = 0;
    pp.corr_rho = 0.0f;
    return pp;
  };
  // FP64 FORMULA of queue entry ee in this thread
  auto fp64_lane = [&](unsigned long long ee) {
    const int mi = (int)(ee >> 32);
    const unsigned node = (unsigned)(ee & 0xffffffffu) & ~kTagRefine;
    const MemberDesc& m = bp.members[mi];
    const float* in = pick(m, m.parity0 + bp.step);
    float* out = pick(m, m.parity0 + bp.step + 1);
    StepParams g;   // geometry for src_index
    g.nx = m.nx;
    g.ny = m.ny;
    g.nz = m.nz;
    int x, y, z;
    coords(m, node, x, y, z);
    Acc acc;
    acc.init();
    const StepParams pp = params(m);
    auto run = [&](auto lat) {
      using L = decltype(lat);
      Node64<L> nd;
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        nd.f[i] = L::w(i) * m.rho0 +
                  (double)in[(size_t)i * m.n + src_index<L>(g, i, x, y, z)];
      auto store = [&](int i, double val) {
        if (i < 0)
          m.alpha_map[node] = (float)val;
        else
          out[(size_t)i * m.n + node] = (float)(val - L::w(i) * m.rho0);
      };
      collide64<L, MODE_FORMULA, 0>(nd, pp, true, acc, DIAG != 0, store);
    };
    if (m.lattice == 1)
      run(D3Q27{});
    else
      run(D2Q9{});
    if (DIAG) member_stats_add(bp, mi, m, acc, true);
  };
  // FP64 FORMULA of queue entry ee by the whole warp (every lane calls)
  auto fp64_warp = [&](unsigned long long ee) {
    const int mi = (int)(ee >> 32);
    const unsigned node = (unsigned)(ee & 0xffffffffu) & ~kTagRefine;
    const MemberDesc& m = bp.members[mi];
    const float* in = pick(m, m.parity0 + bp.step);
    float* out = pick(m, m.parity0 + bp.step + 1);
    int x, y, z;
    coords(m, node, x, y, z);
    auto run = [&](auto lat, const LanePop& lp) {
      using L = decltype(lat);
      double f = 0.0;
      if (lp.on) {
        int xs = x - lp.c[0], ys = y - lp.c[1], zs = z - lp.c[2];
        xs = xs < 0 ? xs + m.nx : (xs >= m.nx ? xs - m.nx : xs);
        ys = ys < 0 ? ys + m.ny : (ys >= m.ny ? ys - m.ny : ys);
        zs = zs < 0 ? zs + m.nz : (zs >= m.nz ? zs - m.nz : zs);
        const size_t src =
            ((size_t)zs * (size_t)m.ny + (size_t)ys) * (size_t)m.nx +
            (size_t)xs;
        f = lp.w * m.rho0 + (double)in[(size_t)lane * m.n + src];
      }
      return formula64_warp<L>(lp, f, m.beta64, [&](double val) {
        out[(size_t)lane * m.n + node] = (float)(val - lp.w * m.rho0);
      });
    };
    const Warp64 r = m.lattice == 1 ? run(D3Q27{}, lp27) : run(D2Q9{}, lp9);
    if (lane == 0) {
      if (r.flags & (NF_BAD_NEG | NF_BAD_NONFINITE)) {
        atomicOr(bp.err_flags, r.flags);
      } else {
        if (m.alpha_map) m.alpha_map[node] = (float)r.alpha;
        if (DIAG) {
          Acc acc;
          acc.init();
          acc.add_moments(r.rho - m.rho0, r.j, r.rho);
          acc.add_alpha(r.alpha, r.flags, 0);
          member_stats_add(bp, mi, m, acc, true);
        }
      }
    }
  };
  __shared__ unsigned long long pend_s[8][32];   // 256 threads: 8 warps
  unsigned long long* pend = pend_s[threadIdx.x >> 5];
  int npend = 0;
  auto flush = [&]() {   // every lane calls
    __syncwarp();
    if (lane < npend) fp64_lane(pend[lane]);
    __syncwarp();
    npend = 0;
  };
  for (unsigned base = 0; base < count; base += 32u * W) {
    const unsigned k = base + (unsigned)lane * W + wid;
    bool need64 = false;
    unsigned long long e = 0;
    if (k < count) {
      e = bp.far_queue[k];
      const int mi = (int)(e >> 32);
      const unsigned tagged = (unsigned)(e & 0xffffffffu);
      const unsigned node = tagged & ~kTagRefine;
      need64 = true;
      if (tagged & kTagRefine) {
        const MemberDesc& m = bp.members[mi];
        const float* in = pick(m, m.parity0 + bp.step);
        float* out = pick(m, m.parity0 + bp.step + 1);
        StepParams g;   // geometry for src_index
        g.nx = m.nx;
        g.ny = m.ny;
        g.nz = m.nz;
        int x, y, z;
        coords(m, node, x, y, z);
        Acc acc;
        acc.init();
        const StepParams pp = params(m);
        auto run = [&](auto lat) {
          using L = decltype(lat);
          float v[L::Q];
#pragma unroll
          for (int i = 0; i < L::Q; ++i)
            v[i] = in[(size_t)i * m.n + src_index<L>(g, i, x, y, z)];
          auto store32 = [&](int i, float val) {
            out[(size_t)i * m.n + node] = val;
          };
          const float nan = __int_as_float(0x7fc00000);
          int st = refine_deferred<L, true, DIAG, 0, false>(pp, v, node, nan,
                                                            acc, store32);
          // as in k_far_fixup: no series pass on a queue longer than the grid
          if (st == kStageRetry && !bulk)
            st = refine_deferred<L, true, DIAG, 0, true>(pp, v, node, nan,
                                                         acc, store32);
          return st == kStageDone;
        };
        need64 = !(m.lattice == 1 ? run(D3Q27{}) : run(D2Q9{}));
        if (DIAG && !need64) member_stats_add(bp, mi, m, acc, false);
      }
    }
    // FP64 nodes of this round, as in k_far_fixup: one per warp for a few,
    // one per lane for many; a queue longer than the grid (new members'
    // first steps) collects them per warp and runs them 32 at a time
    const unsigned todo = __ballot_sync(0xffffffffu, need64);
    if (!bulk && __popc(todo) > 16) {
      if (need64) fp64_lane(e);
    } else if (bulk) {
      const int nk = __popc(todo);
      if (npend + nk > 32) flush();
      if (need64) pend[npend + __popc(todo & ((1u << lane) - 1u))] = e;
      npend += nk;
    } else {
      unsigned m = todo;
      while (m) {
        const int src_lane = __ffs(m) - 1;
        m &= m - 1;
        fp64_warp(__shfl_sync(0xffffffffu, e, src_lane));
      }
    }
  }
  if (npend > 0) {   // bulk remainder: few nodes run one per warp
    __syncwarp();
    if (npend > 5) {
      flush();
    } else {
      for (int j = 0; j < npend; ++j) fp64_warp(pend[j]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) bp.far_count[(bp.step & 1) ^ 1] = 0u;
}

}  // namespace elbm

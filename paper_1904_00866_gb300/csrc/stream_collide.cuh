// Fused pull-scheme stream + collide kernel (Eq. (5b) gather, Eq. (5a)
// relax) for one periodic lattice.
//
// Storage: SoA populations [Q][nz][ny][nx], x fastest.  The buffer holds the
// post-collision values f~ of the previous step; the pre-collision state at
// node x is the gather f_i(x) = f~_i(x - c_i), so each population array is
// read once and written once per step (HBM traffic 2 Q sizeof(T) per node).
//
// Work decomposition: a tile is 32 consecutive x-nodes of one (y, z) row,
// one warp per tile; warps stride over tiles (grid sized to the SM count).
// The 27 (or 9) gathers of a tile are warp-coalesced 128-byte rows; the
// +-1 x-shift of a row is absorbed by L1/L2.
//
// Template parameters: lattice L, storage type T (double: FP64 arithmetic
// for every alpha mode; float / half_t: FP32 or FP16-shifted storage with
// ROOT / SECANT in FP64 -- their FORMULA runs in the pipelined k_sc32 /
// k_sc16), alpha MODE, DIAG (fused statistics), CHECK (FP64 entropy check;
// implies DIAG).
#pragma once
#include <stdint.h>

#include "fp16_storage.cuh"
#include "lattice.cuh"
#include "node_fp64.cuh"
#include "stats.cuh"

namespace elbm {

// Division by a runtime-invariant 32-bit divisor d >= 1 by multiply-high
// and shifts (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994): q = (t + ((n - t) >> s1)) >> s2, t = mulhi(m, n),
// with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, s1 = min(l, 1),
// s2 = max(l - 1, 0).  Exact for every n < 2^32.
struct FastDiv {
  unsigned m;
  int s1, s2;
  __host__ void init(unsigned d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    m = (unsigned)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    s1 = l < 1 ? l : 1;
    s2 = l > 1 ? l - 1 : 0;
  }
  __device__ __forceinline__ unsigned div(unsigned n) const {
    const unsigned t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// Largest stream-collide grid whose undecided-node buffer segments the
// second stage reads (8 resident blocks on each of up to 256 SMs).
constexpr int kMaxRefineBlocks = 2048;

// Floats per record of the undecided-node buffer: the Q stored values,
// the node key and the provisional alpha, padded to whole 16-byte vectors
// (32 = 128 bytes for D3Q27, 12 for D2Q9).
template <class L>
__host__ __device__ constexpr int refine_record() {
  return (L::Q + 2 + 3) / 4 * 4;
}

struct StepParams {
  const void* f_in;
  void* f_out;
  float* alpha_map;       // nullptr: not written this step
  double* partials;       // [gridDim.x][NSTAT] when DIAG
  unsigned* err_flags;    // OR of NF_BAD_* over the lattice
  int nx, ny, nz;
  int chunks;             // ceil(nx / 32)
  long long n;            // nodes
  long long ps;           // population stride in elements (n, or n padded
                          // to a multiple of 64 for FP16 storage)
  long long tiles;        // chunks * ny * nz
  double beta;
  double rho0;            // shift reference (0 for FP64 storage)
  // the same rounded to FP32 on the host: a kernel that converted them
  // itself could repeat the conversion (an FP64-pipe instruction) per node
  // to save the registers
  float betaf, rho0f;
  int unshifted;          // FP32 storage of f itself (not f - W rho0)
  float corr_rho;         // unshifted: sum_i fl(W_i rho0) - rho0
  float corr[27];         // unshifted: W_i rho0 - fl(W_i rho0)
  int secant_iters;
  unsigned* far_count;    // [2] deferred-node counters, indexed by parity
  unsigned* far_queue;    // node indices deferred to the FP64 fixup
  unsigned far_cap;       // capacity of far_queue (entries)
  int parity;             // step parity selecting far_count[parity]
  FastDiv div_nx, div_ny; // node -> (x, y, z)
  // FP32 / FP16 storage: f_in + i ps and f_out + i ps, per population (for
  // FP16 the pointers address binary16 arrays; the kernels cast them)
  const float* in_pop[27];
  float* out_pop[27];
  // Second stage of undecided FP32 decisions (exact: 1; certified: 0, the
  // certified alpha is final).  Its buffer holds refine_cap records
  // (stored values, node key, provisional alpha); block b of a
  // stream-collide launch of G blocks owns the segment of
  // refine_cap / G records from b (refine_cap / G) on and writes how many
  // it used to refine_counts[b].
  int exact;
  float* refine_buf;
  unsigned refine_cap;    // 0: no buffer (undecided nodes use the queue)
  unsigned* refine_counts;
};

template <class L>
__device__ __forceinline__ void tile_coords(const StepParams& p, long long t,
                                            int lane, int& x, int& y, int& z) {
  const long long row = t / p.chunks;
  const int chunk = (int)(t - row * p.chunks);
  x = chunk * 32 + lane;
  y = (int)(row % p.ny);
  z = (int)(row / p.ny);
}

// Flat index of the pull source x - c_i of population i.
template <class L>
__device__ __forceinline__ long long src_index(const StepParams& p, int i,
                                               int x, int y, int z) {
  const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
  int xs = x - cx, ys = y - cy, zs = z - cz;
  xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
  ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
  zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
  return ((long long)zs * p.ny + ys) * p.nx + xs;
}

// FP64 collision of one node from FP64 populations f64; writes the new
// populations through `store(i, value)`.
template <class L, int MODE, int CHECK, class Store>
__device__ __forceinline__ void collide64(Node64<L>& nd, const StepParams& p,
                                          bool round_alpha_down, Acc& acc,
                                          bool diag, Store store) {
  unsigned flags = node64_prepare(nd);
  int iters = 0;
  double alpha = 2.0;
  if (flags) {
    atomicOr(p.err_flags, flags);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) store(i, nd.f[i]);
    return;
  }
  alpha = node64_alpha<L, MODE>(nd, p.secant_iters, flags, iters);
  if (round_alpha_down) alpha = (double)__double2float_rd(alpha);
  const double ab = alpha * p.beta;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) store(i, fma(ab, nd.f[i] * nd.x[i], nd.f[i]));
  if (diag) {
    acc.add_moments(nd.rho - p.rho0, nd.j, nd.rho);
    acc.add_alpha(alpha, flags, iters);
    if (CHECK) {
      Check64 ck = node64_check(nd, alpha);
      acc.add_check(ck.h, ck.violation,
                    decision_mismatch(flags, ck.accept_ref),
                    fabs(alpha - ck.alpha_ref));
    }
  }
  if (p.alpha_map) store(-1, alpha);
}

template <class L, class T, int MODE, int DIAG, int CHECK>
__global__ void __launch_bounds__(256)
    k_stream_collide(const StepParams p) {
  constexpr int Q = L::Q;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const T* __restrict__ fin = static_cast<const T*>(p.f_in);
  T* __restrict__ fout = static_cast<T*>(p.f_out);
  Acc acc;
  acc.init();

  for (long long t = warp0; t < p.tiles; t += nwarps) {
    int x, y, z;
    tile_coords<L>(p, t, lane, x, y, z);
    if (x >= p.nx) continue;
    const long long node = ((long long)z * p.ny + y) * p.nx + x;

    T v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = fin[(long long)i * p.ps + src_index<L>(p, i, x, y, z)];

    auto store_T = [&](int i, double val) {
      if (i < 0) {
        p.alpha_map[node] = (float)val;
      } else {
        fout[(long long)i * p.ps + node] = (T)val;
      }
    };

    if constexpr (sizeof(T) == 8) {
      // ---------------- FP64 storage: FP64 arithmetic -------------------
      Node64<L> nd;
#pragma unroll
      for (int i = 0; i < Q; ++i) nd.f[i] = (double)v[i];
      collide64<L, MODE, CHECK>(nd, p, false, acc, DIAG != 0, store_T);
    } else if constexpr (MODE != MODE_FORMULA) {
      // ------------- FP32 storage, ROOT / SECANT in FP64 -----------------
      Node64<L> nd;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double s = L::w(i) * p.rho0;
        if constexpr (sizeof(T) == 2)
          nd.f[i] = h16_to_f<L>(v[i], i, p.rho0);
        else
          nd.f[i] = p.unshifted ? (double)v[i] : s + (double)v[i];
      }
      auto store_s = [&](int i, double val) {
        if (i < 0) {
          p.alpha_map[node] = (float)val;
        } else {
          const double s = L::w(i) * p.rho0;
          if constexpr (sizeof(T) == 2)
            fout[(long long)i * p.ps + node] = h16_from_dev<L>(val - s, i);
          else
            fout[(long long)i * p.ps + node] =
                (T)(p.unshifted ? val : val - s);
        }
      };
      collide64<L, MODE, CHECK>(nd, p, true, acc, DIAG != 0, store_s);
    } else {
      static_assert(sizeof(T) == 8 || MODE != MODE_FORMULA,
                    "FP32 / FP16 FORMULA runs in k_sc32 / k_sc16");
    }
  }
  if (DIAG) acc.block_reduce_store(p.partials);
}

}  // namespace elbm

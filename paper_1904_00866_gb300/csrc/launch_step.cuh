// Launch helpers for the stream-collide kernels; each translation unit
// instantiates the subset it owns so the kernels compile in parallel.
#pragma once
#include "fixup.cuh"
#include "internal.h"
#include "sc16.cuh"
#include "sc32.cuh"
#include "sc32_tma.cuh"
#include "sc32w.cuh"

#include <stdlib.h>
#include <string.h>

#include <atomic>

namespace elbm {

// Raise a kernel's dynamic shared-memory limit once per device (the
// attribute belongs to the device's context; `done` is per kernel
// instantiation, one bit per device ordinal, safe under concurrent calls).
template <class Kernel>
static cudaError_t set_smem_limit(Kernel k, int bytes,
                                  std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(
      k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

template <class Kernel>
static int occupancy_grid(Kernel k, int block, long long threads_needed) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, 0);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2048 / block) per_sm = 2048 / block;   // partials rows bound
  long long g = (long long)sms * per_sm;
  const long long need = (threads_needed + block - 1) / block;
  if (need < g) g = need;
  return g < 1 ? 1 : (int)g;
}

template <class L, class T, int MODE, int DIAG, int CHECK>
static cudaError_t launch_one(const StepParams& p, int grid, int block,
                              cudaStream_t s, int* grid_used) {
  auto k = k_stream_collide<L, T, MODE, DIAG, CHECK>;
  if (grid <= 0) grid = occupancy_grid(k, block, p.tiles * 32);
  if (grid_used) *grid_used = grid;
  k<<<grid, block, 0, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <class L, class T, int MODE>
static cudaError_t launch_diag(int diag, int check, const StepParams& p,
                               int grid, int block, cudaStream_t s,
                               int* grid_used) {
  if (check) return launch_one<L, T, MODE, 1, 1>(p, grid, block, s, grid_used);
  if (diag) return launch_one<L, T, MODE, 1, 0>(p, grid, block, s, grid_used);
  return launch_one<L, T, MODE, 0, 0>(p, grid, block, s, grid_used);
}

template <class L, class T>
static cudaError_t launch_fp64_modes(int mode, int diag, int check,
                                     const StepParams& p, int grid, int block,
                                     cudaStream_t s, int* grid_used) {
  if (mode == MODE_ROOT)
    return launch_diag<L, T, MODE_ROOT>(diag, check, p, grid, block, s,
                                        grid_used);
  if (mode == MODE_SECANT)
    return launch_diag<L, T, MODE_SECANT>(diag, check, p, grid, block, s,
                                          grid_used);
  return launch_diag<L, T, MODE_FORMULA>(diag, check, p, grid, block, s,
                                         grid_used);
}

// Pipelined FP32 FORMULA kernel (dynamic shared memory: 2 stages x Q x 256).
template <class L, bool SHIFTED, int DIAG, int CHECK>
static cudaError_t launch_sc32_one(const StepParams& p, int grid,
                                   cudaStream_t s, int* grid_used) {
  auto k = k_sc32<L, SHIFTED, DIAG, CHECK>;
  const int smem = 2 * L::Q * kSc32Threads * (int)sizeof(float);
  static std::atomic<unsigned long long> configured{0};   // per instantiation
  const cudaError_t se = set_smem_limit(k, smem, configured);
  if (se != cudaSuccess) return se;
  if (grid <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kSc32Threads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2048 / kSc32Threads) per_sm = 2048 / kSc32Threads;
    long long g = (long long)sms * per_sm;
    const long long tiles = (p.n + kSc32Threads - 1) / kSc32Threads;
    if (tiles < g) g = tiles;
    grid = g < 1 ? 1 : (int)g;
  }
  if (grid_used) *grid_used = grid;
  k<<<grid, kSc32Threads, smem, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <class L, bool SHIFTED>
static cudaError_t launch_sc32_s(int diag, int check, const StepParams& p,
                                 int grid, cudaStream_t s, int* grid_used) {
  if (check) return launch_sc32_one<L, SHIFTED, 1, 1>(p, grid, s, grid_used);
  if (diag) return launch_sc32_one<L, SHIFTED, 1, 0>(p, grid, s, grid_used);
  return launch_sc32_one<L, SHIFTED, 0, 0>(p, grid, s, grid_used);
}

// Bulk-copy (TMA) row staging for FP32-shifted lattices with nx % 256 == 0.
template <class L, int DIAG, int CHECK>
static cudaError_t launch_tma_one(const StepParams& p, int grid,
                                  cudaStream_t s, int* grid_used) {
  auto k = k_sc32_tma<L, DIAG, CHECK>;
  const int smem = kTmaStages * L::Q * kTmaRow * (int)sizeof(float);
  static std::atomic<unsigned long long> configured{0};   // per instantiation
  const cudaError_t se = set_smem_limit(k, smem, configured);
  if (se != cudaSuccess) return se;
  if (grid <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    long long g = (long long)sms * per_sm;
    const long long tiles = p.n / 256;
    if (tiles < g) g = tiles;
    grid = g < 1 ? 1 : (int)g;
  }
  if (grid_used) *grid_used = grid;
  k<<<grid, 256, smem, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

// Wide-gather kernel for FP32-shifted lattices with nx % 64 == 0.
template <class L, int DIAG, int CHECK>
static cudaError_t launch_wide_one(const StepParams& p, int grid,
                                   cudaStream_t s, int* grid_used) {
  auto k = k_sc32w<L, DIAG, CHECK>;
  const int smem =
      kWideWarps * 2 * wide_stage_floats<L>() * (int)sizeof(float);
  static std::atomic<unsigned long long> configured{0};   // per instantiation
  const cudaError_t se = set_smem_limit(k, smem, configured);
  if (se != cudaSuccess) return se;
  if (grid <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWideThreads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;   // partials rows bound
    long long g = (long long)sms * per_sm;
    const long long blocks = (p.n / kWideSeg + kWideWarps - 1) / kWideWarps;
    if (blocks < g) g = blocks;
    grid = g < 1 ? 1 : (int)g;
  }
  if (grid_used) *grid_used = grid;
  k<<<grid, kWideThreads, smem, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

// Kernel variant for FP32-shifted lattices, chosen once per process by
// ELBM_SC32_VARIANT: "cpasync" (default; per-element gathers, any size),
// "wide" (16-byte row-segment gathers, nx % 64 == 0) or "tma" (bulk-copy
// row staging, nx % 256 == 0).  Both alternatives read exactly the
// algorithmic bytes but fit fewer warps per SM; on the D3Q27 512^3 workload
// "wide" ties with the default and "tma" runs about a quarter slower.
// Sizes a variant does not cover use the per-element kernel.
enum Sc32Variant { kVarCpAsync = 0, kVarWide = 1, kVarTma = 2 };
static int sc32_variant() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("ELBM_SC32_VARIANT");
    v = kVarCpAsync;
    if (e && strcmp(e, "wide") == 0) v = kVarWide;
    if (e && strcmp(e, "tma") == 0) v = kVarTma;
  }
  return v;
}

template <class L>
static cudaError_t launch_sc32(int diag, int check, const StepParams& p,
                               int grid, cudaStream_t s, int* grid_used) {
  if (p.unshifted)
    return launch_sc32_s<L, false>(diag, check, p, grid, s, grid_used);
  const int var = sc32_variant();
  if (var == kVarTma && p.nx % 256 == 0) {
    if (check) return launch_tma_one<L, 1, 1>(p, grid, s, grid_used);
    if (diag) return launch_tma_one<L, 1, 0>(p, grid, s, grid_used);
    return launch_tma_one<L, 0, 0>(p, grid, s, grid_used);
  }
  if (var == kVarWide && p.nx % kWideSeg == 0) {
    if (check) return launch_wide_one<L, 1, 1>(p, grid, s, grid_used);
    if (diag) return launch_wide_one<L, 1, 0>(p, grid, s, grid_used);
    return launch_wide_one<L, 0, 0>(p, grid, s, grid_used);
  }
  return launch_sc32_s<L, true>(diag, check, p, grid, s, grid_used);
}

// Pipelined FP16-shifted FORMULA kernel (dynamic shared memory: 2 stages x
// Q x 256 words).
template <class L, int DIAG, int CHECK>
static cudaError_t launch_sc16_one(const StepParams& p, int grid,
                                   cudaStream_t s, int* grid_used) {
  auto k = k_sc16<L, DIAG, CHECK>;
  const int smem = 2 * L::Q * kSc32Threads * (int)sizeof(unsigned);
  static std::atomic<unsigned long long> configured{0};   // per instantiation
  const cudaError_t se = set_smem_limit(k, smem, configured);
  if (se != cudaSuccess) return se;
  if (grid <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kSc32Threads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2048 / kSc32Threads) per_sm = 2048 / kSc32Threads;
    long long g = (long long)sms * per_sm;
    const long long tiles = (p.n + kSc32Threads - 1) / kSc32Threads;
    if (tiles < g) g = tiles;
    grid = g < 1 ? 1 : (int)g;
  }
  if (grid_used) *grid_used = grid;
  k<<<grid, kSc32Threads, smem, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <class L>
static cudaError_t launch_sc16(int diag, int check, const StepParams& p,
                               int grid, cudaStream_t s, int* grid_used) {
  if (check) return launch_sc16_one<L, 1, 1>(p, grid, s, grid_used);
  if (diag) return launch_sc16_one<L, 1, 0>(p, grid, s, grid_used);
  return launch_sc16_one<L, 0, 0>(p, grid, s, grid_used);
}

// The fixup grid must equal the grid of the FP32 / FP16 step when DIAG is
// set (its partials rows follow the step's rows); without DIAG any grid
// works.  S: storage type (float or half_t).
template <class L, class S = float>
static cudaError_t launch_far_lattice(int diag, int check,
                                      const StepParams& p, int grid,
                                      cudaStream_t s) {
  if (grid <= 0) grid = 152;
  if (check)
    k_far_fixup<L, S, 1, 1><<<grid, 256, 0, s>>>(p);
  else if (diag)
    k_far_fixup<L, S, 1, 0><<<grid, 256, 0, s>>>(p);
  else
    k_far_fixup<L, S, 0, 0><<<grid, 256, 0, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

// Second stage of the undecided nodes a stream-collide launch of `blocks`
// blocks buffered (S: storage type).
template <class L, class S = float>
static cudaError_t launch_refine_lattice(int diag, int check,
                                         const StepParams& p, int blocks,
                                         int grid, cudaStream_t s) {
  if (blocks > kMaxRefineBlocks) return cudaErrorInvalidValue;
  if (grid <= 0) grid = 152;
  if (check)
    k_refine_stage<L, S, 1, 1><<<grid, 256, 0, s>>>(p, blocks);
  else if (diag)
    k_refine_stage<L, S, 1, 0><<<grid, 256, 0, s>>>(p, blocks);
  else
    k_refine_stage<L, S, 0, 0><<<grid, 256, 0, s>>>(p, blocks);
  count_launch();
  return cudaGetLastError();
}

}  // namespace elbm

// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "stream_collide.cuh"

namespace elbm {

// Launch counter shared by all launch sites.
void count_launch();
void count_launches(long long n);

// Message returned by elbm_last_error(NULL) (thread-local).
void set_global_error(const std::string& msg);

// Sum `rows` partial rows (NSTAT doubles each) into out[NSTAT].
cudaError_t launch_finish(const double* partials, int rows, double* out,
                          cudaStream_t s);

// Public statistics record from the NSTAT reduced slots.
void stats_from_slots(const double* slots, double rho0, long long n,
                      long long step, int checked, void* out_stats);

// Per-translation-unit launchers.  grid <= 0 picks the occupancy-sized grid
// (SM count x resident blocks, capped by the work); *grid_used receives it.
#define ELBM_DECLARE_LAUNCHERS(LAT)                                          \
  cudaError_t launch_fp32_formula_##LAT(int diag, int check,                 \
                                        const StepParams& p, int grid,        \
                                        int block, cudaStream_t s,            \
                                        int* grid_used);                      \
  cudaError_t launch_far_##LAT(int diag, int check, const StepParams& p,     \
                               int grid, cudaStream_t s);                    \
  cudaError_t launch_fp32_fp64mode_##LAT(int mode, int diag, int check,      \
                                         const StepParams& p, int grid,       \
                                         int block, cudaStream_t s,           \
                                         int* grid_used);                     \
  cudaError_t launch_fp64_##LAT(int mode, int diag, int check,               \
                                const StepParams& p, int grid, int block,     \
                                cudaStream_t s, int* grid_used);              \
  cudaError_t launch_fp16_formula_##LAT(int diag, int check,                 \
                                        const StepParams& p, int grid,        \
                                        cudaStream_t s, int* grid_used);      \
  cudaError_t launch_far16_##LAT(int diag, int check, const StepParams& p,   \
                                 int grid, cudaStream_t s);                  \
  cudaError_t launch_refine_##LAT(int diag, int check, const StepParams& p,  \
                                  int blocks, int grid, cudaStream_t s);     \
  cudaError_t launch_refine16_##LAT(int diag, int check,                     \
                                    const StepParams& p, int blocks,         \
                                    int grid, cudaStream_t s);               \
  cudaError_t launch_fp16_fp64mode_##LAT(int mode, int diag, int check,      \
                                         const StepParams& p, int grid,       \
                                         int block, cudaStream_t s,           \
                                         int* grid_used);
ELBM_DECLARE_LAUNCHERS(d2q9)
ELBM_DECLARE_LAUNCHERS(d3q27)
#undef ELBM_DECLARE_LAUNCHERS

cudaError_t launch_fp64_d1q3(int mode, int diag, int check,
                             const StepParams& p, int grid, int block,
                             cudaStream_t s, int* grid_used);

}  // namespace elbm

// D1Q3: FP64-storage kernels (FP64 arithmetic, all alpha modes).  The
// one-dimensional lattice is offered with FP64 storage only.
#include "launch_step.cuh"
#include "lattice_d1q3.cuh"

namespace elbm {
cudaError_t launch_fp64_d1q3(int mode, int diag, int check, const StepParams& p,
                             int grid, int block, cudaStream_t s,
                             int* grid_used) {
  return launch_fp64_modes<D1Q3, double>(mode, diag, check, p, grid, block, s,
                                         grid_used);
}
}  // namespace elbm

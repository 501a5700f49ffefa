// D2Q9: FP32-storage certified FORMULA kernels and the FP64 far-node fixup.
#include "launch_step.cuh"

namespace elbm {
cudaError_t launch_fp32_formula_d2q9(int diag, int check, const StepParams& p,
                                      int grid, int block, cudaStream_t s,
                                      int* grid_used) {
  (void)block;
  return launch_sc32<D2Q9>(diag, check, p, grid, s, grid_used);
}
cudaError_t launch_far_d2q9(int diag, int check, const StepParams& p, int grid,
                             cudaStream_t s) {
  return launch_far_lattice<D2Q9>(diag, check, p, grid, s);
}
cudaError_t launch_refine_d2q9(int diag, int check, const StepParams& p,
                                int blocks, int grid, cudaStream_t s) {
  return launch_refine_lattice<D2Q9>(diag, check, p, blocks, grid, s);
}
}  // namespace elbm

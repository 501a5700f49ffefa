// D2Q9: FP16-shifted storage -- certified FORMULA kernel, its FP64
// far-node fixup, and ROOT / SECANT (FP64 arithmetic).
#include "launch_step.cuh"

namespace elbm {
cudaError_t launch_fp16_formula_d2q9(int diag, int check, const StepParams& p,
                                      int grid, cudaStream_t s,
                                      int* grid_used) {
  return launch_sc16<D2Q9>(diag, check, p, grid, s, grid_used);
}
cudaError_t launch_far16_d2q9(int diag, int check, const StepParams& p,
                               int grid, cudaStream_t s) {
  return launch_far_lattice<D2Q9, half_t>(diag, check, p, grid, s);
}
cudaError_t launch_fp16_fp64mode_d2q9(int mode, int diag, int check,
                                       const StepParams& p, int grid, int block,
                                       cudaStream_t s, int* grid_used) {
  if (mode == MODE_SECANT)
    return launch_diag<D2Q9, half_t, MODE_SECANT>(diag, check, p, grid, block,
                                                  s, grid_used);
  return launch_diag<D2Q9, half_t, MODE_ROOT>(diag, check, p, grid, block, s,
                                              grid_used);
}
cudaError_t launch_refine16_d2q9(int diag, int check, const StepParams& p,
                                  int blocks, int grid, cudaStream_t s) {
  return launch_refine_lattice<D2Q9, half_t>(diag, check, p, blocks, grid, s);
}
}  // namespace elbm

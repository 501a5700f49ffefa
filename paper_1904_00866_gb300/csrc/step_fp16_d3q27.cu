// D3Q27: FP16-shifted storage -- certified FORMULA kernel, its FP64
// far-node fixup, and ROOT / SECANT (FP64 arithmetic).
#include "launch_step.cuh"

namespace elbm {
cudaError_t launch_fp16_formula_d3q27(int diag, int check, const StepParams& p,
                                      int grid, cudaStream_t s,
                                      int* grid_used) {
  return launch_sc16<D3Q27>(diag, check, p, grid, s, grid_used);
}
cudaError_t launch_far16_d3q27(int diag, int check, const StepParams& p,
                               int grid, cudaStream_t s) {
  return launch_far_lattice<D3Q27, half_t>(diag, check, p, grid, s);
}
cudaError_t launch_fp16_fp64mode_d3q27(int mode, int diag, int check,
                                       const StepParams& p, int grid, int block,
                                       cudaStream_t s, int* grid_used) {
  if (mode == MODE_SECANT)
    return launch_diag<D3Q27, half_t, MODE_SECANT>(diag, check, p, grid, block,
                                                  s, grid_used);
  return launch_diag<D3Q27, half_t, MODE_ROOT>(diag, check, p, grid, block, s,
                                              grid_used);
}
cudaError_t launch_refine16_d3q27(int diag, int check, const StepParams& p,
                                  int blocks, int grid, cudaStream_t s) {
  return launch_refine_lattice<D3Q27, half_t>(diag, check, p, blocks, grid, s);
}
}  // namespace elbm

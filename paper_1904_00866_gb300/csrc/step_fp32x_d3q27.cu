// D3Q27: FP32-storage ROOT / SECANT kernels (FP64 arithmetic).
#include "launch_step.cuh"

namespace elbm {
cudaError_t launch_fp32_fp64mode_d3q27(int mode, int diag, int check,
                                       const StepParams& p, int grid, int block,
                                       cudaStream_t s, int* grid_used) {
  if (mode == MODE_SECANT)
    return launch_diag<D3Q27, float, MODE_SECANT>(diag, check, p, grid, block, s,
                                                   grid_used);
  return launch_diag<D3Q27, float, MODE_ROOT>(diag, check, p, grid, block, s,
                                               grid_used);
}
}  // namespace elbm

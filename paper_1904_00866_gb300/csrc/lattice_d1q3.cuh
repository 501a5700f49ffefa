// D1Q3 lattice descriptor (velocities {0, +1, -1}, weights {2/3, 1/6, 1/6},
// c_s^2 = 1/3), with the same members as the D2Q9 / D3Q27 descriptors.
#pragma once

// D1Q3 itself, for one-dimensional problems (the shock tube of Fig. 2);
// the library runs it with FP64 storage only.
struct D1Q3 {
  static constexpr int D = 1;
  static constexpr int Q = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    return a != 0 ? 0 : (i == 0 ? 0 : (i == 1 ? 1 : -1));
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0;
  }
  __host__ __device__ static constexpr float wf(int i) {
    return i == 0 ? 2.0f / 3.0f : 1.0f / 6.0f;
  }
  __host__ __device__ static constexpr int nonzero(int i) {
    return i != 0;
  }
  // round(log2(1 / W_i)): 1 for the rest population, 3 for the movers
  __host__ __device__ static constexpr float hscale(int i) {
    return i == 0 ? 2.0f : 8.0f;
  }
  __host__ __device__ static constexpr float hscale_inv(int i) {
    return i == 0 ? 0.5f : 0.125f;
  }
};

// Lattice descriptors for the sm_103a kernels.
//
// D2Q9 and D3Q27 are tensor products of D1Q3 (velocities {0, +1, -1},
// weights {2/3, 1/6, 1/6}, c_s^2 = 1/3).  Ordering follows the public ABI:
// rest first, then +/- pairs (index 2k-1 and 2k are opposite).  All members
// are constexpr so that, inside fully unrolled loops over i, every velocity
// component and weight is a compile-time constant.
#pragma once

struct D2Q9 {
  static constexpr int D = 2;
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},
                             {0, 1, 0},  {0, -1, 0},  {1, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    return t[i][a];
  }
  // product of the per-axis D1Q3 weights, (2/3)^(2-k) (1/6)^k for k
  // nonzero components; literal fractions fold to correctly rounded
  // constants at compile time
  __host__ __device__ static constexpr double w(int i) {
    return nonzero(i) == 0 ? 4.0 / 9.0
                           : (nonzero(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr float wf(int i) {
    return nonzero(i) == 0 ? 4.0f / 9.0f
                           : (nonzero(i) == 1 ? 1.0f / 9.0f : 1.0f / 36.0f);
  }
  __host__ __device__ static constexpr int nonzero(int i) {
    return (c(i, 0) != 0) + (c(i, 1) != 0) + (c(i, 2) != 0);
  }
  // binary16 storage scale 2^k_i, k_i = round(log2(1 / W_i)): the stored
  // value is (f_i - W_i rho0) 2^k_i, so every population class uses the
  // same part of the binary16 range; powers of two scale exactly
  __host__ __device__ static constexpr float hscale(int i) {
    return nonzero(i) == 0 ? 2.0f : (nonzero(i) == 1 ? 8.0f : 32.0f);
  }
  __host__ __device__ static constexpr float hscale_inv(int i) {
    return nonzero(i) == 0 ? 0.5f : (nonzero(i) == 1 ? 0.125f : 0.03125f);
  }
};

struct D3Q27 {
  static constexpr int D = 3;
  static constexpr int Q = 27;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[27][3] = {
        {0, 0, 0},    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
        {0, 0, 1},    {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
        {-1, 1, 0},   {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
        {0, 1, 1},    {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},
        {-1, -1, -1}, {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1},
        {-1, 1, 1},   {1, -1, -1}};
    return t[i][a];
  }
  // (2/3)^(3-k) (1/6)^k for k nonzero components (literal fractions)
  __host__ __device__ static constexpr double w(int i) {
    return nonzero(i) == 0
               ? 8.0 / 27.0
               : (nonzero(i) == 1 ? 2.0 / 27.0
                                  : (nonzero(i) == 2 ? 1.0 / 54.0
                                                     : 1.0 / 216.0));
  }
  __host__ __device__ static constexpr float wf(int i) {
    return nonzero(i) == 0
               ? 8.0f / 27.0f
               : (nonzero(i) == 1 ? 2.0f / 27.0f
                                  : (nonzero(i) == 2 ? 1.0f / 54.0f
                                                     : 1.0f / 216.0f));
  }
  __host__ __device__ static constexpr int nonzero(int i) {
    return (c(i, 0) != 0) + (c(i, 1) != 0) + (c(i, 2) != 0);
  }
  // binary16 storage scale 2^k_i, k_i = round(log2(1 / W_i))
  __host__ __device__ static constexpr float hscale(int i) {
    return nonzero(i) == 0
               ? 4.0f
               : (nonzero(i) == 1 ? 16.0f : (nonzero(i) == 2 ? 64.0f : 256.0f));
  }
  __host__ __device__ static constexpr float hscale_inv(int i) {
    return nonzero(i) == 0
               ? 0.25f
               : (nonzero(i) == 1 ? 0.0625f
                                  : (nonzero(i) == 2 ? 0.015625f : 0.00390625f));
  }
};

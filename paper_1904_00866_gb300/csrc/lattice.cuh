// Lattice descriptors for the sm_103a kernels.
//
// D2Q9 and D3Q27 are tensor products of D1Q3 (velocities {0, +1, -1},
// weights {2/3, 1/6, 1/6}, c_s^2 = 1/3).  Ordering follows the public ABI:
// rest first, then +/- pairs (index 2k-1 and 2k are opposite).  All members
// are constexpr so that, inside fully unrolled loops over i, every velocity
// component and weight is a compile-time constant.
#pragma once

// (2/3)^(D-k) (1/6)^k = 2^(D-k) / (3^(D-k) 6^k)
template <int D>
__host__ __device__ constexpr double weight(int k) {
  long long num = 1, den = 1;
  for (int a = 0; a < D - k; ++a) {
    num *= 2;
    den *= 3;
  }
  for (int a = 0; a < k; ++a) den *= 6;
  return (double)num / (double)den;
}

struct D2Q9 {
  static constexpr int D = 2;
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},
                             {0, 1, 0},  {0, -1, 0},  {1, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    return t[i][a];
  }
  // product of the per-axis D1Q3 weights, (2/3)^(D-k) (1/6)^k for k
  // nonzero components, as one correctly rounded quotient of integers
  __host__ __device__ static constexpr double w(int i) {
    return weight<D>(nonzero(i));
  }
  __host__ __device__ static constexpr int nonzero(int i) {
    return (c(i, 0) != 0) + (c(i, 1) != 0) + (c(i, 2) != 0);
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
  __host__ __device__ static constexpr double w(int i) {
    return weight<D>(nonzero(i));
  }
  __host__ __device__ static constexpr int nonzero(int i) {
    return (c(i, 0) != 0) + (c(i, 1) != 0) + (c(i, 2) != 0);
  }
};

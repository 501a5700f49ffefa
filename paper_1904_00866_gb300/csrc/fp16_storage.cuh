// FP16-shifted population storage: the deviation delta_i = f_i - W_i rho0
// from the lattice weights (rho0 a per-lattice constant kept on the host)
// is stored as binary16 after scaling by the exact power of two
// L::hscale(i) ~ 1 / W_i.  Decoding is exact (binary16 -> FP32 and a
// power-of-two scale); encoding rounds once, to nearest even.
//
// Arrays: population i starts at i * ps elements with the population stride
// ps = n rounded up to a multiple of 64, so every array is 128-byte aligned
// and the 4-byte word holding any element lies inside the allocation.
#pragma once
#include <cuda_fp16.h>

namespace elbm {

typedef __half half_t;

__host__ __device__ inline long long fp16_pop_stride(long long n) {
  return (n + 63) / 64 * 64;
}

template <class L>
__device__ __forceinline__ float h16_dev(unsigned short bits, int i) {
  return __half2float(__ushort_as_half(bits)) * L::hscale_inv(i);
}

template <class L>
__device__ __forceinline__ unsigned short h16_bits(float dev, int i) {
  return __half_as_ushort(__float2half_rn(dev * L::hscale(i)));
}

// FP64 helpers for initialisation, readout and the FP64 collision paths.
template <class L>
__device__ __forceinline__ double h16_to_f(half_t v, int i, double rho0) {
  return L::w(i) * rho0 + (double)__half2float(v) * (double)L::hscale_inv(i);
}

template <class L>
__device__ __forceinline__ half_t h16_from_dev(double dev, int i) {
  return __double2half(dev * (double)L::hscale(i));
}

}  // namespace elbm

// Initialisation and readout kernels of the pull-layout storage (FP64,
// FP32, FP32-shifted or FP16-shifted populations), shared by the
// single-lattice runtime and the batched runtime.
#pragma once
#include <math.h>

#include "fp16_storage.cuh"
#include "lattice.cuh"
#include "node_fp64.cuh"

namespace elbm {

// ------------------------------------------------------------------------
// Initialisation / readout kernels (grid-stride over nodes).
// ------------------------------------------------------------------------

// Entropic equilibrium in FP64: per-axis factors 1 + d(c), d(0) = -s,
// d(+-1) = +-3u + 2s, s = 3u^2 / (1 + sqrt(1 + 3u^2)).
template <class L>
__device__ __forceinline__ void equilibrium_dev(double rho, const double* u,
                                                double rho0, double* dev_out,
                                                double* f_out) {
  double dp[3], dm[3], d0[3];
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const double s = 3.0 * u[a] * u[a] / (1.0 + sqrt(1.0 + 3.0 * u[a] * u[a]));
    dp[a] = 3.0 * u[a] + 2.0 * s;
    dm[a] = -3.0 * u[a] + 2.0 * s;
    d0[a] = -s;
  }
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    double pm1 = 0.0;   // prod (1 + d) - 1
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
      const int c = L::c(i, a);
      const double d = c == 1 ? dp[a] : (c == -1 ? dm[a] : d0[a]);
      pm1 = fma(pm1, d, pm1 + d);
    }
    // f^eq_i - W_i rho0 = W_i ((rho - rho0) + rho (P_i - 1))
    dev_out[i] = L::w(i) * ((rho - rho0) + rho * pm1);
    f_out[i] = L::w(i) * rho * (1.0 + pm1);
  }
}

struct Geo {
  int nx, ny, nz;
  long long n;
  long long ps;  // population stride (elements)
  double rho0;
  int shifted;   // FP32_SHIFTED storage (FP16 storage is always shifted)
};

// The same in FP32 for FP32 storage (the stored value is rounded to FP32
// anyway): deviation W_i (drho + rho (P_i - 1)) formed
// without cancellation, a few FP32 ulp of the deviation; FP32 runs at 64x
// the FP64 rate on this GPU, which makes initialisation memory-bound.
// f_out (unshifted storage) = W_i rho (1 + (P_i - 1)).
template <class L>
__device__ __forceinline__ void equilibrium_dev32(float rho, float drho,
                                                  const float* u,
                                                  float* dev_out,
                                                  float* f_out) {
  float dp[3], dm[3], d0[3];
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const float s = 3.0f * u[a] * u[a] / (1.0f + sqrtf(fmaf(3.0f * u[a], u[a], 1.0f)));
    dp[a] = fmaf(3.0f, u[a], 2.0f * s);
    dm[a] = fmaf(-3.0f, u[a], 2.0f * s);
    d0[a] = -s;
  }
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    float pm1 = 0.0f;   // prod (1 + d) - 1
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
      const int c = L::c(i, a);
      const float d = c == 1 ? dp[a] : (c == -1 ? dm[a] : d0[a]);
      pm1 = fmaf(pm1, d, pm1 + d);
    }
    dev_out[i] = L::wf(i) * fmaf(rho, pm1, drho);
    f_out[i] = L::wf(i) * fmaf(rho, pm1, rho);
  }
}

// Storage value of population i, f, whose deviation from W_i rho0 is dev.
template <class L, class T>
__device__ __forceinline__ T to_storage(const Geo& g, int i, double f,
                                        double dev) {
  if constexpr (sizeof(T) == 8)
    return (T)f;
  else if constexpr (sizeof(T) == 4)
    return g.shifted ? (T)dev : (T)f;
  else
    return h16_from_dev<L>(dev, i);
}

// Population i from its storage value.
template <class L, class T>
__device__ __forceinline__ double from_storage(const Geo& g, int i, T v) {
  if constexpr (sizeof(T) == 8)
    return v;
  else if constexpr (sizeof(T) == 4)
    return g.shifted ? L::w(i) * g.rho0 + (double)v : (double)v;
  else
    return h16_to_f<L>(v, i, g.rho0);
}

// (x, y, z) of a flat node index, in 32-bit arithmetic (every lattice has
// fewer than 2^32 nodes), computed once per node.
struct Coord {
  int x, y, z;
};
__device__ __forceinline__ Coord node_coord(const Geo& g, long long node) {
  const unsigned nd = (unsigned)node;
  const unsigned row = nd / (unsigned)g.nx;
  const unsigned zq = row / (unsigned)g.ny;
  Coord c;
  c.x = (int)(nd - row * (unsigned)g.nx);
  c.y = (int)(row - zq * (unsigned)g.ny);
  c.z = (int)zq;
  return c;
}

// Flat index of node + sign * c_i (periodic).
template <class L>
__device__ __forceinline__ long long shifted_node(const Geo& g, const Coord& c,
                                                  int i, int sign) {
  int x = c.x + sign * L::c(i, 0);
  int y = c.y + sign * L::c(i, 1);
  int z = c.z + sign * L::c(i, 2);
  x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
  y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
  z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
  return (long long)(((unsigned)z * (unsigned)g.ny + (unsigned)y) *
                         (unsigned)g.nx +
                     (unsigned)x);
}

// f^0 = f^eq(rho, u); stored at x - c_i so that the pull gather of step 0
// returns it at x.  FP32 storage: the FP32 deviation form above; FP64 and
// FP16 storage: the FP64 equilibrium (binary16 values are then rounded once
// from FP64).
template <class L, class T>
__global__ void k_init_feq(Geo g, const double* __restrict__ rho,
                           const double* __restrict__ u, void* fv,
                           unsigned* err) {
  T* __restrict__ f = static_cast<T*>(fv);
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       node < g.n; node += (long long)gridDim.x * blockDim.x) {
    double uu[3] = {0.0, 0.0, 0.0};
    const double r = rho[node];
    bool bad = !(r > 0.0) || !isfinite(r);
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
      uu[a] = u[a * g.n + node];
      bad |= !(fabs(uu[a]) < 1.0);
    }
    if (bad) atomicOr(err, NF_BAD_NONFINITE);
    const Coord c = node_coord(g, node);
    if constexpr (sizeof(T) != 4) {
      double dev[L::Q], fe[L::Q];
      equilibrium_dev<L>(bad ? 1.0 : r, uu, g.rho0, dev, fe);
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        f[i * g.ps + shifted_node<L>(g, c, i, -1)] =
            to_storage<L, T>(g, i, fe[i], dev[i]);
    } else {
      const double rr = bad ? 1.0 : r;
      float u32[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) u32[a] = bad ? 0.0f : (float)uu[a];
      float dev[L::Q], fe[L::Q];
      equilibrium_dev32<L>((float)rr, (float)(rr - g.rho0), u32, dev, fe);
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        f[i * g.ps + shifted_node<L>(g, c, i, -1)] =
            g.shifted ? dev[i] : fe[i];
    }
  }
}

// Pre-collision populations f^n (FP64, [Q][N]) -> pull storage.
template <class L, class T>
__global__ void k_set_pop(Geo g, const double* __restrict__ fin, void* fv) {
  T* __restrict__ f = static_cast<T*>(fv);
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       node < g.n; node += (long long)gridDim.x * blockDim.x) {
    const Coord c = node_coord(g, node);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double v = fin[i * g.n + node];
      const double s = L::w(i) * g.rho0;
      f[i * g.ps + shifted_node<L>(g, c, i, -1)] =
          to_storage<L, T>(g, i, v, v - s);
    }
  }
}

template <class L, class T>
__device__ __forceinline__ double load_pre(const Geo& g, const T* f,
                                           const Coord& c, int i) {
  return from_storage<L, T>(g, i, f[i * g.ps + shifted_node<L>(g, c, i, -1)]);
}

// Storage -> pre-collision populations / moments (gather).
template <class L, class T>
__global__ void k_get_pop(Geo g, const void* fv, double* __restrict__ out) {
  const T* __restrict__ f = static_cast<const T*>(fv);
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       node < g.n; node += (long long)gridDim.x * blockDim.x) {
    const Coord c = node_coord(g, node);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) out[i * g.n + node] = load_pre<L, T>(g, f, c, i);
  }
}

template <class L, class T>
__global__ void k_get_nodes(Geo g, const void* fv,
                            const long long* __restrict__ nodes, int count,
                            double* __restrict__ out) {
  const T* __restrict__ f = static_cast<const T*>(fv);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += gridDim.x * blockDim.x) {
    const Coord c = node_coord(g, nodes[k]);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      out[(long long)k * L::Q + i] = load_pre<L, T>(g, f, c, i);
  }
}

template <class L, class T>
__global__ void k_moments(Geo g, const void* fv, double* __restrict__ rho_out,
                          double* __restrict__ u_out) {
  const T* __restrict__ f = static_cast<const T*>(fv);
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       node < g.n; node += (long long)gridDim.x * blockDim.x) {
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    const Coord c = node_coord(g, node);
    if (sizeof(T) == 4 && g.shifted) {
      // FP32 deviations: rho = rho0 + sum delta, j = sum c delta (the
      // W_i rho0 terms carry no momentum), with each delta split into a
      // 2^-20-grid part (summed exactly in FP32) and a remainder below
      // 2^-21 (summed in FP32: error ~1e-11), combined in FP64
      float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const float v = (float)f[i * g.ps + shifted_node<L>(g, c, i, -1)];
        const float hi = (v + 12.0f) - 12.0f, lo = v - hi;
        h[0] += hi;
        l[0] += lo;
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
          if (L::c(i, a) == 1) { h[a + 1] += hi; l[a + 1] += lo; }
          if (L::c(i, a) == -1) { h[a + 1] -= hi; l[a + 1] -= lo; }
        }
      }
      rho = g.rho0 + ((double)h[0] + (double)l[0]);
#pragma unroll
      for (int a = 0; a < L::D; ++a) j[a] = (double)h[a + 1] + (double)l[a + 1];
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const double v = load_pre<L, T>(g, f, c, i);
        rho += v;
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
          if (L::c(i, a) == 1) j[a] += v;
          if (L::c(i, a) == -1) j[a] -= v;
        }
      }
    }
    if (rho_out) rho_out[node] = rho;
    if (u_out) {
#pragma unroll
      for (int a = 0; a < L::D; ++a) u_out[a * g.n + node] = j[a] / rho;
    }
  }
}

// Block partial sums of |curl u|^2 (second-order central differences,
// periodic) from a velocity field u[d][nz][ny][nx].  2D: omega_z only.
template <int DIM>
__global__ void k_vorticity2(Geo g, const double* __restrict__ u,
                             double* __restrict__ partials) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       node < g.n; node += (long long)gridDim.x * blockDim.x) {
    const Coord c = node_coord(g, node);
    const int x = c.x, y = c.y, z = c.z;
    auto at = [&](int a, int xx, int yy, int zz) {
      xx = xx < 0 ? xx + g.nx : (xx >= g.nx ? xx - g.nx : xx);
      yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
      zz = zz < 0 ? zz + g.nz : (zz >= g.nz ? zz - g.nz : zz);
      return u[a * g.n + ((long long)zz * g.ny + yy) * g.nx + xx];
    };
    const double dvdx = 0.5 * (at(1, x + 1, y, z) - at(1, x - 1, y, z));
    const double dudy = 0.5 * (at(0, x, y + 1, z) - at(0, x, y - 1, z));
    const double wz = dvdx - dudy;
    double w2 = wz * wz;
    if (DIM == 3) {
      const double dwdy = 0.5 * (at(2, x, y + 1, z) - at(2, x, y - 1, z));
      const double dvdz = 0.5 * (at(1, x, y, z + 1) - at(1, x, y, z - 1));
      const double dudz = 0.5 * (at(0, x, y, z + 1) - at(0, x, y, z - 1));
      const double dwdx = 0.5 * (at(2, x + 1, y, z) - at(2, x - 1, y, z));
      const double wx = dwdy - dvdz, wy = dudz - dwdx;
      w2 += wx * wx + wy * wy;
    }
    acc += w2;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

}  // namespace elbm

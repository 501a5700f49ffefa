// Host runtime and C ABI of the ELBM library (declared in include/elbm.h):
// handle and buffer management, initialisation / readout kernels, the
// per-step launch sequence and the diagnostics finish kernel.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/elbm.h"
#include "internal.h"
#include "io_kernels.cuh"
#include "lattice_d1q3.cuh"

namespace elbm {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
}

// Sum the partial rows of one step in a fixed order.
__global__ void k_finish(const double* __restrict__ partials, int rows,
                         double* __restrict__ out) {
  const int k = blockIdx.x;  // slot
  __shared__ double sm[256];
  double v = k < S_NSUM ? 0.0 : (k == S_AMIN ? INFINITY : -INFINITY);
  if (k == S_ADEV) v = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const double x = partials[(long long)r * NSTAT + k];
    v = k < S_NSUM ? v + x : (k == S_AMIN ? fmin(v, x) : fmax(v, x));
  }
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double a = sm[threadIdx.x], b = sm[threadIdx.x + w];
      sm[threadIdx.x] =
          k < S_NSUM ? a + b : (k == S_AMIN ? fmin(a, b) : fmax(a, b));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = sm[0];
}

// Block partial sums of x[0..n) (one row per block, fixed order).
__global__ void k_partial_sum(const double* __restrict__ x, long long n,
                              double* __restrict__ partials) {
  __shared__ double sm[256];
  double v = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    v += x[k];
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

cudaError_t launch_finish(const double* partials, int rows, double* out,
                          cudaStream_t s) {
  k_finish<<<NSTAT, 256, 0, s>>>(partials, rows, out);
  count_launch();
  return cudaGetLastError();
}

void stats_from_slots(const double* s, double rho0, long long n,
                      long long step, int checked, void* out_stats) {
  elbm_entropy_stats_t* out = static_cast<elbm_entropy_stats_t*>(out_stats);
  memset(out, 0, sizeof(*out));
  out->step = step;
  out->n_nodes = (long long)s[S_NODES];
  out->mass = s[S_DRHO] + rho0 * (double)n;
  out->momentum[0] = s[S_J0];
  out->momentum[1] = s[S_J1];
  out->momentum[2] = s[S_J2];
  out->kinetic_energy = s[S_KE];
  out->alpha_min = s[S_AMIN];
  out->alpha_max = s[S_AMAX];
  out->alpha_sum = s[S_ASUM];
  out->n_accept_two = (long long)s[S_ACC2];
  out->n_accept_star = (long long)s[S_ACCSTAR];
  out->n_formula = (long long)s[S_FORMULA];
  out->n_band = (long long)s[S_BAND];
  out->n_far = (long long)s[S_FAR];
  out->n_degenerate = (long long)s[S_DEGEN];
  out->n_root_iters = (long long)s[S_ITERS];
  out->n_root_cap = (long long)s[S_CAP];
  out->n_no_root = (long long)s[S_NOROOT];
  out->checked = checked;
  out->h_total = s[S_H];
  out->n_violations = (long long)s[S_VIOL];
  out->n_decision_mismatch = (long long)s[S_MISMATCH];
  out->alpha_dev_max = s[S_ADEV];
}

}  // namespace elbm

using namespace elbm;

// ------------------------------------------------------------------------
// Handle
// ------------------------------------------------------------------------
struct elbm_handle {
  elbm_lattice lattice;
  int nx, ny, nz, q, d;
  long long n;
  double nu, beta;
  elbm_dtype dtype;
  double rho0 = 1.0;
  cudaStream_t stream = nullptr;
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* alloc_ctx = nullptr;
  bool allocated = false;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  float* alpha_map = nullptr;
  bool alpha_map_valid = false;
  double* partials = nullptr;
  int partial_rows_max = 0;
  double* stats_dev = nullptr;
  double* fields = nullptr;   // (1 + D) x n doubles: rho, u staging
  unsigned* err_flags = nullptr;
  unsigned* far_count = nullptr;   // [0..1] deferred, [2..3] undecided
  unsigned* far_queue = nullptr;
  float* refine_buf = nullptr;     // undecided-node records [cap][rec]
  unsigned refine_cap = 0;
  unsigned* refine_counts = nullptr;   // per stream-collide block
  int exact = 1;                   // second stage of undecided decisions
  long long step = 0;
  int diag_every = 1, check_every = 0, amap_every = 0, secant_iters = 4;
  bool stats_valid = false;
  long long stats_step = 0;
  int stats_checked = 0;
  size_t bytes = 0;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  size_t events_used = 0;
  std::vector<std::pair<void*, size_t>> owned;
  std::string err;
};

static thread_local std::string g_create_err;

namespace elbm {
void set_global_error(const std::string& msg) { g_create_err = msg; }
}  // namespace elbm

static size_t elem_size(elbm_dtype t) {
  return t == ELBM_FP64 ? 8 : (t == ELBM_FP16_SHIFTED ? 2 : 4);
}

// Population stride of the storage arrays (elements).
static long long pop_stride(const elbm_handle* h) {
  return h->dtype == ELBM_FP16_SHIFTED ? fp16_pop_stride(h->n) : h->n;
}

static elbm_status fail(elbm_handle* h, elbm_status st, const std::string& m) {
  if (h)
    h->err = m;
  else
    g_create_err = m;
  return st;
}

static elbm_status cuda_fail(elbm_handle* h, cudaError_t e, const char* what) {
  return fail(h, ELBM_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

static void* dev_alloc(elbm_handle* h, size_t bytes) {
  void* p = nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, h->alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    h->owned.push_back({p, bytes});
    h->bytes += bytes;
  }
  return p;
}

static void dev_free(elbm_handle* h, void* p) {
  if (!p) return;
  for (size_t k = 0; k < h->owned.size(); ++k) {
    if (h->owned[k].first == p) {
      h->bytes -= h->owned[k].second;
      h->owned.erase(h->owned.begin() + k);
      break;
    }
  }
  if (h->free_fn)
    h->free_fn(p, h->alloc_ctx);
  else
    cudaFree(p);
}

static int max_grid_rows() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 8;   // at most 8 resident 256-thread blocks per SM
}

static elbm_status ensure_buffers(elbm_handle* h) {
  if (h->allocated) return ELBM_OK;
  const size_t fb = (size_t)h->q * pop_stride(h) * elem_size(h->dtype);
  h->f[0] = dev_alloc(h, fb);
  h->f[1] = dev_alloc(h, fb);
  h->partial_rows_max = 3 * max_grid_rows();
  h->partials =
      (double*)dev_alloc(h, sizeof(double) * NSTAT * h->partial_rows_max);
  h->stats_dev = (double*)dev_alloc(h, sizeof(double) * NSTAT);
  h->err_flags = (unsigned*)dev_alloc(h, 256);
  h->far_count = (unsigned*)dev_alloc(h, 256);
  if (h->dtype != ELBM_FP64) {
    h->far_queue = (unsigned*)dev_alloc(h, sizeof(unsigned) * h->n);
    // Undecided nodes of a step: about 1-3 % of a developed 3D flow, but
    // most nodes of a flow whose non-equilibrium part is near FP32
    // resolution (a thin shear layer at Re 30,000) and of the first step
    // after initialisation; a full buffer sends the rest to the gathering
    // queue, where each node costs ~3x more (gather, FP32 stage again).
    // D2Q9: every node (48-byte records); D3Q27: half the nodes, at most
    // 2^26 records (8.6 GB) unless n / 16 is more, at least 65,536.
    const long long cap =
        h->q == 9
            ? h->n
            : std::min<long long>(
                  h->n, std::max<long long>(
                            65536, std::min<long long>(
                                       h->n / 2,
                                       std::max<long long>(h->n / 16,
                                                           1LL << 26))));
    const int rec = h->q == 27 ? refine_record<D3Q27>() : refine_record<D2Q9>();
    h->refine_buf =
        (float*)dev_alloc(h, sizeof(float) * (size_t)rec * (size_t)cap);
    h->refine_counts =
        (unsigned*)dev_alloc(h, sizeof(unsigned) * kMaxRefineBlocks);
    h->refine_cap = h->refine_buf && h->refine_counts ? (unsigned)cap : 0u;
  }
  if (!h->f[0] || !h->f[1] || !h->partials || !h->stats_dev ||
      !h->err_flags || !h->far_count ||
      (h->dtype != ELBM_FP64 && !h->far_queue))
    return fail(h, ELBM_ENOMEM, "device allocation failed");
  cudaMemsetAsync(h->err_flags, 0, 256, h->stream);
  cudaMemsetAsync(h->far_count, 0, 256, h->stream);
  h->allocated = true;
  return ELBM_OK;
}

static elbm_status ensure_alpha_map(elbm_handle* h) {
  if (h->alpha_map) return ELBM_OK;
  h->alpha_map = (float*)dev_alloc(h, sizeof(float) * h->n);
  if (!h->alpha_map) return fail(h, ELBM_ENOMEM, "alpha map allocation failed");
  return ELBM_OK;
}

// Device staging of one density and D velocity fields (FP64), used by
// initialisation, moments and enstrophy.  Allocated on first use and kept
// until the handle is destroyed, so repeated calls allocate nothing.
static double* fields_staging(elbm_handle* h) {
  if (!h->fields)
    h->fields = (double*)dev_alloc(h, sizeof(double) * (1 + h->d) * h->n);
  return h->fields;
}

static Geo geo(const elbm_handle* h) {
  Geo g;
  g.nx = h->nx;
  g.ny = h->ny;
  g.nz = h->nz;
  g.n = h->n;
  g.ps = pop_stride(h);
  g.rho0 = h->dtype == ELBM_FP64 ? 0.0 : h->rho0;
  g.shifted = h->dtype == ELBM_FP32_SHIFTED || h->dtype == ELBM_FP16_SHIFTED;
  return g;
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  int cap = max_grid_rows();
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

// Dispatch a node-parallel helper kernel on (lattice, storage type); D1Q3
// handles hold FP64 storage only.
#define DISPATCH_LT(h, KERNEL, ...)                                          \
  do {                                                                       \
    const int grid_ = grid_for((h)->n);                                      \
    if ((h)->lattice == ELBM_D1Q3) {                                         \
      KERNEL<D1Q3, double><<<grid_, 256, 0, (h)->stream>>>(__VA_ARGS__);     \
    } else if ((h)->lattice == ELBM_D2Q9) {                                  \
      if ((h)->dtype == ELBM_FP64)                                           \
        KERNEL<D2Q9, double><<<grid_, 256, 0, (h)->stream>>>(__VA_ARGS__);   \
      else if ((h)->dtype == ELBM_FP16_SHIFTED)                              \
        KERNEL<D2Q9, half_t><<<grid_, 256, 0, (h)->stream>>>(__VA_ARGS__);   \
      else                                                                   \
        KERNEL<D2Q9, float><<<grid_, 256, 0, (h)->stream>>>(__VA_ARGS__);    \
    } else {                                                                 \
      if ((h)->dtype == ELBM_FP64)                                           \
        KERNEL<D3Q27, double><<<grid_, 256, 0, (h)->stream>>>(__VA_ARGS__);  \
      else if ((h)->dtype == ELBM_FP16_SHIFTED)                              \
        KERNEL<D3Q27, half_t><<<grid_, 256, 0, (h)->stream>>>(__VA_ARGS__);  \
      else                                                                   \
        KERNEL<D3Q27, float><<<grid_, 256, 0, (h)->stream>>>(__VA_ARGS__);   \
    }                                                                        \
    count_launch();                                                          \
  } while (0)

static elbm_status check_errors(elbm_handle* h) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
  if (!h->allocated) return ELBM_OK;
  unsigned flags = 0;
  e = cudaMemcpy(&flags, h->err_flags, sizeof(unsigned),
                 cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "read error flags");
  if (flags & NF_TIMEOUT)
    return fail(h, ELBM_ECUDA, "a kernel's bounded copy wait timed out");
  if (flags & NF_BAD_NEG)
    return fail(h, ELBM_ENEGATIVE, "a node had a population <= 0");
  if (flags & NF_BAD_NONFINITE)
    return fail(h, ELBM_ENONFINITE,
                "a node had non-finite moments or |u| >= 1");
  return ELBM_OK;
}

extern "C" {

elbm_status elbm_create(elbm_handle** out, elbm_lattice lattice, int nx,
                        int ny, int nz, double nu, elbm_dtype dtype) {
  if (!out) return fail(nullptr, ELBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27 && lattice != ELBM_D1Q3)
    return fail(nullptr, ELBM_EINVAL, "unknown lattice");
  if (dtype != ELBM_FP64 && dtype != ELBM_FP32 && dtype != ELBM_FP32_SHIFTED &&
      dtype != ELBM_FP16_SHIFTED)
    return fail(nullptr, ELBM_EINVAL, "unknown dtype");
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(nullptr, ELBM_EINVAL, "lattice dimensions must be >= 1");
  if (lattice == ELBM_D2Q9 && nz != 1)
    return fail(nullptr, ELBM_EINVAL, "D2Q9 needs nz == 1");
  if (lattice == ELBM_D1Q3 && (ny != 1 || nz != 1))
    return fail(nullptr, ELBM_EINVAL, "D1Q3 needs ny == nz == 1");
  if (lattice == ELBM_D1Q3 && dtype != ELBM_FP64)
    return fail(nullptr, ELBM_EINVAL, "D1Q3 supports FP64 storage only");
  if (!(nu > 0.0) || !(nu < 1e6))
    return fail(nullptr, ELBM_EINVAL, "nu must be > 0");
  const long long n = (long long)nx * ny * nz;
  const int q = lattice == ELBM_D1Q3 ? 3 : (lattice == ELBM_D2Q9 ? 9 : 27);
  if (n > 0xffffffffLL || (long long)q * n > (1LL << 40))
    return fail(nullptr, ELBM_EINVAL, "lattice too large");
  // the deferred-node queue of FP32 / FP16 storage tags entries in bit 31
  if (dtype != ELBM_FP64 && n >= (1LL << 31))
    return fail(nullptr, ELBM_EINVAL,
                "FP32 / FP16 storage supports fewer than 2^31 nodes");
  elbm_handle* h = new elbm_handle();
  h->lattice = lattice;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->q = q;
  h->d = lattice == ELBM_D1Q3 ? 1 : (lattice == ELBM_D2Q9 ? 2 : 3);
  h->n = n;
  h->nu = nu;
  const double cs2 = 1.0 / 3.0;
  h->beta = cs2 / (2.0 * nu + cs2);   // Eq. (2), dt = 1
  h->dtype = dtype;
  *out = h;
  return ELBM_OK;
}

void elbm_destroy(elbm_handle* h) {
  if (!h) return;
  if (!h->owned.empty()) cudaStreamSynchronize(h->stream);
  for (auto& ev : h->events) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  while (!h->owned.empty()) dev_free(h, h->owned.back().first);
  delete h;
}

const char* elbm_last_error(const elbm_handle* h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

elbm_status elbm_set_stream(elbm_handle* h, void* s) {
  if (!h) return ELBM_EINVAL;
  h->stream = (cudaStream_t)s;
  return ELBM_OK;
}

elbm_status elbm_set_allocator(elbm_handle* h, void* (*alloc)(size_t, void*),
                               void (*free_fn)(void*, void*), void* ctx) {
  if (!h) return ELBM_EINVAL;
  if (h->allocated || !h->owned.empty())
    return fail(h, ELBM_ESTATE, "allocator must be set before allocation");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(h, ELBM_EINVAL, "alloc and free must both be set or NULL");
  h->alloc = alloc;
  h->free_fn = free_fn;
  h->alloc_ctx = ctx;
  return ELBM_OK;
}

elbm_status elbm_set_diagnostics(elbm_handle* h, int diag_every,
                                 int check_every, int alpha_map_every,
                                 int secant_iters) {
  if (!h) return ELBM_EINVAL;
  if (diag_every < 0 || check_every < 0 || alpha_map_every < 0 ||
      secant_iters < 1 || secant_iters > 1000)
    return fail(h, ELBM_EINVAL, "invalid diagnostics schedule");
  h->diag_every = diag_every;
  h->check_every = check_every;
  h->amap_every = alpha_map_every;
  h->secant_iters = secant_iters;
  return ELBM_OK;
}

// Mean of a device array (deterministic: fixed grid, rows summed in order
// on the host).
static elbm_status device_mean(elbm_handle* h, const double* x, double* mean) {
  const int grid = grid_for(h->n);
  k_partial_sum<<<grid, 256, 0, h->stream>>>(x, h->n, h->partials);
  count_launch();
  std::vector<double> rows(grid);
  cudaError_t e = cudaMemcpyAsync(rows.data(), h->partials,
                                  sizeof(double) * grid,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "density mean");
  double s = 0.0;
  for (double r : rows) s += r;
  *mean = s / (double)h->n;
  return ELBM_OK;
}

// f^0 = f^eq(rho, u) from device fields; rho0 = FP32-rounded mean density.
static elbm_status init_common(elbm_handle* h, const double* rho_dev,
                               const double* u_dev) {
  double mean = 1.0;
  elbm_status st = device_mean(h, rho_dev, &mean);
  if (st) return st;
  if (!(mean > 0.0) || !(mean < 1e30))
    return fail(h, ELBM_EINVAL, "rho must be > 0 and finite");
  h->rho0 = (double)(float)mean;
  cudaMemsetAsync(h->err_flags, 0, 256, h->stream);
  cudaMemsetAsync(h->far_count, 0, 256, h->stream);
  h->cur = 0;
  Geo g = geo(h);
  DISPATCH_LT(h, k_init_feq, g, rho_dev, u_dev, h->f[0], h->err_flags);
  h->step = 0;
  h->stats_valid = false;
  h->alpha_map_valid = false;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
  st = check_errors(h);
  if (st == ELBM_ENONFINITE || st == ELBM_ENEGATIVE)
    return fail(h, ELBM_EINVAL, "invalid initial fields (rho <= 0, "
                                "non-finite, or |u| >= 1)");
  return st;
}

// The device-side address of a host buffer the GPU can access directly
// (page-locked host memory, e.g. cudaHostAlloc or a pinned framework
// tensor), else null.  Kernels then read or write it over the host link
// themselves, with no staging copy in device memory.
static void* host_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // clear the error state of the query
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

elbm_status elbm_init_fields(elbm_handle* h, const double* rho,
                             const double* u) {
  if (!h || !rho || !u) return h ? fail(h, ELBM_EINVAL, "NULL field") : ELBM_EINVAL;
  elbm_status st = ensure_buffers(h);
  if (st) return st;
  const double* rho_v = (const double*)host_view(rho);
  const double* u_v = (const double*)host_view(u);
  if (rho_v && u_v) {   // page-locked: the init kernels read them directly
    st = init_common(h, rho_v, u_v);
    cudaStreamSynchronize(h->stream);
    return st;
  }
  double* tmp = fields_staging(h);
  if (!tmp) return fail(h, ELBM_ENOMEM, "staging allocation failed");
  cudaError_t e = cudaMemcpyAsync(tmp, rho, sizeof(double) * h->n,
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tmp + h->n, u, sizeof(double) * h->d * h->n,
                        cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(h->stream);
    return cuda_fail(h, e, "copy fields");
  }
  st = init_common(h, tmp, tmp + h->n);
  cudaStreamSynchronize(h->stream);
  return st;
}

elbm_status elbm_init_fields_device(elbm_handle* h, const double* rho_device,
                                    const double* u_device) {
  if (!h || !rho_device || !u_device) return h ? fail(h, ELBM_EINVAL, "NULL field") : ELBM_EINVAL;
  elbm_status st = ensure_buffers(h);
  if (st) return st;
  return init_common(h, rho_device, u_device);
}

elbm_status elbm_set_populations(elbm_handle* h, const double* f) {
  if (!h || !f) return h ? fail(h, ELBM_EINVAL, "NULL populations") : ELBM_EINVAL;
  double mass = 0.0;
  for (long long k = 0; k < (long long)h->q * h->n; ++k) {
    if (!(f[k] > 0.0)) return fail(h, ELBM_EINVAL, "populations must be > 0");
    mass += f[k];
  }
  h->rho0 = (double)(float)(mass / (double)h->n);
  elbm_status st = ensure_buffers(h);
  if (st) return st;
  const size_t bytes = sizeof(double) * h->q * h->n;
  double* tmp = (double*)dev_alloc(h, bytes);
  if (!tmp) return fail(h, ELBM_ENOMEM, "staging allocation failed");
  cudaError_t e =
      cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    dev_free(h, tmp);
    return cuda_fail(h, e, "copy populations");
  }
  cudaMemsetAsync(h->err_flags, 0, 256, h->stream);
  cudaMemsetAsync(h->far_count, 0, 256, h->stream);
  h->cur = 0;
  Geo g = geo(h);
  DISPATCH_LT(h, k_set_pop, g, (const double*)tmp, h->f[0]);
  cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  h->step = 0;
  h->stats_valid = false;
  h->alpha_map_valid = false;
  return check_errors(h);
}

elbm_status elbm_step(elbm_handle* h, long long nsteps, elbm_alpha_mode mode) {
  if (!h) return ELBM_EINVAL;
  if (nsteps < 0) return fail(h, ELBM_EINVAL, "nsteps must be >= 0");
  if (mode != ELBM_ALPHA_FORMULA && mode != ELBM_ALPHA_ROOT &&
      mode != ELBM_ALPHA_SECANT)
    return fail(h, ELBM_EINVAL, "unknown alpha mode");
  if (!h->allocated)
    return fail(h, ELBM_ESTATE, "fields not initialised");
  if (h->amap_every > 0) {
    elbm_status st = ensure_alpha_map(h);
    if (st) return st;
  }
  StepParams p;
  memset(&p, 0, sizeof(p));
  p.nx = h->nx;
  p.ny = h->ny;
  p.nz = h->nz;
  p.n = h->n;
  p.ps = pop_stride(h);
  p.chunks = (h->nx + 31) / 32;
  p.tiles = (long long)p.chunks * h->ny * h->nz;
  p.beta = h->beta;
  p.rho0 = h->dtype == ELBM_FP64 ? 0.0 : h->rho0;
  p.betaf = (float)p.beta;
  p.rho0f = (float)p.rho0;
  p.unshifted = h->dtype == ELBM_FP32;
  if (p.unshifted) {
    const float r0 = (float)h->rho0;
    double ssum = 0.0;
    for (int i = 0; i < h->q; ++i) {
      const double w = h->lattice == ELBM_D2Q9 ? D2Q9::w(i) : D3Q27::w(i);
      const float s = (float)w * r0;
      ssum += (double)s;
      p.corr[i] = (float)(w * h->rho0 - (double)s);
    }
    p.corr_rho = (float)(ssum - h->rho0);
  }
  p.secant_iters = h->secant_iters;
  p.div_nx.init((unsigned)h->nx);
  p.div_ny.init((unsigned)h->ny);
  p.partials = h->partials;
  p.err_flags = h->err_flags;
  p.far_count = h->far_count;
  p.far_queue = h->far_queue;
  p.far_cap = h->far_queue ? (unsigned)h->n : 0u;
  p.exact = h->exact;
  p.refine_buf = h->refine_buf;
  p.refine_cap = h->refine_cap;
  p.refine_counts = h->refine_counts;
  // the deferred-node counters start every call at zero; within the call
  // each step's fixup clears the counter the next step uses
  if (nsteps > 0) cudaMemsetAsync(h->far_count, 0, 2 * sizeof(unsigned),
                                  h->stream);
  const bool d2 = h->lattice == ELBM_D2Q9;
  // 0: FP64, 1: FP32 (shifted or not), 2: FP16-shifted
  const int storage =
      h->dtype == ELBM_FP64 ? 0 : (h->dtype == ELBM_FP16_SHIFTED ? 2 : 1);
  const size_t esz = elem_size(h->dtype);
  for (long long s = 0; s < nsteps; ++s) {
    const long long n = h->step;
    const int check = h->check_every > 0 && n % h->check_every == 0;
    const int diag = check || (h->diag_every > 0 && n % h->diag_every == 0);
    const bool amap = h->amap_every > 0 && n % h->amap_every == 0;
    p.f_in = h->f[h->cur];
    p.f_out = h->f[h->cur ^ 1];
    if (storage != 0) {
      for (int i = 0; i < h->q; ++i) {
        p.in_pop[i] = (const float*)((const char*)p.f_in +
                                     (size_t)i * p.ps * esz);
        p.out_pop[i] = (float*)((char*)p.f_out + (size_t)i * p.ps * esz);
      }
    }
    p.alpha_map = amap ? h->alpha_map : nullptr;
    p.parity = (int)(n & 1);
    int grid = 0;
    cudaError_t e;
    const bool fp32_formula = storage != 0 && mode == ELBM_ALPHA_FORMULA;
    std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
    if (h->profiling) {
      if (h->events_used == h->events.size()) {
        std::pair<cudaEvent_t, cudaEvent_t> pr;
        cudaEventCreate(&pr.first);
        cudaEventCreate(&pr.second);
        h->events.push_back(pr);
      }
      ev = &h->events[h->events_used++];
      cudaEventRecord(ev->first, h->stream);
    }
    if (h->lattice == ELBM_D1Q3)
      e = launch_fp64_d1q3(mode, diag, check, p, 0, 256, h->stream, &grid);
    else if (storage == 0)
      e = d2 ? launch_fp64_d2q9(mode, diag, check, p, 0, 256, h->stream, &grid)
             : launch_fp64_d3q27(mode, diag, check, p, 0, 256, h->stream, &grid);
    else if (fp32_formula && storage == 2)
      e = d2 ? launch_fp16_formula_d2q9(diag, check, p, 0, h->stream, &grid)
             : launch_fp16_formula_d3q27(diag, check, p, 0, h->stream, &grid);
    else if (fp32_formula)
      e = d2 ? launch_fp32_formula_d2q9(diag, check, p, 0, 256, h->stream, &grid)
             : launch_fp32_formula_d3q27(diag, check, p, 0, 256, h->stream,
                                         &grid);
    else if (storage == 2)
      e = d2 ? launch_fp16_fp64mode_d2q9(mode, diag, check, p, 0, 256,
                                         h->stream, &grid)
             : launch_fp16_fp64mode_d3q27(mode, diag, check, p, 0, 256,
                                          h->stream, &grid);
    else
      e = d2 ? launch_fp32_fp64mode_d2q9(mode, diag, check, p, 0, 256,
                                         h->stream, &grid)
             : launch_fp32_fp64mode_d3q27(mode, diag, check, p, 0, 256,
                                          h->stream, &grid);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream-collide launch");
    if (ev) cudaEventRecord(ev->second, h->stream);
    int rows = grid;
    if (fp32_formula) {
      StepParams pf = p;
      // the second stage and the fixup run at most 2 blocks per SM
      // (their register budgets), so a larger grid only adds waves of
      // blocks with nothing to do
      const int fgrid = std::min(grid, max_grid_rows() / 4);
      if (p.exact && p.refine_cap) {
        // second stage of the undecided nodes the step buffered
        pf.partials = h->partials + (size_t)rows * NSTAT;
        e = storage == 2
                ? (d2 ? launch_refine16_d2q9(diag, check, pf, grid, fgrid,
                                             h->stream)
                      : launch_refine16_d3q27(diag, check, pf, grid, fgrid,
                                              h->stream))
                : (d2 ? launch_refine_d2q9(diag, check, pf, grid, fgrid,
                                           h->stream)
                      : launch_refine_d3q27(diag, check, pf, grid, fgrid,
                                            h->stream));
        if (e != cudaSuccess) return cuda_fail(h, e, "second stage launch");
        rows += fgrid;
      }
      pf.partials = h->partials + (size_t)rows * NSTAT;
      if (storage == 2)
        e = d2 ? launch_far16_d2q9(diag, check, pf, fgrid, h->stream)
               : launch_far16_d3q27(diag, check, pf, fgrid, h->stream);
      else
        e = d2 ? launch_far_d2q9(diag, check, pf, fgrid, h->stream)
               : launch_far_d3q27(diag, check, pf, fgrid, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "far fixup launch");
      rows += fgrid;
    }
    if (diag) {
      launch_finish(h->partials, rows, h->stats_dev, h->stream);
      h->stats_valid = true;
      h->stats_step = n;
      h->stats_checked = check;
    }
    if (amap) h->alpha_map_valid = true;
    h->cur ^= 1;
    h->step += 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "step");
  return ELBM_OK;
}

elbm_status elbm_sync(elbm_handle* h) {
  if (!h) return ELBM_EINVAL;
  return check_errors(h);
}

elbm_status elbm_moments(elbm_handle* h, double* rho_out, double* u_out) {
  if (!h) return ELBM_EINVAL;
  if (!h->allocated) return fail(h, ELBM_ESTATE, "fields not initialised");
  elbm_status st = check_errors(h);
  if (st) return st;
  Geo g = geo(h);
  double* rho_v = rho_out ? (double*)host_view(rho_out) : nullptr;
  double* u_v = u_out ? (double*)host_view(u_out) : nullptr;
  if (rho_v && u_v) {   // page-locked: the kernel writes them directly
    DISPATCH_LT(h, k_moments, g, h->f[h->cur], rho_v, u_v);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments");
    return ELBM_OK;
  }
  double* tmp = fields_staging(h);
  if (!tmp) return fail(h, ELBM_ENOMEM, "staging allocation failed");
  DISPATCH_LT(h, k_moments, g, h->f[h->cur], tmp, tmp + h->n);
  cudaError_t e = cudaSuccess;
  if (rho_out)
    e = cudaMemcpyAsync(rho_out, tmp, sizeof(double) * h->n,
                        cudaMemcpyDeviceToHost, h->stream);
  if (u_out && e == cudaSuccess)
    e = cudaMemcpyAsync(u_out, tmp + h->n, sizeof(double) * h->d * h->n,
                        cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy moments");
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "moments");
  return ELBM_OK;
}

elbm_status elbm_get_populations(elbm_handle* h, double* f_out) {
  if (!h || !f_out) return h ? fail(h, ELBM_EINVAL, "NULL output") : ELBM_EINVAL;
  if (!h->allocated) return fail(h, ELBM_ESTATE, "fields not initialised");
  elbm_status st = check_errors(h);
  if (st) return st;
  const size_t bytes = sizeof(double) * h->q * h->n;
  double* tmp = (double*)dev_alloc(h, bytes);
  if (!tmp) return fail(h, ELBM_ENOMEM, "staging allocation failed");
  Geo g = geo(h);
  DISPATCH_LT(h, k_get_pop, g, h->f[h->cur], tmp);
  cudaError_t e =
      cudaMemcpyAsync(f_out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy populations");
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "populations");
  return ELBM_OK;
}

elbm_status elbm_get_populations_nodes(elbm_handle* h, const long long* nodes,
                                       int count, double* f_out) {
  if (!h || (count > 0 && (!nodes || !f_out)) || count < 0)
    return h ? fail(h, ELBM_EINVAL, "invalid node list") : ELBM_EINVAL;
  if (!h->allocated) return fail(h, ELBM_ESTATE, "fields not initialised");
  for (int k = 0; k < count; ++k)
    if (nodes[k] < 0 || nodes[k] >= h->n)
      return fail(h, ELBM_EINVAL, "node index out of range");
  elbm_status st = check_errors(h);
  if (st || count == 0) return st;
  const size_t ib = sizeof(long long) * count;
  const size_t ob = sizeof(double) * h->q * count;
  char* tmp = (char*)dev_alloc(h, ib + ob);
  if (!tmp) return fail(h, ELBM_ENOMEM, "staging allocation failed");
  cudaMemcpyAsync(tmp, nodes, ib, cudaMemcpyHostToDevice, h->stream);
  Geo g = geo(h);
  const long long* dn = (const long long*)tmp;
  double* dout = (double*)(tmp + ib);
  DISPATCH_LT(h, k_get_nodes, g, (const void*)h->f[h->cur], dn, count, dout);
  cudaError_t e =
      cudaMemcpyAsync(f_out, dout, ob, cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy node populations");
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "node populations");
  return ELBM_OK;
}

elbm_status elbm_alpha_map(elbm_handle* h, float* alpha_out) {
  if (!h || !alpha_out) return h ? fail(h, ELBM_EINVAL, "NULL output") : ELBM_EINVAL;
  if (!h->alpha_map_valid)
    return fail(h, ELBM_ESTATE, "no step has written the alpha map");
  elbm_status st = check_errors(h);
  if (st) return st;
  cudaError_t e = cudaMemcpy(alpha_out, h->alpha_map, sizeof(float) * h->n,
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy alpha map");
  return ELBM_OK;
}

elbm_status elbm_entropy_stats(elbm_handle* h, elbm_entropy_stats_t* out) {
  if (!h || !out) return h ? fail(h, ELBM_EINVAL, "NULL output") : ELBM_EINVAL;
  if (!h->stats_valid)
    return fail(h, ELBM_ESTATE, "no step has computed diagnostics");
  elbm_status st = check_errors(h);
  if (st) return st;
  double s[NSTAT];
  cudaError_t e = cudaMemcpy(s, h->stats_dev, sizeof(s), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy stats");
  stats_from_slots(s, h->dtype == ELBM_FP64 ? 0.0 : h->rho0, h->n,
                   h->stats_step, h->stats_checked, out);
  if (out->n_root_cap > 0)
    return fail(h, ELBM_EROOT_CAP,
                std::to_string(out->n_root_cap) +
                    " node(s) stopped ROOT bisection at the iteration cap");
  return ELBM_OK;
}

elbm_status elbm_enstrophy(elbm_handle* h, double* out) {
  if (!h || !out) return h ? fail(h, ELBM_EINVAL, "NULL output") : ELBM_EINVAL;
  if (!h->allocated) return fail(h, ELBM_ESTATE, "fields not initialised");
  elbm_status st = check_errors(h);
  if (st) return st;
  if (h->d == 1) {   // a one-dimensional velocity field has no curl
    *out = 0.0;
    return ELBM_OK;
  }
  double* tmp = fields_staging(h);
  if (!tmp) return fail(h, ELBM_ENOMEM, "staging allocation failed");
  Geo g = geo(h);
  DISPATCH_LT(h, k_moments, g, h->f[h->cur], tmp, tmp + h->n);
  const int grid = grid_for(h->n);
  if (h->d == 3)
    k_vorticity2<3><<<grid, 256, 0, h->stream>>>(g, tmp + h->n, h->partials);
  else
    k_vorticity2<2><<<grid, 256, 0, h->stream>>>(g, tmp + h->n, h->partials);
  count_launch();
  std::vector<double> rows(grid);
  cudaError_t e = cudaMemcpyAsync(rows.data(), h->partials,
                                  sizeof(double) * grid,
                                  cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy enstrophy");
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "enstrophy");
  double s = 0.0;
  for (double r : rows) s += r;
  *out = 0.5 * s / (double)h->n;
  return ELBM_OK;
}

long long elbm_step_count(const elbm_handle* h) { return h ? h->step : -1; }

size_t elbm_device_bytes(const elbm_handle* h) { return h ? h->bytes : 0; }

long long elbm_launch_count(void) { return g_launches.load(); }

double elbm_rho0(const elbm_handle* h) { return h ? h->rho0 : 0.0; }

double elbm_beta(const elbm_handle* h) { return h ? h->beta : NAN; }

elbm_status elbm_set_decision(elbm_handle* h, elbm_decision decision) {
  if (!h) return ELBM_EINVAL;
  if (decision != ELBM_DECISION_EXACT && decision != ELBM_DECISION_CERTIFIED)
    return fail(h, ELBM_EINVAL, "unknown decision mode");
  h->exact = decision == ELBM_DECISION_EXACT;
  return ELBM_OK;
}

elbm_status elbm_set_profiling(elbm_handle* h, int enable) {
  if (!h) return ELBM_EINVAL;
  h->profiling = enable != 0;
  return ELBM_OK;
}

elbm_status elbm_profile(elbm_handle* h, double* ms, long long* launches) {
  if (!h) return ELBM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
  double total = 0.0;
  for (size_t k = 0; k < h->events_used; ++k) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, h->events[k].first, h->events[k].second);
    if (e != cudaSuccess) return cuda_fail(h, e, "event elapsed time");
    total += t;
  }
  if (ms) *ms = total;
  if (launches) *launches = (long long)h->events_used;
  h->events_used = 0;
  return ELBM_OK;
}

}  // extern "C"

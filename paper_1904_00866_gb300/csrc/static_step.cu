// elbm_step_static: one FP32-shifted FORMULA step that allocates no device
// memory.
//
// Some callers cannot call cudaMalloc: a host application that reserves its
// whole device-memory budget up front in its own pool and hands the library
// only buffers from that pool, or a latency-critical loop that must not pay
// for (or be blocked by) the allocator's implicit device synchronisation.
// For them this entry point runs the same kernels as elbm_step on buffers
// the caller owns.  The kernels' scratch memory -- the queue of nodes
// deferred to the FP64 fixup, the per-block diagnostic rows, the reduced
// statistics and the error/counter words -- lives in one file-scope
// __device__ array of fixed size (below), which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/elbm.h"
#include "internal.h"

namespace elbm {
namespace {

constexpr unsigned kStaticMaxNodes = 1u << 21;   // 2,097,152 lattice nodes
constexpr int kStaticMaxRows = 4096;             // diagnostic partial rows
constexpr size_t kCountersBytes = 256;           // far_count[2], err_flags
constexpr size_t kPartialsBytes = sizeof(double) * NSTAT * kStaticMaxRows;
constexpr size_t kStatsBytes = 256;              // NSTAT doubles, padded
constexpr size_t kQueueBytes = sizeof(unsigned) * kStaticMaxNodes;
constexpr size_t kScratchBytes =
    kCountersBytes + kPartialsBytes + kStatsBytes + kQueueBytes;
static_assert(NSTAT * sizeof(double) <= kStatsBytes, "stats slots");

// The scratch array.  Host code must not use its name as an address (it is
// a host-side stand-in); the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};
elbm_status fail(elbm_status st, const std::string& m) {
  set_global_error(m);   // read back with elbm_last_error(NULL)
  return st;
}

}  // namespace
}  // namespace elbm

using namespace elbm;

extern "C" elbm_status elbm_step_static(
    elbm_lattice lattice, int nx, int ny, int nz, double nu, double rho0,
    const float* f_in_device, float* f_out_device, float* alpha_out_device,
    void* cuda_stream, elbm_entropy_stats_t* stats_out) {
  if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27)
    return fail(ELBM_EINVAL, lattice == ELBM_D1Q3
                                 ? "elbm_step_static takes D2Q9 and D3Q27 only"
                                 : "unknown lattice");
  if (nx < 1 || ny < 1 || nz < 1 || (lattice == ELBM_D2Q9 && nz != 1))
    return fail(ELBM_EINVAL, "invalid lattice dimensions");
  const long long n = (long long)nx * ny * nz;
  if (n > (long long)kStaticMaxNodes)
    return fail(ELBM_EINVAL,
                "lattice has " + std::to_string(n) +
                    " nodes; elbm_step_static supports at most " +
                    std::to_string(kStaticMaxNodes) +
                    " (its scratch array has a fixed size)");
  if (!(nu > 0.0) || !(rho0 > 0.0))
    return fail(ELBM_EINVAL, "nu and rho0 must be > 0");
  if (!f_in_device || !f_out_device || f_in_device == f_out_device)
    return fail(ELBM_EINVAL, "f_in and f_out must be distinct device buffers");
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // one-time set-up on this device: device address of the scratch array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ELBM_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(ELBM_EINVAL, "device ordinal out of range");
  // Every stream-collide launcher sizes its grid to at most 8 resident
  // blocks per SM, and the fixup uses at most 152 blocks; each block writes
  // one diagnostic row.  Refuse before anything is queued if the rows could
  // overflow the fixed array on this device.
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(ELBM_ECUDA, cudaGetErrorString(e));
  if ((long long)sms * 8 + 152 > kStaticMaxRows)
    return fail(ELBM_EINVAL,
                "device has too many SMs for the static diagnostic rows");
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr)
        return fail(ELBM_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                    cudaGetErrorString(e));
      g_scratch_addr[dev] = ptr;
    }
    scratch = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  unsigned* counters = reinterpret_cast<unsigned*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + kCountersBytes);
  double* stats = reinterpret_cast<double*>(scratch + kCountersBytes +
                                            kPartialsBytes);
  unsigned* queue = reinterpret_cast<unsigned*>(
      scratch + kCountersBytes + kPartialsBytes + kStatsBytes);

  // the array keeps the previous call's contents: clear the counters
  e = cudaMemsetAsync(counters, 0, kCountersBytes, stream);
  if (e != cudaSuccess) return fail(ELBM_ECUDA, cudaGetErrorString(e));

  StepParams p;
  memset(&p, 0, sizeof(p));
  const int q = lattice == ELBM_D2Q9 ? 9 : 27;
  p.f_in = f_in_device;
  p.f_out = f_out_device;
  for (int i = 0; i < q; ++i) {
    p.in_pop[i] = f_in_device + (size_t)i * n;
    p.out_pop[i] = f_out_device + (size_t)i * n;
  }
  p.alpha_map = alpha_out_device;
  p.partials = partials;
  p.err_flags = counters + 2;
  p.far_count = counters;
  p.far_queue = queue;
  p.far_cap = (unsigned)n;
  p.parity = 0;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.n = n;
  p.ps = n;
  p.chunks = (nx + 31) / 32;
  p.tiles = (long long)p.chunks * ny * nz;
  const double cs2 = 1.0 / 3.0;
  p.beta = cs2 / (2.0 * nu + cs2);
  p.rho0 = (double)(float)rho0;
  p.betaf = (float)p.beta;
  p.rho0f = (float)p.rho0;
  p.unshifted = 0;
  p.secant_iters = 1;
  // the exact decision of elbm_step's default; without a buffer the
  // undecided nodes take the fixup's gathering path
  p.exact = 1;
  p.div_nx.init((unsigned)nx);
  p.div_ny.init((unsigned)ny);

  const int diag = stats_out != nullptr;
  int grid = 0;
  e = lattice == ELBM_D2Q9
          ? launch_fp32_formula_d2q9(diag, 0, p, 0, 256, stream, &grid)
          : launch_fp32_formula_d3q27(diag, 0, p, 0, 256, stream, &grid);
  if (e != cudaSuccess) return fail(ELBM_ECUDA, cudaGetErrorString(e));
  const int fgrid = grid < 152 ? grid : 152;   // grid + fgrid <= rows (above)
  StepParams pf = p;
  pf.partials = partials + (size_t)grid * NSTAT;
  e = lattice == ELBM_D2Q9 ? launch_far_d2q9(diag, 0, pf, fgrid, stream)
                           : launch_far_d3q27(diag, 0, pf, fgrid, stream);
  if (e != cudaSuccess) return fail(ELBM_ECUDA, cudaGetErrorString(e));
  if (!diag) return ELBM_OK;

  e = launch_finish(partials, grid + fgrid, stats, stream);
  if (e != cudaSuccess) return fail(ELBM_ECUDA, cudaGetErrorString(e));
  double slots[NSTAT];
  unsigned flags = 0;
  e = cudaMemcpyAsync(slots, stats, sizeof(slots), cudaMemcpyDeviceToHost,
                      stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flags, counters + 2, sizeof(unsigned),
                        cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(ELBM_ECUDA, cudaGetErrorString(e));
  stats_from_slots(slots, p.rho0, n, 0, 0, stats_out);
  if (flags & NF_TIMEOUT)
    return fail(ELBM_ECUDA,
                "a bounded wait in the stream-collide kernel ran out; the "
                "step is incomplete");
  if (flags & NF_BAD_NEG)
    return fail(ELBM_ENEGATIVE, "a node had a population <= 0");
  if (flags & NF_BAD_NONFINITE)
    return fail(ELBM_ENONFINITE, "a node had non-finite moments or |u| >= 1");
  return ELBM_OK;
}

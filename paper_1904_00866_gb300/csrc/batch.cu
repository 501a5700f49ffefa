// Host runtime of the batched multi-lattice stepper (C ABI elbm_batch_*).
//
// A batch owns up to kBatchMaxMembers independent periodic lattices
// (FP32-shifted storage, FORMULA alpha), each with its own type, size and
// viscosity, and advances them in bursts of steps.  A burst is launched as a
// captured CUDA graph (k_batch, k_batch_refine, k_batch_fixup per step) when its length
// equals the tuned burst length, else as direct launches.  The member table
// and tile prefix are copied to the device before each burst; the graph
// reads them at run time, so it stays valid when members come and go.
//
// The autotuner times dry steps (read buf[p], write buf[p^1] without
// advancing p, so the state is untouched) for each candidate block size and
// blocks-per-SM, and keeps the fastest per membership signature (lattice
// types present and the power-of-two class of the total node count) in a
// process-wide cache, optionally persisted as JSON in the file named by
// ELBM_AUTOTUNE_CACHE.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/elbm.h"
#include "batch.cuh"
#include "internal.h"
#include "io_kernels.cuh"

namespace elbm {
namespace {

struct TuneResult {
  int threads = 256;
  int blocks_per_sm = 2;
};

std::mutex g_tune_mu;
std::map<std::string, TuneResult> g_tune_cache;
bool g_tune_loaded = false;

void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("ELBM_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  // one entry per line: {"key": "...", "threads": T, "blocks_per_sm": B}
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    char key[900];
    int t = 0, b = 0;
    if (sscanf(line, " {\"key\": \"%899[^\"]\", \"threads\": %d, "
                     "\"blocks_per_sm\": %d}", key, &t, &b) == 3 &&
        (t == 128 || t == 256) && b >= 1 && b <= 8) {
      g_tune_cache[key] = TuneResult{t, b};
    }
  }
  fclose(f);
}

void tune_cache_save() {
  const char* path = getenv("ELBM_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  for (const auto& kv : g_tune_cache)
    fprintf(f, "{\"key\": \"%s\", \"threads\": %d, \"blocks_per_sm\": %d}\n",
            kv.first.c_str(), kv.second.threads, kv.second.blocks_per_sm);
  fclose(f);
}

// Dynamic shared memory of k_batch: the gather stages and `cap` member
// descriptors.
int batch_smem(int tb, int cap) {
  return 2 * 27 * tb * (int)sizeof(float) + cap * (int)sizeof(MemberDesc);
}

// Member-descriptor capacity staged for `count` members: a multiple of 16,
// so that members joining a batch rarely change the launch's smem size.
int desc_cap_for(int count) { return (count + 15) / 16 * 16; }

template <int TB, int DIAG>
cudaError_t launch_batch_kernel(const BatchParams& bp, int grid,
                                cudaStream_t s) {
  auto k = k_batch<TB, DIAG>;
  const int smem = batch_smem(TB, bp.desc_cap);
  k<<<grid, TB, smem, s>>>(bp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch(int tb, int diag, const BatchParams& bp, int grid,
                         cudaStream_t s) {
  if (tb == 128)
    return diag ? launch_batch_kernel<128, 1>(bp, grid, s)
                : launch_batch_kernel<128, 0>(bp, grid, s);
  return diag ? launch_batch_kernel<256, 1>(bp, grid, s)
              : launch_batch_kernel<256, 0>(bp, grid, s);
}

cudaError_t launch_batch_refine(int diag, const BatchParams& bp, int blocks,
                                cudaStream_t s) {
  if (blocks > kMaxRefineBlocks) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = 2 * sms;   // two 128-register blocks per SM
  if (diag)
    k_batch_refine<1><<<grid, 256, 0, s>>>(bp, blocks);
  else
    k_batch_refine<0><<<grid, 256, 0, s>>>(bp, blocks);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_fixup(int diag, const BatchParams& bp,
                               cudaStream_t s) {
  if (diag)
    k_batch_fixup<1><<<152, 256, 0, s>>>(bp);
  else
    k_batch_fixup<0><<<152, 256, 0, s>>>(bp);
  count_launch();
  return cudaGetLastError();
}

int max_blocks_per_sm(int tb, int cap) {
  int per_sm = 0;
  // the attribute allows the largest table; the query uses this one
  const int smem_max = batch_smem(tb, kBatchMaxMembers);
  const int smem = batch_smem(tb, cap);
  if (tb == 128) {
    cudaFuncSetAttribute(k_batch<128, 0>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    cudaFuncSetAttribute(k_batch<128, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<128, 0>,
                                                  tb, smem);
  } else {
    cudaFuncSetAttribute(k_batch<256, 0>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    cudaFuncSetAttribute(k_batch<256, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<256, 0>,
                                                  tb, smem);
  }
  return per_sm < 1 ? 1 : per_sm;
}

}  // namespace
}  // namespace elbm

using namespace elbm;

struct BatchMember {
  bool live = false;
  elbm_lattice lattice = ELBM_D2Q9;
  int nx = 0, ny = 0, nz = 0;
  unsigned n = 0;
  double nu = 0, beta = 0, rho0 = 1.0;
  float* buf[2] = {nullptr, nullptr};
  float* alpha_map = nullptr;
  int parity = 0;
  long long steps_done = 0;
  long long remaining = LLONG_MAX;
  bool stats_valid = false;
  long long stats_step = 0;
  MemberStats stats;
  size_t bytes = 0;
};

struct elbm_batch {
  int max_members = 0;
  std::vector<BatchMember> m;
  cudaStream_t stream = nullptr;
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* alloc_ctx = nullptr;
  // device tables
  MemberDesc* d_desc = nullptr;
  unsigned* d_begin = nullptr;
  unsigned char* d_tmem = nullptr;   // member index of every tile
  size_t tmem_cap = 0;
  int* d_count = nullptr;
  MemberStats* d_stats = nullptr;
  unsigned* d_far_count = nullptr;   // [2] deferred nodes by step parity
  float* d_refine = nullptr;         // undecided-node buffer
  unsigned refine_cap = 0;
  unsigned* d_refine_counts = nullptr;   // entries per batch-kernel block
  int exact = 1;                         // second stage of undecided nodes
  unsigned* d_err = nullptr;
  unsigned long long* d_queue = nullptr;
  size_t queue_cap = 0;
  // host mirrors
  std::vector<MemberDesc> h_desc;
  std::vector<unsigned> h_begin;
  std::vector<unsigned char> h_tmem;
  std::vector<int> h_member_of;   // position in the tile list -> member id
  // options
  int diag_every = 0;
  int burst = 16;
  int use_graphs = 1;
  int autotune = 1;
  int tb = 256, bps = 2;
  bool tuned = false;
  // graph cache
  cudaGraphExec_t exec = nullptr;
  int exec_burst = 0, exec_tb = 0, exec_grid = 0, exec_diag = -1;
  int exec_cap = 0;   // member-descriptor capacity the graph was captured with
  size_t bytes = 0;
  long long bursts = 0;
  std::string err;
};

static elbm_status bfail(elbm_batch* b, elbm_status st, const std::string& m) {
  if (b)
    b->err = m;
  else
    set_global_error(m);
  return st;
}

static void* balloc(elbm_batch* b, size_t bytes) {
  void* p = nullptr;
  if (b->alloc) {
    p = b->alloc(bytes, b->alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->bytes += bytes;
  return p;
}

static void bfree(elbm_batch* b, void* p, size_t bytes) {
  if (!p) return;
  b->bytes -= bytes;
  if (b->free_fn)
    b->free_fn(p, b->alloc_ctx);
  else
    cudaFree(p);
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static elbm_status ensure_tables(elbm_batch* b) {
  if (b->d_desc) return ELBM_OK;
  b->d_desc = (MemberDesc*)balloc(b, sizeof(MemberDesc) * kBatchMaxMembers);
  b->d_begin = (unsigned*)balloc(b, sizeof(unsigned) * (kBatchMaxMembers + 1));
  b->d_count = (int*)balloc(b, 256);
  b->d_stats = (MemberStats*)balloc(b, sizeof(MemberStats) * kBatchMaxMembers);
  b->d_far_count = (unsigned*)balloc(b, 256);
  b->d_err = (unsigned*)balloc(b, 256);
  b->d_refine_counts =
      (unsigned*)balloc(b, sizeof(unsigned) * kMaxRefineBlocks);
  if (!b->d_desc || !b->d_begin || !b->d_count || !b->d_stats ||
      !b->d_far_count || !b->d_err || !b->d_refine_counts)
    return bfail(b, ELBM_ENOMEM, "batch table allocation failed");
  cudaMemsetAsync(b->d_err, 0, 256, b->stream);
  cudaMemsetAsync(b->d_far_count, 0, 256, b->stream);
  // kernel attributes are set here, never during a graph capture
  max_blocks_per_sm(128, 16);
  max_blocks_per_sm(256, 16);
  return ELBM_OK;
}

static void drop_graph(elbm_batch* b);

static elbm_status ensure_queue(elbm_batch* b) {
  size_t need = 0;
  for (auto& mm : b->m)
    if (mm.live) need += mm.n;
  if (need <= b->queue_cap) return ELBM_OK;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);   // the captured launches hold the old queue pointer
  const size_t old_cap = b->queue_cap;
  bfree(b, b->d_queue, old_cap * sizeof(unsigned long long));
  b->d_queue = nullptr;
  b->queue_cap = 0;
  // geometric growth: admissions rarely have to wait for a reallocation
  const size_t cap = std::max(need + need / 4 + 1024, 2 * old_cap);
  b->d_queue = (unsigned long long*)balloc(b, cap * sizeof(unsigned long long));
  if (!b->d_queue) return bfail(b, ELBM_ENOMEM, "far queue allocation failed");
  b->queue_cap = cap;
  // undecided-node buffer: a sixteenth of the queue, at least 65,536
  // entries (a full buffer falls back to the gathering queue)
  bfree(b, b->d_refine,
        sizeof(float) * kBatchRecord * (size_t)b->refine_cap);
  const size_t rcap =
      std::min<size_t>(0xffffffffu, std::max<size_t>(cap / 16, 65536));
  b->d_refine =
      (float*)balloc(b, sizeof(float) * kBatchRecord * rcap);
  b->refine_cap = b->d_refine ? (unsigned)rcap : 0u;
  return ELBM_OK;
}

static BatchParams batch_params(elbm_batch* b) {
  BatchParams bp;
  bp.members = b->d_desc;
  bp.tile_begin = b->d_begin;
  bp.tile_member = b->d_tmem;
  bp.desc_cap = desc_cap_for((int)b->h_desc.size());
  bp.count = b->d_count;
  bp.stats = b->d_stats;
  bp.far_queue = b->d_queue;
  bp.far_cap = (unsigned)std::min<size_t>(b->queue_cap, 0xffffffffu);
  bp.far_count = b->d_far_count;
  bp.refine_buf = b->d_refine;
  bp.refine_cap = b->refine_cap;
  bp.refine_counts = b->d_refine_counts;
  bp.exact = b->exact;
  bp.err_flags = b->d_err;
  bp.step = 0;
  return bp;
}

// Member table for the next burst: members with steps > 0 in tile order.
// `dry` keeps every member at steps_left = 1 without advancing anything.
static int build_tables(elbm_batch* b, int burst, bool diag, int tb,
                        bool dry) {
  b->h_desc.clear();
  b->h_begin.assign(1, 0u);
  b->h_member_of.clear();
  for (int id = 0; id < (int)b->m.size(); ++id) {
    BatchMember& mm = b->m[id];
    if (!mm.live) continue;
    const long long take =
        dry ? 1 : std::min<long long>((long long)burst, mm.remaining);
    if (take <= 0) continue;
    MemberDesc d;
    memset(&d, 0, sizeof(d));
    d.buf[0] = mm.buf[0];
    d.buf[1] = mm.buf[1];
    d.alpha_map = mm.alpha_map;
    d.n = mm.n;
    d.nx = mm.nx;
    d.ny = mm.ny;
    d.nz = mm.nz;
    d.div_nx.init((unsigned)mm.nx);
    d.div_ny.init((unsigned)mm.ny);
    d.beta = (float)mm.beta;
    d.beta64 = mm.beta;
    d.rho0f = (float)mm.rho0;
    d.rho0 = mm.rho0;
    d.lattice = mm.lattice == ELBM_D3Q27 ? 1 : 0;
    d.parity0 = mm.parity;
    d.steps_left = (int)take;
    d.diag = diag ? 1 : 0;
    b->h_desc.push_back(d);
    b->h_member_of.push_back(id);
    b->h_begin.push_back(b->h_begin.back() + (mm.n + tb - 1) / tb);
  }
  b->h_tmem.resize(b->h_begin.back());
  for (size_t k = 0; k + 1 < b->h_begin.size(); ++k)
    std::fill(b->h_tmem.begin() + b->h_begin[k],
              b->h_tmem.begin() + b->h_begin[k + 1], (unsigned char)k);
  return (int)b->h_desc.size();
}

static elbm_status upload_tables(elbm_batch* b) {
  const int count = (int)b->h_desc.size();
  const size_t tiles = b->h_tmem.size();
  if (tiles > b->tmem_cap) {
    // the captured launches hold the table pointer: re-capture after growth
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    const size_t cap = std::max(tiles + tiles / 4 + 4096, 2 * b->tmem_cap);
    bfree(b, b->d_tmem, b->tmem_cap);
    b->d_tmem = nullptr;
    b->tmem_cap = 0;
    b->d_tmem = (unsigned char*)balloc(b, cap);
    if (!b->d_tmem) return bfail(b, ELBM_ENOMEM, "tile table allocation failed");
    b->tmem_cap = cap;
  }
  cudaError_t e = cudaSuccess;
  if (tiles > 0)
    e = cudaMemcpyAsync(b->d_tmem, b->h_tmem.data(), tiles,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && count > 0)
    e = cudaMemcpyAsync(b->d_desc, b->h_desc.data(),
                        sizeof(MemberDesc) * count, cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_begin, b->h_begin.data(),
                        sizeof(unsigned) * (count + 1), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_count, &count, sizeof(int),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_far_count, 0, 2 * sizeof(unsigned), b->stream);
  // the sources are pageable host memory: each copy is staged before the
  // call returns, so the host tables may be rebuilt right away
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  return ELBM_OK;
}

static elbm_status reset_stats(elbm_batch* b) {
  std::vector<MemberStats> init(kBatchMaxMembers);
  for (auto& s : init) {
    memset(&s, 0, sizeof(s));
    s.amin_bits = 0x7f800000u;   // +inf
    s.amax_bits = 0u;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_stats, init.data(),
                                  sizeof(MemberStats) * kBatchMaxMembers,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  return ELBM_OK;
}

static cudaError_t run_steps(elbm_batch* b, int nsteps, int diag, int grid) {
  BatchParams bp = batch_params(b);
  // Both deferred-node counters start every run at zero (within the run,
  // step s's fixup clears the counter of step s + 1).  Without this the
  // autotuner's dry steps, which all run as step 0, would never clear
  // counter 0 and its stale entries would pile up.
  cudaError_t e0 =
      cudaMemsetAsync(b->d_far_count, 0, 2 * sizeof(unsigned), b->stream);
  if (e0 != cudaSuccess) return e0;
  for (int s = 0; s < nsteps; ++s) {
    bp.step = s;
    cudaError_t e = launch_batch(b->tb, diag, bp, grid, b->stream);
    if (e != cudaSuccess) return e;
    if (bp.exact) {
      e = launch_batch_refine(diag, bp, grid, b->stream);
      if (e != cudaSuccess) return e;
    }
    e = launch_batch_fixup(diag, bp, b->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static void drop_graph(elbm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->exec_burst = 0;
}

static elbm_status autotune(elbm_batch* b) {
  // Signature of the membership: which lattice types are present and the
  // power-of-two class of the total node count.  The best launch shape
  // depends on these (per-node cost, tail of the tile list), not on the
  // individual members, so members joining or leaving rarely re-tune.
  std::string key;
  {
    bool q9 = false, q27 = false;
    unsigned long long total = 0;
    for (auto& mm : b->m) {
      if (!mm.live) continue;
      (mm.lattice == ELBM_D3Q27 ? q27 : q9) = true;
      total += mm.n;
    }
    int cls = 0;
    while ((1ull << cls) < total) ++cls;
    key = std::string(q9 ? "Q9" : "") + (q27 ? "Q27" : "") + ":" +
          std::to_string(cls);
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      b->tb = it->second.threads;
      b->bps = it->second.blocks_per_sm;
      b->tuned = true;
      return ELBM_OK;
    }
  }
  const int sms = sm_count();
  float best = 1e30f;
  TuneResult bestr{b->tb, b->bps};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int tb : {128, 256}) {
    const int maxb = max_blocks_per_sm(tb, desc_cap_for((int)b->h_desc.size()));
    for (int bps = 1; bps <= maxb; ++bps) {
      b->tb = tb;
      if (build_tables(b, 1, false, tb, true) == 0) break;
      elbm_status st = upload_tables(b);
      if (st) return st;
      const int grid = sms * bps;
      run_steps(b, 1, 0, grid);   // warm-up (dry: steps_left = 1, step 0)
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 3; ++r) run_steps(b, 1, 0, grid);
      cudaEventRecord(e1, b->stream);
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(ce));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bestr = TuneResult{tb, bps};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tb = bestr.threads;
  b->bps = bestr.blocks_per_sm;
  b->tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = bestr;
  tune_cache_save();
  return ELBM_OK;
}

// member geometry helpers for init / readout
static Geo member_geo(const BatchMember& mm) {
  Geo g;
  g.nx = mm.nx;
  g.ny = mm.ny;
  g.nz = mm.nz;
  g.n = mm.n;
  g.ps = mm.n;
  g.rho0 = mm.rho0;
  g.shifted = 1;
  return g;
}

extern "C" {

elbm_status elbm_batch_create(elbm_batch** out, int max_members) {
  if (!out) return bfail(nullptr, ELBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_members < 1 || max_members > kBatchMaxMembers)
    return bfail(nullptr, ELBM_EINVAL,
                 "max_members must be in [1, " +
                     std::to_string(kBatchMaxMembers) + "]");
  elbm_batch* b = new elbm_batch();
  b->max_members = max_members;
  b->m.resize(max_members);
  *out = b;
  return ELBM_OK;
}

void elbm_batch_destroy(elbm_batch* b) {
  if (!b) return;
  if (b->d_desc) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& mm : b->m) {
    if (!mm.live) continue;
    bfree(b, mm.buf[0], mm.bytes / 2);
    bfree(b, mm.buf[1], mm.bytes / 2);
    if (mm.alpha_map) bfree(b, mm.alpha_map, sizeof(float) * mm.n);
  }
  bfree(b, b->d_queue, b->queue_cap * sizeof(unsigned long long));
  bfree(b, b->d_desc, sizeof(MemberDesc) * kBatchMaxMembers);
  bfree(b, b->d_begin, sizeof(unsigned) * (kBatchMaxMembers + 1));
  bfree(b, b->d_tmem, b->tmem_cap);
  bfree(b, b->d_count, 256);
  bfree(b, b->d_stats, sizeof(MemberStats) * kBatchMaxMembers);
  bfree(b, b->d_far_count, 256);
  bfree(b, b->d_refine_counts, sizeof(unsigned) * kMaxRefineBlocks);
  bfree(b, b->d_refine, sizeof(float) * kBatchRecord * (size_t)b->refine_cap);
  bfree(b, b->d_err, 256);
  delete b;
}

const char* elbm_batch_last_error(const elbm_batch* b) {
  return b ? b->err.c_str() : elbm_last_error(nullptr);
}

elbm_status elbm_batch_set_stream(elbm_batch* b, void* s) {
  if (!b) return ELBM_EINVAL;
  b->stream = (cudaStream_t)s;
  drop_graph(b);
  return ELBM_OK;
}

elbm_status elbm_batch_set_allocator(elbm_batch* b,
                                     void* (*alloc)(size_t, void*),
                                     void (*free_fn)(void*, void*),
                                     void* ctx) {
  if (!b) return ELBM_EINVAL;
  if (b->d_desc) return bfail(b, ELBM_ESTATE, "allocator must be set first");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return bfail(b, ELBM_EINVAL, "alloc and free must both be set or NULL");
  b->alloc = alloc;
  b->free_fn = free_fn;
  b->alloc_ctx = ctx;
  return ELBM_OK;
}

elbm_status elbm_batch_set_options(elbm_batch* b, int diag_every, int burst,
                                   int use_graphs, int autotune_on) {
  if (!b) return ELBM_EINVAL;
  if (diag_every < 0 || burst < 1 || burst > 4096)
    return bfail(b, ELBM_EINVAL, "invalid batch options");
  b->diag_every = diag_every;
  if (burst != b->burst) drop_graph(b);
  b->burst = burst;
  b->use_graphs = use_graphs != 0;
  b->autotune = autotune_on != 0;
  return ELBM_OK;
}

elbm_status elbm_batch_add(elbm_batch* b, const elbm_member_spec* spec,
                           const double* rho, const double* u, int* id_out) {
  if (!b || !spec || !rho || !u || !id_out)
    return bfail(b, ELBM_EINVAL, "NULL argument");
  *id_out = -1;
  if (spec->lattice != ELBM_D2Q9 && spec->lattice != ELBM_D3Q27)
    return bfail(b, ELBM_EINVAL, spec->lattice == ELBM_D1Q3
                                     ? "batch members are D2Q9 or D3Q27"
                                     : "unknown lattice");
  if (spec->nx < 1 || spec->ny < 1 || spec->nz < 1 ||
      (spec->lattice == ELBM_D2Q9 && spec->nz != 1))
    return bfail(b, ELBM_EINVAL, "invalid lattice dimensions");
  if (!(spec->nu > 0.0)) return bfail(b, ELBM_EINVAL, "nu must be > 0");
  const long long n = (long long)spec->nx * spec->ny * spec->nz;
  const int q = spec->lattice == ELBM_D2Q9 ? 9 : 27;
  if ((long long)q * n >= (1LL << 32))
    return bfail(b, ELBM_EINVAL, "member too large for the batched kernel");
  int id = -1;
  for (int k = 0; k < b->max_members; ++k)
    if (!b->m[k].live) {
      id = k;
      break;
    }
  if (id < 0) return bfail(b, ELBM_ESTATE, "batch is full");
  elbm_status st = ensure_tables(b);
  if (st) return st;
  double sum = 0.0;
  for (long long k = 0; k < n; ++k) {
    if (!(rho[k] > 0.0)) return bfail(b, ELBM_EINVAL, "rho must be > 0");
    sum += rho[k];
  }
  const int d = spec->lattice == ELBM_D2Q9 ? 2 : 3;
  for (long long k = 0; k < (long long)d * n; ++k)
    if (!(u[k] > -1.0 && u[k] < 1.0))
      return bfail(b, ELBM_EINVAL, "|u| must be < 1");
  BatchMember mm;
  mm.lattice = spec->lattice;
  mm.nx = spec->nx;
  mm.ny = spec->ny;
  mm.nz = spec->nz;
  mm.n = (unsigned)n;
  mm.nu = spec->nu;
  mm.beta = (1.0 / 3.0) / (2.0 * spec->nu + 1.0 / 3.0);   // Eq. (2)
  mm.rho0 = (double)(float)(sum / (double)n);
  const size_t half = sizeof(float) * (size_t)q * n;
  mm.buf[0] = (float*)balloc(b, half);
  mm.buf[1] = (float*)balloc(b, half);
  const size_t fb = sizeof(double) * (1 + d) * n;
  double* tmp = (double*)balloc(b, fb);
  if (!mm.buf[0] || !mm.buf[1] || !tmp) {
    bfree(b, mm.buf[0], mm.buf[0] ? half : 0);
    bfree(b, mm.buf[1], mm.buf[1] ? half : 0);
    bfree(b, tmp, tmp ? fb : 0);
    return bfail(b, ELBM_ENOMEM, "member allocation failed");
  }
  mm.bytes = 2 * half;
  cudaMemcpyAsync(tmp, rho, sizeof(double) * n, cudaMemcpyHostToDevice,
                  b->stream);
  cudaMemcpyAsync(tmp + n, u, sizeof(double) * d * n, cudaMemcpyHostToDevice,
                  b->stream);
  Geo g = member_geo(mm);
  const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
  if (mm.lattice == ELBM_D2Q9)
    k_init_feq<D2Q9, float><<<grid, 256, 0, b->stream>>>(g, tmp, tmp + n,
                                                          mm.buf[0], b->d_err);
  else
    k_init_feq<D3Q27, float><<<grid, 256, 0, b->stream>>>(g, tmp, tmp + n,
                                                           mm.buf[0], b->d_err);
  count_launch();
  cudaError_t e = cudaStreamSynchronize(b->stream);
  bfree(b, tmp, fb);
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  mm.live = true;
  b->m[id] = mm;
  st = ensure_queue(b);
  if (st) return st;
  b->tuned = false;
  *id_out = id;
  return ELBM_OK;
}

elbm_status elbm_batch_remove(elbm_batch* b, int id) {
  if (!b || id < 0 || id >= b->max_members || !b->m[id].live)
    return bfail(b, ELBM_EINVAL, "no such member");
  cudaStreamSynchronize(b->stream);
  BatchMember& mm = b->m[id];
  bfree(b, mm.buf[0], mm.bytes / 2);
  bfree(b, mm.buf[1], mm.bytes / 2);
  if (mm.alpha_map) bfree(b, mm.alpha_map, sizeof(float) * mm.n);
  mm = BatchMember();
  b->tuned = false;
  return ELBM_OK;
}

elbm_status elbm_batch_set_steps(elbm_batch* b, int id, long long remaining) {
  if (!b || id < 0 || id >= b->max_members || !b->m[id].live)
    return bfail(b, ELBM_EINVAL, "no such member");
  if (remaining < 0) return bfail(b, ELBM_EINVAL, "remaining must be >= 0");
  b->m[id].remaining = remaining;
  return ELBM_OK;
}

elbm_status elbm_batch_member_info(elbm_batch* b, int id, long long* steps_done,
                                   long long* remaining) {
  if (!b || id < 0 || id >= b->max_members || !b->m[id].live)
    return bfail(b, ELBM_EINVAL, "no such member");
  if (steps_done) *steps_done = b->m[id].steps_done;
  if (remaining) *remaining = b->m[id].remaining;
  return ELBM_OK;
}

elbm_status elbm_batch_record_alpha(elbm_batch* b, int id, int enable) {
  if (!b || id < 0 || id >= b->max_members || !b->m[id].live)
    return bfail(b, ELBM_EINVAL, "no such member");
  BatchMember& mm = b->m[id];
  if (enable && !mm.alpha_map) {
    mm.alpha_map = (float*)balloc(b, sizeof(float) * mm.n);
    if (!mm.alpha_map) return bfail(b, ELBM_ENOMEM, "alpha map allocation");
  } else if (!enable && mm.alpha_map) {
    cudaStreamSynchronize(b->stream);
    bfree(b, mm.alpha_map, sizeof(float) * mm.n);
    mm.alpha_map = nullptr;
  }
  return ELBM_OK;
}

elbm_status elbm_batch_step(elbm_batch* b, long long nsteps) {
  if (!b) return ELBM_EINVAL;
  if (nsteps < 0) return bfail(b, ELBM_EINVAL, "nsteps must be >= 0");
  if (!b->d_desc) return bfail(b, ELBM_ESTATE, "batch has no members");
  if (b->autotune && !b->tuned) {
    // a changed launch shape makes the graph check below re-capture
    elbm_status st = autotune(b);
    if (st) return st;
  }
  const int grid = sm_count() * b->bps;
  long long left = nsteps;
  while (left > 0) {
    const int k = (int)std::min<long long>(left, (long long)b->burst);
    // statistics on the members' last step of every diag_every-th burst
    const bool diag = b->diag_every > 0 && b->bursts % b->diag_every == 0;
    const int count = build_tables(b, k, diag, b->tb, false);
    if (count == 0) break;
    elbm_status st = upload_tables(b);
    if (st) return st;
    if (diag) {
      st = reset_stats(b);
      if (st) return st;
    }
    int steps_here = 0;   // longest member participation in this burst
    for (auto& d : b->h_desc) steps_here = std::max(steps_here, d.steps_left);
    cudaError_t e = cudaSuccess;
    if (b->use_graphs && steps_here == b->burst && b->burst > 1) {
      if (!b->exec || b->exec_burst != b->burst || b->exec_tb != b->tb ||
          b->exec_grid != grid || b->exec_diag != (int)diag ||
          b->exec_cap != desc_cap_for(count)) {
        drop_graph(b);
        cudaStream_t cs;
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        cudaGraph_t graph;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaStream_t keep = b->stream;
          b->stream = cs;
          const long long before = elbm_launch_count();
          run_steps(b, b->burst, diag, grid);
          count_launches(before - elbm_launch_count());   // capture only
          b->stream = keep;
          e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) {
          e = cudaGraphInstantiate(&b->exec, graph, 0);
          cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess)
          return bfail(b, ELBM_ECUDA,
                       std::string("graph capture: ") + cudaGetErrorString(e));
        b->exec_burst = b->burst;
        b->exec_tb = b->tb;
        b->exec_cap = desc_cap_for(count);
        b->exec_grid = grid;
        b->exec_diag = diag;
      }
      e = cudaGraphLaunch(b->exec, b->stream);
      count_launches((b->exact ? 3 : 2) * b->burst);   // launches per step
    } else {
      e = run_steps(b, steps_here, diag, grid);
    }
    if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
    for (size_t t = 0; t < b->h_desc.size(); ++t) {
      BatchMember& mm = b->m[b->h_member_of[t]];
      const int took = b->h_desc[t].steps_left;
      if (diag) mm.stats_step = mm.steps_done + took - 1;
      mm.parity ^= (took & 1);
      mm.steps_done += took;
      if (mm.remaining != LLONG_MAX) mm.remaining -= took;
    }
    if (diag) {
      std::vector<MemberStats> hs(count);
      e = cudaMemcpyAsync(hs.data(), b->d_stats, sizeof(MemberStats) * count,
                          cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
      for (int t = 0; t < count; ++t) {
        BatchMember& mm = b->m[b->h_member_of[t]];
        mm.stats = hs[t];
        mm.stats_valid = true;
      }
    }
    b->bursts += 1;
    left -= k;
  }
  return ELBM_OK;
}

elbm_status elbm_batch_sync(elbm_batch* b) {
  if (!b) return ELBM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  if (!b->d_err) return ELBM_OK;
  unsigned flags = 0;
  e = cudaMemcpy(&flags, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  if (flags & NF_BAD_NEG)
    return bfail(b, ELBM_ENEGATIVE, "a node had a population <= 0");
  if (flags & NF_BAD_NONFINITE)
    return bfail(b, ELBM_ENONFINITE,
                 "a node had non-finite moments or |u| >= 1");
  return ELBM_OK;
}

static elbm_status member_check(elbm_batch* b, int id) {
  if (!b) return ELBM_EINVAL;
  if (id < 0 || id >= b->max_members || !b->m[id].live)
    return bfail(b, ELBM_EINVAL, "no such member");
  return elbm_batch_sync(b);
}

elbm_status elbm_batch_moments(elbm_batch* b, int id, double* rho_out,
                               double* u_out) {
  elbm_status st = member_check(b, id);
  if (st) return st;
  BatchMember& mm = b->m[id];
  const int d = mm.lattice == ELBM_D2Q9 ? 2 : 3;
  const size_t bytes = sizeof(double) * (1 + d) * mm.n;
  double* tmp = (double*)balloc(b, bytes);
  if (!tmp) return bfail(b, ELBM_ENOMEM, "staging allocation failed");
  Geo g = member_geo(mm);
  const int grid = (int)std::min<long long>((mm.n + 255) / 256, 4096);
  const void* f = mm.buf[mm.parity];
  if (mm.lattice == ELBM_D2Q9)
    k_moments<D2Q9, float><<<grid, 256, 0, b->stream>>>(g, f, tmp, tmp + mm.n);
  else
    k_moments<D3Q27, float><<<grid, 256, 0, b->stream>>>(g, f, tmp, tmp + mm.n);
  count_launch();
  cudaError_t e = cudaSuccess;
  if (rho_out)
    e = cudaMemcpyAsync(rho_out, tmp, sizeof(double) * mm.n,
                        cudaMemcpyDeviceToHost, b->stream);
  if (u_out && e == cudaSuccess)
    e = cudaMemcpyAsync(u_out, tmp + mm.n, sizeof(double) * d * mm.n,
                        cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  bfree(b, tmp, bytes);
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  if (e2 != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e2));
  return ELBM_OK;
}

elbm_status elbm_batch_get_populations(elbm_batch* b, int id, double* f_out) {
  elbm_status st = member_check(b, id);
  if (st) return st;
  if (!f_out) return bfail(b, ELBM_EINVAL, "NULL output");
  BatchMember& mm = b->m[id];
  const int q = mm.lattice == ELBM_D2Q9 ? 9 : 27;
  const size_t bytes = sizeof(double) * q * mm.n;
  double* tmp = (double*)balloc(b, bytes);
  if (!tmp) return bfail(b, ELBM_ENOMEM, "staging allocation failed");
  Geo g = member_geo(mm);
  const int grid = (int)std::min<long long>((mm.n + 255) / 256, 4096);
  const void* f = mm.buf[mm.parity];
  if (mm.lattice == ELBM_D2Q9)
    k_get_pop<D2Q9, float><<<grid, 256, 0, b->stream>>>(g, f, tmp);
  else
    k_get_pop<D3Q27, float><<<grid, 256, 0, b->stream>>>(g, f, tmp);
  count_launch();
  cudaError_t e =
      cudaMemcpyAsync(f_out, tmp, bytes, cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  bfree(b, tmp, bytes);
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  if (e2 != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e2));
  return ELBM_OK;
}

elbm_status elbm_batch_alpha_map(elbm_batch* b, int id, float* alpha_out) {
  elbm_status st = member_check(b, id);
  if (st) return st;
  BatchMember& mm = b->m[id];
  if (!mm.alpha_map || mm.steps_done == 0)
    return bfail(b, ELBM_ESTATE, "alpha map not recorded");
  cudaError_t e = cudaMemcpy(alpha_out, mm.alpha_map, sizeof(float) * mm.n,
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bfail(b, ELBM_ECUDA, cudaGetErrorString(e));
  return ELBM_OK;
}

elbm_status elbm_batch_entropy_stats(elbm_batch* b, int id,
                                     elbm_entropy_stats_t* out) {
  elbm_status st = member_check(b, id);
  if (st) return st;
  BatchMember& mm = b->m[id];
  if (!mm.stats_valid)
    return bfail(b, ELBM_ESTATE, "no burst has computed statistics");
  const MemberStats& s = mm.stats;
  memset(out, 0, sizeof(*out));
  out->step = mm.stats_step;
  out->n_nodes = (long long)s.nodes;
  out->mass = s.drho + mm.rho0 * (double)mm.n;
  out->momentum[0] = s.j0;
  out->momentum[1] = s.j1;
  out->momentum[2] = s.j2;
  out->kinetic_energy = s.ke;
  float amin, amax;
  memcpy(&amin, &s.amin_bits, sizeof(float));
  memcpy(&amax, &s.amax_bits, sizeof(float));
  out->alpha_min = amin;
  out->alpha_max = amax;
  out->alpha_sum = s.asum;
  out->n_accept_two = (long long)s.acc2;
  out->n_accept_star = (long long)s.acc2;
  out->n_formula = (long long)s.formula;
  out->n_band = (long long)s.band;
  out->n_far = (long long)s.far;
  out->n_degenerate = (long long)s.degen;
  return ELBM_OK;
}

elbm_status elbm_batch_set_decision(elbm_batch* b, elbm_decision decision) {
  if (!b) return ELBM_EINVAL;
  if (decision != ELBM_DECISION_EXACT && decision != ELBM_DECISION_CERTIFIED)
    return bfail(b, ELBM_EINVAL, "unknown decision mode");
  const int exact = decision == ELBM_DECISION_EXACT;
  if (exact != b->exact) drop_graph(b);   // the graph's launches differ
  b->exact = exact;
  return ELBM_OK;
}

elbm_status elbm_batch_tuning(const elbm_batch* b, int* threads,
                              int* blocks_per_sm, int* burst) {
  if (!b) return ELBM_EINVAL;
  if (threads) *threads = b->tb;
  if (blocks_per_sm) *blocks_per_sm = b->bps;
  if (burst) *burst = b->burst;
  return ELBM_OK;
}

size_t elbm_batch_device_bytes(const elbm_batch* b) { return b ? b->bytes : 0; }

}  // extern "C"

// The C ABI of libmochy (declared in include/mochy.h): contexts, memory
// accounting and the entry points.  Every computation runs in the kernels of
// the other files; this file only moves arguments and results.
#include <atomic>
#include <map>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "common.cuh"

namespace mochy {

static thread_local std::string t_last_error;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { t_last_error = msg; }

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e),
           what, file, line);
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? MOCHY_E_NOMEM : MOCHY_E_CUDA;
}

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// A kernel's dynamic shared-memory limit is one setting per device, shared by
// every host thread that launches the kernel; lowering it while another
// thread is about to launch with a larger size would make that launch fail.
// So the limit is only ever raised, under a lock.
int ensure_dynamic_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set;
  int dev = 0;
  MOCHY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[{dev, func}];
  if (bytes <= cur) return MOCHY_OK;
  MOCHY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return MOCHY_OK;
}

int dev_alloc(mochy_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->budget > 0 && ctx->held + (int64_t)bytes > ctx->budget)
    return fail(MOCHY_E_NOMEM, "device memory budget exceeded (" + std::to_string(ctx->held) +
                                   " + " + std::to_string(bytes) + " > " +
                                   std::to_string(ctx->budget) + " bytes)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(MOCHY_E_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->held += (int64_t)bytes;
  return MOCHY_OK;
}

void dev_free(mochy_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  if (bytes == 0) bytes = 16;
  ctx->held -= (int64_t)bytes;
}

int scratch(mochy_ctx* ctx, int slot, size_t bytes, void** p) {
  Buffer& b = ctx->scratch[slot];
  if (b.bytes < bytes) {
    if (b.p) {
      MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
      dev_free(ctx, b.p, b.bytes);
      b.p = nullptr;
      b.bytes = 0;
    }
    const size_t grow = bytes + bytes / 4 + 4096;
    MOCHY_TRY(dev_alloc(ctx, &b.p, grow));
    b.bytes = grow;
  }
  *p = b.p;
  return MOCHY_OK;
}

// frees the scratch arena (it grows with the largest call and is kept
// otherwise)
void release_scratch(mochy_ctx* ctx) {
  bool any = false;
  for (auto& b : ctx->scratch) any = any || b.p;
  if (!any) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& b : ctx->scratch) {
    if (b.p) dev_free(ctx, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
  }
}

static size_t graph_bytes(const mochy_ctx* c, int which) {
  switch (which) {
    case 0: return sizeof(int64_t) * (size_t)(c->n_edges + 1);
    case 1: return sizeof(int32_t) * (size_t)std::max<int64_t>(c->n_inc, 1);
    case 2: return (size_t)std::max<int64_t>(c->n_edges, 1);
    case 3: return sizeof(int64_t) * (size_t)(c->n_nodes + 1);
    case 4: return sizeof(int32_t) * (size_t)std::max<int64_t>(c->n_inc, 1);
  }
  return 0;
}

void release_projection(mochy_ctx* ctx) {
  const int64_t E = ctx->n_edges;
  release_split(ctx);
  if (ctx->nadj || ctx->noff) cudaStreamSynchronize(ctx->stream);
  if (ctx->nadj) {
    int64_t total = 2 * ctx->n_wedges;
    dev_free(ctx, ctx->nadj, (size_t)std::max<int64_t>(total, 1) * sizeof(uint2));
  }
  if (ctx->noff) dev_free(ctx, ctx->noff, sizeof(int64_t) * (size_t)(E + 1));
  if (ctx->ustart) dev_free(ctx, ctx->ustart, sizeof(int64_t) * (size_t)std::max<int64_t>(E, 1));
  if (ctx->uprefix) dev_free(ctx, ctx->uprefix, sizeof(int64_t) * (size_t)(E + 1));
  if (ctx->row_order)
    dev_free(ctx, ctx->row_order, sizeof(int32_t) * (size_t)std::max<int64_t>(E, 1));
  ctx->nadj = nullptr;
  ctx->noff = ctx->ustart = ctx->uprefix = nullptr;
  ctx->row_order = nullptr;
  ctx->projected = false;
  ctx->n_wedges = 0;
  ctx->max_deg = 0;
}

void release_graph(mochy_ctx* ctx) {
  release_projection(ctx);
  release_onthefly(ctx);
  if (ctx->eoff) {
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, ctx->eoff, graph_bytes(ctx, 0));
    dev_free(ctx, ctx->enode, graph_bytes(ctx, 1));
    dev_free(ctx, ctx->esize, graph_bytes(ctx, 2));
    dev_free(ctx, ctx->voff, graph_bytes(ctx, 3));
    dev_free(ctx, ctx->vedge, graph_bytes(ctx, 4));
  }
  if (ctx->d_nseg) dev_free(ctx, ctx->d_nseg, ctx->nseg_bytes);
  ctx->d_nseg = nullptr;
  ctx->nseg_bytes = 0;
  ctx->n_units = 1;
  ctx->h_nseg.clear();
  ctx->h_eseg.clear();
  ctx->eoff = nullptr;
  ctx->enode = nullptr;
  ctx->esize = nullptr;
  ctx->voff = nullptr;
  ctx->vedge = nullptr;
  ctx->n_nodes = ctx->n_edges = ctx->n_inc = 0;
  ctx->max_size = 0;
}

bool host_patterns(int kind, int32_t id, uint8_t* out);  // tables.cu

// Results staging: device int64[457] + double[4*457], mirrored in pinned host memory.
constexpr size_t kResBytes = 8 * 457 * 5 + 64;

// The exact count through the kernel the configuration selects.
static int exact_dispatch(mochy_ctx* ctx, unsigned long long* d_hist) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  if (ctx->exact_kernel == 1) return count_exact(ctx, nullptr, 0, d_hist);
  MOCHY_CUDA(cudaMemsetAsync(d_hist, 0, 432 * 8, ctx->stream));
  if (ctx->n_edges == 0) return MOCHY_OK;
  return count_exact_split(ctx, d_hist);
}

static int device_guard(mochy_ctx* ctx) {
  MOCHY_CUDA(cudaSetDevice(ctx->device));
  return MOCHY_OK;
}

}  // namespace mochy

using namespace mochy;

extern "C" {

void mochy_config_default(mochy_config* cfg) {
  if (!cfg) return;
  cfg->theta = 1;
  cfg->eps = 1.0;
  cfg->hbm_budget_bytes = 0;
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->exact_kernel = 0;
  cfg->dense_threshold = 0;
  cfg->rest_path = 0;
}

int mochy_create(mochy_ctx** out, const mochy_config* cfg_in) {
  if (!out) return fail(MOCHY_E_INVALID, "null output handle");
  *out = nullptr;
  mochy_config cfg;
  mochy_config_default(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.theta < 1) return fail(MOCHY_E_INVALID, "theta must be >= 1");
  if (!(cfg.eps >= 0.0)) return fail(MOCHY_E_INVALID, "eps must be >= 0");
  if (cfg.exact_kernel < 0 || cfg.exact_kernel > 1) return fail(MOCHY_E_INVALID, "bad exact_kernel");
  if (cfg.dense_threshold < 0) return fail(MOCHY_E_INVALID, "bad dense_threshold");
  if (cfg.rest_path < 0 || cfg.rest_path > 2) return fail(MOCHY_E_INVALID, "bad rest_path");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(MOCHY_E_CUDA, "no CUDA device is available");
  }
  if (cfg.device < 0 || cfg.device >= ndev) return fail(MOCHY_E_INVALID, "bad device ordinal");
  mochy_ctx* ctx = new (std::nothrow) mochy_ctx();
  if (!ctx) return fail(MOCHY_E_NOMEM, "host allocation failed");
  ctx->device = cfg.device;
  ctx->theta = cfg.theta;
  ctx->eps = cfg.eps;
  ctx->budget = cfg.hbm_budget_bytes;
  ctx->exact_kernel = cfg.exact_kernel;
  ctx->dense_thr = cfg.dense_threshold;
  ctx->rest_path = cfg.rest_path;
  memset(ctx->last_stats, 0, sizeof(ctx->last_stats));
  int rc = MOCHY_OK;
  auto bail = [&](int code) {
    mochy_destroy(ctx);
    return code;
  };
  if (cudaSetDevice(cfg.device) != cudaSuccess) return bail(fail(MOCHY_E_CUDA, "cudaSetDevice failed"));
  if (cfg.stream) {
    ctx->stream = (cudaStream_t)cfg.stream;
    ctx->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(MOCHY_E_CUDA, "cudaStreamCreate failed"));
    ctx->own_stream = true;
  }
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, cfg.device);
  ctx->num_sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, cfg.device);
  ctx->smem_optin = (size_t)v;
  void* p = nullptr;
  if ((rc = dev_alloc(ctx, &p, 432 * 8 + 64 + kResBytes)) < 0) return bail(rc);
  ctx->hist = (unsigned long long*)p;
  ctx->counters = (int32_t*)((char*)p + 432 * 8);
  if (cudaMallocHost(&ctx->pinned, kResBytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->pinned = nullptr;
    return bail(fail(MOCHY_E_NOMEM, "pinned host allocation failed"));
  }
  if ((rc = build_tables(ctx)) < 0) return bail(rc);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return bail(fail(MOCHY_E_CUDA, "table build failed"));
  *out = ctx;
  return MOCHY_OK;
}

int mochy_destroy(mochy_ctx* ctx) {
  if (!ctx) return MOCHY_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  release_graph(ctx);
  for (auto& b : ctx->scratch) {
    if (b.p) dev_free(ctx, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (ctx->hist) cudaFree(ctx->hist);
  if (ctx->stats) cudaFree(ctx->stats);
  if (ctx->tables.lut3) cudaFree(ctx->tables.lut3);
  if (ctx->kh_block) cudaFree(ctx->kh_block);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return MOCHY_OK;
}

int mochy_load_device(mochy_ctx* ctx, int64_t n_nodes, int64_t n_edges, const int64_t* d_off,
                      const int32_t* d_nodes, int64_t* n_dup) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (n_edges > 0 && (!d_off || !d_nodes)) return fail(MOCHY_E_INVALID, "null array");
  MOCHY_TRY(device_guard(ctx));
  return load_graph(ctx, n_nodes, n_edges, d_off, d_nodes, n_dup);
}

int mochy_load(mochy_ctx* ctx, int64_t n_nodes, int64_t n_edges, const int64_t* h_off,
               const int32_t* h_nodes, int64_t* n_dup) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (n_edges < 0 || n_nodes < 0) return fail(MOCHY_E_INVALID, "negative size");
  if (n_edges > 0 && (!h_off || !h_nodes)) return fail(MOCHY_E_INVALID, "null array");
  MOCHY_TRY(device_guard(ctx));
  if (n_edges == 0) return load_graph(ctx, n_nodes, 0, nullptr, nullptr, n_dup);
  if (h_off[0] != 0) return fail(MOCHY_E_INVALID, "offsets must start at 0");
  const int64_t total = h_off[n_edges];
  if (total < 0) return fail(MOCHY_E_INVALID, "bad offsets");
  if (total > (int64_t)n_edges * MOCHY_MAX_EDGE_SIZE)
    return fail(MOCHY_E_UNSUPPORTED, "hyperedge with more than 63 nodes");
  void* d = nullptr;
  const size_t bytes = (size_t)(n_edges + 1) * 8 + (size_t)std::max<int64_t>(total, 1) * 4 + 256;
  MOCHY_TRY(dev_alloc(ctx, &d, bytes));
  int64_t* d_off = (int64_t*)d;
  int32_t* d_nodes = (int32_t*)((char*)d + (((size_t)(n_edges + 1) * 8 + 255) & ~(size_t)255));
  int rc = MOCHY_OK;
  cudaError_t e1 = cudaMemcpyAsync(d_off, h_off, (size_t)(n_edges + 1) * 8,
                                   cudaMemcpyHostToDevice, ctx->stream);
  cudaError_t e2 = total > 0 ? cudaMemcpyAsync(d_nodes, h_nodes, (size_t)total * 4,
                                               cudaMemcpyHostToDevice, ctx->stream)
                             : cudaSuccess;
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    rc = cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaMemcpyAsync", __FILE__, __LINE__);
  } else {
    rc = load_graph(ctx, n_nodes, n_edges, d_off, d_nodes, n_dup);
  }
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, bytes);
  return rc;
}

int mochy_get_hypergraph(mochy_ctx* ctx, int64_t* n_nodes, int64_t* n_edges, int64_t* n_inc,
                         int64_t* h_off, int32_t* h_nodes) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  MOCHY_TRY(device_guard(ctx));
  if (n_nodes) *n_nodes = ctx->n_nodes;
  if (n_edges) *n_edges = ctx->n_edges;
  if (n_inc) *n_inc = ctx->n_inc;
  if (h_off && ctx->eoff)
    MOCHY_CUDA(cudaMemcpyAsync(h_off, ctx->eoff, (size_t)(ctx->n_edges + 1) * 8,
                               cudaMemcpyDeviceToHost, ctx->stream));
  if (h_nodes && ctx->enode && ctx->n_inc > 0)
    MOCHY_CUDA(cudaMemcpyAsync(h_nodes, ctx->enode, (size_t)ctx->n_inc * 4,
                               cudaMemcpyDeviceToHost, ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  return MOCHY_OK;
}

int mochy_project(mochy_ctx* ctx, int64_t* n_wedges, int32_t* max_deg) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (!ctx->eoff) return fail(MOCHY_E_INVALID, "no hypergraph loaded");
  MOCHY_TRY(device_guard(ctx));
  MOCHY_TRY(project_graph(ctx));
  if (n_wedges) *n_wedges = ctx->n_wedges;
  if (max_deg) *max_deg = ctx->max_deg;
  return MOCHY_OK;
}

int mochy_line_degrees(mochy_ctx* ctx, int64_t* h_deg) {
  if (!ctx || !h_deg) return fail(MOCHY_E_INVALID, "null argument");
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  MOCHY_TRY(device_guard(ctx));
  std::vector<int64_t> off((size_t)ctx->n_edges + 1);
  MOCHY_CUDA(cudaMemcpyAsync(off.data(), ctx->noff, off.size() * 8, cudaMemcpyDeviceToHost,
                             ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int64_t i = 0; i < ctx->n_edges; ++i) h_deg[i] = off[i + 1] - off[i];
  return MOCHY_OK;
}

static int fetch_counts(mochy_ctx* ctx, int64_t* out_h, int64_t* out_3h) {
  int64_t* d_counts = (int64_t*)((char*)ctx->counters + 64);
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters + 8, 0, 4, ctx->stream));
  MOCHY_TRY(finish_counts(ctx, ctx->hist, d_counts, d_counts + MOCHY_N_H));
  int64_t* h = (int64_t*)ctx->pinned;
  MOCHY_CUDA(cudaMemcpyAsync(h, d_counts, 457 * 8, cudaMemcpyDeviceToHost, ctx->stream));
  int32_t bad = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&bad, ctx->counters + 8, 4, cudaMemcpyDeviceToHost, ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  if (bad) return fail(MOCHY_E_CUDA, "internal error: an instance mapped to no motif");
  if (out_h) memcpy(out_h, h, MOCHY_N_H * 8);
  if (out_3h) memcpy(out_3h, h + MOCHY_N_H, MOCHY_N_3H * 8);
  return MOCHY_OK;
}

int mochy_count_exact(mochy_ctx* ctx, int64_t* out_h, int64_t* out_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  MOCHY_TRY(device_guard(ctx));
  MOCHY_TRY(exact_dispatch(ctx, ctx->hist));
  return fetch_counts(ctx, out_h, out_3h);
}

int mochy_count_exact_subset(mochy_ctx* ctx, const int32_t* h_anchors, int64_t n, int64_t* out_h,
                             int64_t* out_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (n < 0 || (n > 0 && !h_anchors)) return fail(MOCHY_E_INVALID, "bad anchors");
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  MOCHY_TRY(device_guard(ctx));
  std::vector<char> seen((size_t)ctx->n_edges, 0);
  for (int64_t a = 0; a < n; ++a) {
    if (h_anchors[a] < 0 || h_anchors[a] >= ctx->n_edges)
      return fail(MOCHY_E_INVALID, "anchor out of range");
    if (seen[(size_t)h_anchors[a]]) return fail(MOCHY_E_INVALID, "repeated anchor");
    seen[(size_t)h_anchors[a]] = 1;
  }
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, (size_t)std::max<int64_t>(n, 1) * 4));
  int rc = MOCHY_OK;
  if (n > 0 && cudaMemcpyAsync(d, h_anchors, (size_t)n * 4, cudaMemcpyHostToDevice,
                               ctx->stream) != cudaSuccess) {
    rc = fail(MOCHY_E_CUDA, "anchor copy failed");
  }
  if (rc == MOCHY_OK) rc = count_exact(ctx, (const int32_t*)d, n, ctx->hist);
  if (rc == MOCHY_OK && n == 0) {
    cudaMemsetAsync(ctx->hist, 0, 432 * 8, ctx->stream);
  }
  if (rc == MOCHY_OK) rc = fetch_counts(ctx, out_h, out_3h);
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, (size_t)std::max<int64_t>(n, 1) * 4);
  return rc;
}

int mochy_count_exact_rows(mochy_ctx* ctx, const int32_t* h_rows, int64_t n, int64_t* out_h,
                           int64_t* out_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (n < 0 || (n > 0 && !h_rows)) return fail(MOCHY_E_INVALID, "bad rows");
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  if (ctx->exact_kernel != 0) return fail(MOCHY_E_INVALID, "row subsets need the split kernel");
  MOCHY_TRY(device_guard(ctx));
  std::vector<char> seen((size_t)ctx->n_edges, 0);
  for (int64_t a = 0; a < n; ++a) {
    if (h_rows[a] < 0 || h_rows[a] >= ctx->n_edges)
      return fail(MOCHY_E_INVALID, "row out of range");
    if (seen[(size_t)h_rows[a]]) return fail(MOCHY_E_INVALID, "repeated row");
    seen[(size_t)h_rows[a]] = 1;
  }
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, (size_t)std::max<int64_t>(n, 1) * 4));
  int rc = MOCHY_OK;
  if (n > 0 && cudaMemcpyAsync(d, h_rows, (size_t)n * 4, cudaMemcpyHostToDevice,
                               ctx->stream) != cudaSuccess) {
    rc = fail(MOCHY_E_CUDA, "row copy failed");
  }
  if (rc == MOCHY_OK) rc = count_split_rows(ctx, (const int32_t*)d, n, ctx->hist);
  if (rc == MOCHY_OK) rc = fetch_counts(ctx, out_h, out_3h);
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, (size_t)std::max<int64_t>(n, 1) * 4);
  return rc;
}

int mochy_tune_dense_threshold(mochy_ctx* ctx, const int32_t* candidates, int32_t n_candidates,
                               double sample_fraction, uint64_t seed, int32_t* best,
                               int32_t* tried, double* ms) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (n_candidates < 0 || (n_candidates > 0 && !candidates))
    return fail(MOCHY_E_INVALID, "bad candidates");
  for (int32_t c = 0; c < n_candidates; ++c)
    if (candidates[c] < 2) return fail(MOCHY_E_INVALID, "thresholds must be at least 2");
  if (!(sample_fraction > 0.0 && sample_fraction <= 1.0))
    return fail(MOCHY_E_INVALID, "sample_fraction must lie in (0, 1]");
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  if (ctx->exact_kernel != 0 || ctx->n_units != 1)
    return fail(MOCHY_E_INVALID, "the tuner needs the split kernel on a lone hypergraph");
  MOCHY_TRY(device_guard(ctx));
  return tune_dense_threshold(ctx, candidates, n_candidates, sample_fraction, seed, best, tried,
                              ms);
}

int mochy_hyperedge_profile(mochy_ctx* ctx, int64_t* hp_h, int64_t* hp_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  MOCHY_TRY(device_guard(ctx));
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  const int64_t E = ctx->n_edges;
  if (E == 0) return MOCHY_OK;
  const size_t bytes = (size_t)E * 432 * 8;
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, bytes));
  std::vector<unsigned long long> h((size_t)E * 432);
  uint8_t t2h[432];
  int rc = hyperedge_profiles(ctx, (unsigned long long*)d);
  if (rc == MOCHY_OK &&
      (cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
       cudaMemcpyAsync(t2h, ctx->tables.t2h, 432, cudaMemcpyDeviceToHost, ctx->stream) !=
           cudaSuccess ||
       cudaStreamSynchronize(ctx->stream) != cudaSuccess))
    rc = fail(MOCHY_E_CUDA, "profile copy failed");
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, bytes);
  if (rc < 0) return rc;
  for (int64_t e = 0; e < E; ++e) {
    const unsigned long long* r = h.data() + (size_t)e * 432;
    if (r[0] != 0ull) return fail(MOCHY_E_CUDA, "internal error: an instance mapped to no motif");
    if (hp_3h)
      for (int t = 1; t <= MOCHY_N_3H; ++t) hp_3h[e * MOCHY_N_3H + t - 1] = (int64_t)r[t];
    if (hp_h) {
      int64_t* o = hp_h + e * MOCHY_N_H;
      for (int t = 0; t < MOCHY_N_H; ++t) o[t] = 0;
      for (int t = 1; t <= MOCHY_N_3H; ++t) o[t2h[t] - 1] += (int64_t)r[t];
    }
  }
  return MOCHY_OK;
}

int mochy_star_node_profile(mochy_ctx* ctx, int64_t* np_h, int64_t* np_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  MOCHY_TRY(device_guard(ctx));
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  const int64_t N = ctx->n_nodes;
  if (N == 0) return MOCHY_OK;
  const size_t bytes = (size_t)N * 432 * 8;
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, bytes));
  std::vector<unsigned long long> h((size_t)N * 432);
  uint8_t t2h[432];
  int rc = star_node_profiles(ctx, (unsigned long long*)d);
  if (rc == MOCHY_OK &&
      (cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
       cudaMemcpyAsync(t2h, ctx->tables.t2h, 432, cudaMemcpyDeviceToHost, ctx->stream) !=
           cudaSuccess ||
       cudaStreamSynchronize(ctx->stream) != cudaSuccess))
    rc = fail(MOCHY_E_CUDA, "profile copy failed");
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, bytes);
  if (rc < 0) return rc;
  for (int64_t v = 0; v < N; ++v) {
    const unsigned long long* r = h.data() + (size_t)v * 432;
    if (r[0] != 0ull) return fail(MOCHY_E_CUDA, "internal error: an instance mapped to no motif");
    if (np_3h)
      for (int t = 1; t <= MOCHY_N_3H; ++t) np_3h[v * MOCHY_N_3H + t - 1] = (int64_t)r[t];
    if (np_h) {
      int64_t* o = np_h + v * MOCHY_N_H;
      for (int t = 0; t < MOCHY_N_H; ++t) o[t] = 0;
      for (int t = 1; t <= MOCHY_N_3H; ++t) o[t2h[t] - 1] += (int64_t)r[t];
    }
  }
  return MOCHY_OK;
}

int mochy_radial_node_profile(mochy_ctx* ctx, int64_t* np_h, int64_t* np_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  MOCHY_TRY(device_guard(ctx));
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  const int64_t N = ctx->n_nodes;
  if (N == 0) return MOCHY_OK;
  const size_t bytes = (size_t)N * 432 * 8;
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, bytes));
  std::vector<unsigned long long> h((size_t)N * 432);
  uint8_t t2h[432];
  int rc = radial_node_profiles(ctx, (unsigned long long*)d);
  if (rc == MOCHY_OK &&
      (cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
       cudaMemcpyAsync(t2h, ctx->tables.t2h, 432, cudaMemcpyDeviceToHost, ctx->stream) !=
           cudaSuccess ||
       cudaStreamSynchronize(ctx->stream) != cudaSuccess))
    rc = fail(MOCHY_E_CUDA, "profile copy failed");
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, bytes);
  if (rc < 0) return rc;
  for (int64_t v = 0; v < N; ++v) {
    const unsigned long long* r = h.data() + (size_t)v * 432;
    if (r[0] != 0ull) return fail(MOCHY_E_CUDA, "internal error: an instance mapped to no motif");
    if (np_3h)
      for (int t = 1; t <= MOCHY_N_3H; ++t) np_3h[v * MOCHY_N_3H + t - 1] = (int64_t)r[t];
    if (np_h) {
      int64_t* o = np_h + v * MOCHY_N_H;
      for (int t = 0; t < MOCHY_N_H; ++t) o[t] = 0;
      for (int t = 1; t <= MOCHY_N_3H; ++t) o[t2h[t] - 1] += (int64_t)r[t];
    }
  }
  return MOCHY_OK;
}

int mochy_count_kh(mochy_ctx* ctx, int32_t k, const int32_t* thresholds, int64_t* out_h,
                   int64_t* out_kh, int64_t cap, int64_t* n_motifs) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (k < 2 || k > 4) return fail(MOCHY_E_UNSUPPORTED, "kh-motifs are provided for k = 2..4");
  if (k > 2 && !thresholds) return fail(MOCHY_E_INVALID, "thresholds needed");
  const int thr1 = k > 2 ? thresholds[0] : 1, thr2 = k > 3 ? thresholds[1] : thr1 + 1;
  if (k > 2 && (thr1 < 1 || thr1 > MOCHY_MAX_EDGE_SIZE))
    return fail(MOCHY_E_INVALID, "thresholds must lie in [1, 63]");
  if (k > 3 && (thr2 <= thr1 || thr2 > MOCHY_MAX_EDGE_SIZE))
    return fail(MOCHY_E_INVALID, "thresholds must ascend");
  MOCHY_TRY(device_guard(ctx));
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  MOCHY_TRY(build_kh_tables(ctx, k));
  const int n = ctx->kh_n;
  if (n_motifs) *n_motifs = n;
  if (out_kh && cap < n) return fail(MOCHY_E_INVALID, "out_kh holds fewer than X(k) entries");
  const size_t bytes = (size_t)(n + 1) * 8;
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, bytes));
  std::vector<unsigned long long> h((size_t)n + 1);
  std::vector<uint8_t> to_h((size_t)n + 1);
  int rc = count_kh(ctx, k, thr1, thr2, (unsigned long long*)d);
  if (rc == MOCHY_OK &&
      (cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
       cudaMemcpyAsync(to_h.data(), ctx->kh_to_h, (size_t)n + 1, cudaMemcpyDeviceToHost,
                       ctx->stream) != cudaSuccess ||
       cudaStreamSynchronize(ctx->stream) != cudaSuccess))
    rc = fail(MOCHY_E_CUDA, "kh count copy failed");
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, bytes);
  if (rc < 0) return rc;
  if (h[0] != 0ull) return fail(MOCHY_E_CUDA, "internal error: an instance mapped to no motif");
  if (out_kh)
    for (int t = 1; t <= n; ++t) out_kh[t - 1] = (int64_t)h[t];
  if (out_h) {
    for (int t = 0; t < MOCHY_N_H; ++t) out_h[t] = 0;
    for (int t = 1; t <= n; ++t) out_h[to_h[t] - 1] += (int64_t)h[t];
  }
  return MOCHY_OK;
}

int mochy_kh_pattern(mochy_ctx* ctx, int32_t k, int32_t id, uint8_t* regions_out) {
  if (!ctx || !regions_out) return fail(MOCHY_E_INVALID, "null argument");
  MOCHY_TRY(device_guard(ctx));
  MOCHY_TRY(build_kh_tables(ctx, k));
  if (id < 1 || id > ctx->kh_n) return fail(MOCHY_E_INVALID, "no such kh-motif");
  MOCHY_CUDA(cudaMemcpyAsync(regions_out, ctx->kh_pattern + (size_t)id * 7, 7,
                             cudaMemcpyDeviceToHost, ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  return MOCHY_OK;
}

int mochy_enumerate(mochy_ctx* ctx, int64_t capacity, int32_t* h_out, int64_t* n_instances) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (capacity < 0 || (capacity > 0 && !h_out)) return fail(MOCHY_E_INVALID, "bad output");
  MOCHY_TRY(device_guard(ctx));
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  const size_t bytes = (size_t)std::max<int64_t>(capacity, 1) * 5 * 4 + 256;
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, bytes));
  unsigned long long* cursor = (unsigned long long*)d;
  int32_t* rows = (int32_t*)((char*)d + 256);
  unsigned long long total = 0;
  int rc = enumerate_instances(ctx, capacity, rows, cursor);
  if (rc == MOCHY_OK &&
      (cudaMemcpyAsync(&total, cursor, 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
       cudaStreamSynchronize(ctx->stream) != cudaSuccess))
    rc = fail(MOCHY_E_CUDA, "enumeration failed");
  const int64_t written = std::min<int64_t>((int64_t)total, capacity);
  if (rc == MOCHY_OK && written > 0 &&
      (cudaMemcpyAsync(h_out, rows, (size_t)written * 5 * 4, cudaMemcpyDeviceToHost,
                       ctx->stream) != cudaSuccess ||
       cudaStreamSynchronize(ctx->stream) != cudaSuccess))
    rc = fail(MOCHY_E_CUDA, "enumeration copy failed");
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, bytes);
  if (rc < 0) return rc;
  if (n_instances) *n_instances = (int64_t)total;
  return MOCHY_OK;
}

int mochy_count_sampled_onthefly(mochy_ctx* ctx, int64_t samples, uint64_t seed,
                                 int64_t budget_bytes, int64_t* raw_h, int64_t* raw_3h,
                                 double* est_h, double* est_3h, int64_t* n_wedges) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (!ctx->eoff) return fail(MOCHY_E_INVALID, "no hypergraph loaded");
  if (ctx->n_units != 1) return fail(MOCHY_E_INVALID, "a lone hypergraph is needed");
  MOCHY_TRY(device_guard(ctx));
  unsigned long long* d_stats = nullptr;
  if (ctx->trace > 1) {
    if (!ctx->stats) {
      void* p;
      MOCHY_TRY(dev_alloc(ctx, &p, 88 * sizeof(unsigned long long)));
      ctx->stats = (unsigned long long*)p;
    }
    d_stats = ctx->stats;
  }
  MOCHY_TRY(count_sampled_onthefly(ctx, samples, seed, budget_bytes, ctx->hist, d_stats));
  int64_t* d_counts = (int64_t*)((char*)ctx->counters + 64);
  double* d_est = (double*)(d_counts + 457);
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters + 8, 0, 4, ctx->stream));
  MOCHY_TRY(finish_counts(ctx, ctx->hist, d_counts, d_counts + MOCHY_N_H));
  MOCHY_TRY(scale_estimates(ctx, d_counts, d_counts + MOCHY_N_H, MOCHY_A_PLUS,
                            (double)ctx->otf_wedges, samples, d_est, d_est + MOCHY_N_H));
  int64_t* h = (int64_t*)ctx->pinned;
  MOCHY_CUDA(cudaMemcpyAsync(h, d_counts, 457 * 16, cudaMemcpyDeviceToHost, ctx->stream));
  if (d_stats)
    MOCHY_CUDA(cudaMemcpyAsync(ctx->last_stats + 19, d_stats, 4 * 8, cudaMemcpyDeviceToHost,
                               ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  int32_t bad = 0;
  MOCHY_CUDA(cudaMemcpy(&bad, ctx->counters + 8, 4, cudaMemcpyDeviceToHost));
  if (bad) return fail(MOCHY_E_CUDA, "internal error: an instance mapped to no motif");
  const double* he = (const double*)(h + 457);
  if (raw_h) memcpy(raw_h, h, MOCHY_N_H * 8);
  if (raw_3h) memcpy(raw_3h, h + MOCHY_N_H, MOCHY_N_3H * 8);
  if (est_h) memcpy(est_h, he, MOCHY_N_H * 8);
  if (est_3h) memcpy(est_3h, he + MOCHY_N_H, MOCHY_N_3H * 8);
  if (n_wedges) *n_wedges = ctx->otf_wedges;
  return MOCHY_OK;
}

int mochy_count_sampled(mochy_ctx* ctx, int method, int64_t samples, uint64_t seed,
                        int64_t* raw_h, int64_t* raw_3h, double* est_h, double* est_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  MOCHY_TRY(device_guard(ctx));
  MOCHY_TRY(count_sampled(ctx, method, samples, seed, ctx->hist));
  int64_t* d_counts = (int64_t*)((char*)ctx->counters + 64);
  double* d_est = (double*)(d_counts + 457);
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters + 8, 0, 4, ctx->stream));
  MOCHY_TRY(finish_counts(ctx, ctx->hist, d_counts, d_counts + MOCHY_N_H));
  const double numer = method == MOCHY_A ? (double)ctx->n_edges : (double)ctx->n_wedges;
  MOCHY_TRY(scale_estimates(ctx, d_counts, d_counts + MOCHY_N_H, method, numer, samples, d_est,
                            d_est + MOCHY_N_H));
  int64_t* h = (int64_t*)ctx->pinned;
  MOCHY_CUDA(cudaMemcpyAsync(h, d_counts, 457 * 16, cudaMemcpyDeviceToHost, ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  const double* he = (const double*)(h + 457);
  if (raw_h) memcpy(raw_h, h, MOCHY_N_H * 8);
  if (raw_3h) memcpy(raw_3h, h + MOCHY_N_H, MOCHY_N_3H * 8);
  if (est_h) memcpy(est_h, he, MOCHY_N_H * 8);
  if (est_3h) memcpy(est_3h, he + MOCHY_N_H, MOCHY_N_3H * 8);
  return MOCHY_OK;
}

static int new_like(mochy_ctx* src, mochy_ctx** out) {
  mochy_config cfg;
  mochy_config_default(&cfg);
  cfg.theta = src->theta;
  cfg.eps = src->eps;
  cfg.device = src->device;
  cfg.hbm_budget_bytes = src->budget;
  cfg.stream = src->own_stream ? nullptr : (void*)src->stream;
  cfg.exact_kernel = src->exact_kernel;
  cfg.dense_threshold = src->dense_thr;
  cfg.rest_path = src->rest_path;
  return mochy_create(out, &cfg);
}

int mochy_randomize(mochy_ctx* src, uint64_t seed, uint32_t copy, mochy_ctx** out) {
  if (!src || !out) return fail(MOCHY_E_INVALID, "null argument");
  if (!src->eoff) return fail(MOCHY_E_INVALID, "no hypergraph loaded");
  *out = nullptr;
  MOCHY_TRY(device_guard(src));
  mochy_ctx* dst = nullptr;
  MOCHY_TRY(new_like(src, &dst));
  int rc = randomize_graph(src, seed, copy, dst);
  if (rc < 0) {
    mochy_destroy(dst);
    return rc;
  }
  *out = dst;
  return MOCHY_OK;
}

int mochy_profile(mochy_ctx* ctx, int32_t n_random, uint64_t seed, double* sig_h, double* cp_h,
                  double* sig_3h, double* cp_3h, int64_t* counts_h, int64_t* counts_3h) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (n_random <= 0) return fail(MOCHY_E_INVALID, "n_random must be positive");
  if (!ctx->eoff) return fail(MOCHY_E_INVALID, "no hypergraph loaded");
  MOCHY_TRY(device_guard(ctx));
  if (!ctx->projected) MOCHY_TRY(project_graph(ctx));
  const size_t rows = (size_t)n_random + 1;
  void* d = nullptr;
  const size_t bytes = rows * 457 * 8 + 457 * 16 + 64;
  MOCHY_TRY(dev_alloc(ctx, &d, bytes));
  int64_t* ch = (int64_t*)d;
  int64_t* c3 = ch + rows * MOCHY_N_H;
  double* out = (double*)(c3 + rows * MOCHY_N_3H);
  int32_t* degen = (int32_t*)(out + 2 * 457);
  int rc = exact_dispatch(ctx, ctx->hist);
  if (rc == MOCHY_OK) rc = finish_counts(ctx, ctx->hist, ch, c3);
  mochy_ctx* copy_ctx = nullptr;
  if (rc == MOCHY_OK) rc = new_like(ctx, &copy_ctx);
  for (int32_t c = 0; rc == MOCHY_OK && c < n_random; ++c) {
    rc = randomize_graph(ctx, seed, (uint32_t)c, copy_ctx);
    if (rc == MOCHY_OK) rc = project_graph(copy_ctx);
    if (rc == MOCHY_OK) rc = exact_dispatch(copy_ctx, copy_ctx->hist);
    if (rc == MOCHY_OK)
      rc = finish_counts(copy_ctx, copy_ctx->hist, ch + (size_t)(c + 1) * MOCHY_N_H,
                         c3 + (size_t)(c + 1) * MOCHY_N_3H);
    if (rc == MOCHY_OK && cudaStreamSynchronize(copy_ctx->stream) != cudaSuccess)
      rc = fail(MOCHY_E_CUDA, "copy count failed");
  }
  if (copy_ctx) mochy_destroy(copy_ctx);
  if (rc == MOCHY_OK) rc = significance_cp(ctx, ch, c3, n_random, ctx->eps, out, degen);
  int32_t hdeg[2] = {0, 0};
  if (rc == MOCHY_OK) {
    std::vector<double> hout(2 * 457);
    if (cudaMemcpyAsync(hout.data(), out, 2 * 457 * 8, cudaMemcpyDeviceToHost, ctx->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(hdeg, degen, 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) {
      rc = fail(MOCHY_E_CUDA, "result copy failed");
    }
    if (rc == MOCHY_OK && counts_h)
      cudaMemcpyAsync(counts_h, ch, rows * MOCHY_N_H * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (rc == MOCHY_OK && counts_3h)
      cudaMemcpyAsync(counts_3h, c3, rows * MOCHY_N_3H * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = fail(MOCHY_E_CUDA, "sync failed");
    if (rc == MOCHY_OK) {
      if (sig_h) memcpy(sig_h, hout.data(), MOCHY_N_H * 8);
      if (cp_h) memcpy(cp_h, hout.data() + MOCHY_N_H, MOCHY_N_H * 8);
      if (sig_3h) memcpy(sig_3h, hout.data() + 2 * MOCHY_N_H, MOCHY_N_3H * 8);
      if (cp_3h) memcpy(cp_3h, hout.data() + 2 * MOCHY_N_H + MOCHY_N_3H, MOCHY_N_3H * 8);
    }
  }
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, bytes);
  if (rc < 0) return rc;
  return (hdeg[0] || hdeg[1]) ? MOCHY_W_DEGENERATE_CP : MOCHY_OK;
}

int mochy_motif_pattern(int kind, int32_t id, uint8_t* regions_out) {
  if (!regions_out) return fail(MOCHY_E_INVALID, "null output");
  if (!host_patterns(kind, id, regions_out))
    return fail(MOCHY_E_INVALID, "unknown motif id, or no context created yet");
  return MOCHY_OK;
}

void* mochy_stream(mochy_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

int mochy_trace(mochy_ctx* ctx, int enable) {
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  ctx->trace = enable < 0 ? 0 : (enable > 2 ? 2 : enable);
  return MOCHY_OK;
}

int mochy_trace_read(mochy_ctx* ctx, char* buf, int64_t len) {
  if (!ctx || !buf || len <= 0) return fail(MOCHY_E_INVALID, "bad argument");
  std::string js = "{\"phases_ms\": {";
  for (int i = 0; i < ctx->n_phases; ++i) {
    char item[96];
    snprintf(item, sizeof(item), "%s\"%s\": %.6f", i ? ", " : "", ctx->phase_name[i],
             ctx->phase_ms[i]);
    js += item;
  }
  char tail[2048];
  const unsigned long long* st = ctx->last_stats;
  snprintf(tail, sizeof(tail),
           "}, \"dense_rows\": %lld, \"dense_threshold\": %d, \"dense_words\": %lld, "
           "\"heavy_nodes\": %lld, \"words_scanned\": %llu, \"candidates\": %llu, "
           "\"table_candidates\": %llu, \"exact_candidates\": %llu, \"light_corrections\": %llu, "
           "\"clk_setup\": %llu, \"clk_words\": %llu, \"clk_finish\": %llu, "
           "\"clk_groups\": %llu, \"clk_light\": %llu, \"clk_sort\": %llu, "
           "\"light_entries\": %llu, \"dense_hyperwedges\": %llu, \"light_nodes\": %llu, "
           "\"heavy_bitmaps\": %llu, \"slots_evicted\": %llu, \"slots_flushed_full\": %llu, "
           "\"dense_rows_counted\": %llu, \"otf_candidates\": %llu, \"otf_words\": %llu, "
           "\"otf_list_entries\": %llu, \"otf_exact\": %llu, \"otf_bitmaps\": %lld}",
           (long long)ctx->n_dense, ctx->dense_thr_used, (long long)ctx->wwords,
           (long long)ctx->n_heavy, st[0], st[1], st[2], st[3], st[4], st[5], st[6], st[7], st[8],
           st[9], st[10], st[11], st[12], st[13], st[14], st[16], st[17], st[18], st[19],
           st[20], st[21], st[22], (long long)ctx->otf_bitmaps);
  js += tail;
  if ((int64_t)js.size() + 1 > len) return fail(MOCHY_E_INVALID, "buffer too small");
  memcpy(buf, js.c_str(), js.size() + 1);
  return MOCHY_OK;
}

int64_t mochy_device_bytes(mochy_ctx* ctx) { return ctx ? ctx->held : 0; }

int64_t mochy_kernel_launches(void) { return (int64_t)g_launches.load(); }

const char* mochy_strerror(int code) {
  switch (code) {
    case MOCHY_OK: return "ok";
    case MOCHY_W_DEGENERATE_CP: return "all significances are zero; the CP is zero";
    case MOCHY_E_INVALID: return "invalid argument or hypergraph";
    case MOCHY_E_NOMEM: return "out of device memory or over the memory budget";
    case MOCHY_E_CUDA: return "CUDA error";
    case MOCHY_E_TIMEOUT: return "a bounded device wait ran out";
    case MOCHY_E_NOT_PROJECTED: return "the line graph is not built (call mochy_project)";
    case MOCHY_E_UNSUPPORTED: return "outside the supported limits";
    case MOCHY_E_BUSY: return "queue full";
  }
  return "unknown error";
}

const char* mochy_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"

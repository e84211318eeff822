// Sampled counting: MoCHy-A (Algorithm "sampling_ver1", hyperedge sampling)
// and MoCHy-A+ (Algorithm "sampling_ver2", hyperwedge sampling), Section 3.3.
//
// Both reduce to hyperwedge work items (e_i, e_j): A+ draws one hyperwedge
// per sample; A draws a hyperedge e_i and takes every hyperwedge (e_i, e_j)
// of it.  For a work item a warp merges the sorted rows of e_i and e_j tile by
// tile and classifies every e_k in N_i u N_j \ {e_i, e_j}:
//   A+ : every such e_k;
//   A  : e_k outside N_i, or e_k in N_i with j < k (the rule of
//        Algorithm sampling_ver1).
// Random draws: Philox4x32-10 (Salmon et al., SC'11) on counter
// (n_lo, n_hi, stream, 0) with key (seed_lo, seed_hi); the 64-bit output u
// selects floor(u * range / 2^64).
#include <mutex>

#include "classify.cuh"
#include "philox.cuh"

namespace mochy {

// index in [0, n) of lower_bound-style search: largest r with pre[r] <= x
__device__ __forceinline__ int64_t upper_index(const int64_t* __restrict__ pre, int64_t n,
                                               int64_t x) {
  int64_t lo = 0, hi = n;  // pre[0] <= x < pre[n]
  while (hi - lo > 1) {
    const int64_t m = (lo + hi) >> 1;
    if (pre[m] <= x) lo = m; else hi = m;
  }
  return lo;
}

namespace {

constexpr int kSampThreads = 256;
constexpr int kSampWarps = kSampThreads / 32;

struct SampleArgs {
  int64_t n_edges;
  int64_t n_wedges;
  const int64_t* eoff;
  const int32_t* enode;
  const int64_t* noff;
  const uint2* nadj;
  const int64_t* ustart;
  const int64_t* uprefix;
  const uint16_t* lut3;
  unsigned long long* hist;
  int theta;
  int method;
  uint64_t seed;
  int64_t samples;
  const int64_t* item_prefix;  // A: prefix of |N_i| over samples [samples + 1]
  const int64_t* sample_row;   // A: sampled row per sample
};

// rows drawn by MoCHy-A and their degrees
__global__ void k_draw_rows(SampleArgs g, int64_t* __restrict__ row, int64_t* __restrict__ deg) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.samples) return;
  const uint64_t u = philox_u64(g.seed, (uint64_t)n, 1u, 0u);
  const int64_t i = (int64_t)__umul64hi(u, (uint64_t)g.n_edges);
  row[n] = i;
  deg[n] = g.noff[i + 1] - g.noff[i];
}

// classify one candidate e_k of work item (i, j)
__device__ __forceinline__ int cand_code(int A, int B, int C, int x, int y, int z, uint32_t mij,
                                         uint32_t mik, bool closed, int64_t i, int64_t j,
                                         int64_t k, const SampleArgs& g,
                                         const int32_t* __restrict__ enode,
                                         const int64_t* __restrict__ eoff) {
  int t = 0;
  if (closed) {
    if (A <= kMaskedMax) {
      t = __popc(mij & mik);
    } else {
      t = sorted_overlap3(enode + eoff[i], A, enode + eoff[j], B, enode + eoff[k], C);
    }
  }
  return ternary_code(A, B, C, x, y, z, t, g.theta);
}

__global__ void __launch_bounds__(kSampThreads)
k_sample_wedges(SampleArgs g, int64_t n_items) {
  __shared__ unsigned long long hist[432];
  __shared__ uint16_t lut[2187];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < 432; q += kSampThreads) hist[q] = 0ull;
  for (int q = threadIdx.x; q < 2187; q += kSampThreads) lut[q] = g.lut3[q];
  __syncthreads();
  RunCache rc;
  const int64_t nwarps = (int64_t)gridDim.x * kSampWarps;
  for (int64_t it = (int64_t)blockIdx.x * kSampWarps + warp; it < n_items; it += nwarps) {
    int64_t i, pj;
    if (g.method == MOCHY_A_PLUS) {
      const uint64_t u = philox_u64(g.seed, (uint64_t)it, 2u, 0u);
      const int64_t w = (int64_t)__umul64hi(u, (uint64_t)g.n_wedges);
      i = upper_index(g.uprefix, g.n_edges, w);
      pj = g.ustart[i] + (w - g.uprefix[i]);
    } else {
      const int64_t n = upper_index(g.item_prefix, g.samples, it);
      i = g.sample_row[n];
      pj = g.noff[i] + (it - g.item_prefix[n]);
    }
    const uint2 eij = g.nadj[pj];
    const int64_t j = ent_id(eij);
    const int A = (int)(g.eoff[i + 1] - g.eoff[i]);
    const int B = ent_size(eij);
    const int x = entry_omega(eij.y, A);
    const uint32_t mij = eij.y;
    int64_t p1 = g.noff[i], e1 = g.noff[i + 1];
    int64_t p2 = g.noff[j], e2 = g.noff[j + 1];
    const uint32_t INF = 0xffffffffu;
    while (p1 < e1 || p2 < e2) {
      const uint2 t1 = p1 + lane < e1 ? g.nadj[p1 + lane] : make_uint2(INF, 0u);
      const uint2 t2 = p2 + lane < e2 ? g.nadj[p2 + lane] : make_uint2(INF, 0u);
      const uint32_t k1 = t1.x == INF ? INF : ent_id(t1);
      const uint32_t k2 = t2.x == INF ? INF : ent_id(t2);
      const uint32_t m1 = __shfl_sync(0xffffffffu, k1, 31);
      const uint32_t m2 = __shfl_sync(0xffffffffu, k2, 31);
      const uint32_t bound = min(m1, m2);
      // search own key in the other tile (keys ascending, INF padded)
      int lo = 0;
#pragma unroll
      for (int s = 16; s; s >>= 1) {
        const uint32_t probe = __shfl_sync(0xffffffffu, k2, lo + s - 1);
        if (probe < k1) lo += s;
      }
      const uint32_t at2 = __shfl_sync(0xffffffffu, k2, lo & 31);
      const uint32_t w2 = __shfl_sync(0xffffffffu, t2.y, lo & 31);
      const bool in2 = lo < 32 && at2 == k1 && k1 != INF;
      int lo2 = 0;
#pragma unroll
      for (int s = 16; s; s >>= 1) {
        const uint32_t probe = __shfl_sync(0xffffffffu, k1, lo2 + s - 1);
        if (probe < k2) lo2 += s;
      }
      const uint32_t at1 = __shfl_sync(0xffffffffu, k1, lo2 & 31);
      const bool in1 = lo2 < 32 && at1 == k2 && k2 != INF;
      // tile 1 elements (k in N_i): closed when also in N_j, else open centre i
      if (k1 <= bound && k1 != INF && (int64_t)k1 != j) {
        const int64_t k = k1;
        const bool keep = g.method == MOCHY_A_PLUS || k > j;
        if (keep) {
          const int C = ent_size(t1);
          const int z = entry_omega(t1.y, A);
          const int y = in2 ? entry_omega(w2, B) : 0;
          rc.add(lut[cand_code(A, B, C, x, y, z, mij, t1.y, in2, i, j, k, g, g.enode, g.eoff)],
                 hist);
        }
      }
      // tile 2 elements only in N_j: open centre j
      if (k2 <= bound && k2 != INF && (int64_t)k2 != i && !in1) {
        const int C = ent_size(t2);
        const int y = entry_omega(t2.y, B);
        rc.add(lut[ternary_code(A, B, C, x, y, 0, 0, g.theta)], hist);
      }
      p1 += __popc(__ballot_sync(0xffffffffu, k1 <= bound && k1 != INF));
      p2 += __popc(__ballot_sync(0xffffffffu, k2 <= bound && k2 != INF));
    }
  }
  rc.flush(hist);
  __syncthreads();
  for (int q = threadIdx.x; q < 432; q += kSampThreads)
    if (hist[q]) atomicAdd(&g.hist[q], hist[q]);
}

}  // namespace

int count_sampled(mochy_ctx* ctx, int method, int64_t samples, uint64_t seed,
                  unsigned long long* d_hist) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  if (method != MOCHY_A && method != MOCHY_A_PLUS) return fail(MOCHY_E_INVALID, "bad method");
  if (samples <= 0) return fail(MOCHY_E_INVALID, "samples must be positive");
  cudaStream_t st = ctx->stream;
  MOCHY_CUDA(cudaMemsetAsync(d_hist, 0, 432 * 8, st));
  SampleArgs g;
  g.n_edges = ctx->n_edges;
  g.n_wedges = ctx->n_wedges;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.ustart = ctx->ustart;
  g.uprefix = ctx->uprefix;
  g.lut3 = ctx->tables.lut3;
  g.hist = d_hist;
  g.theta = ctx->theta;
  g.method = method;
  g.seed = seed;
  g.samples = samples;
  g.item_prefix = nullptr;
  g.sample_row = nullptr;
  int64_t n_items = samples;
  if (method == MOCHY_A_PLUS) {
    if (ctx->n_wedges == 0) return fail(MOCHY_E_INVALID, "the hypergraph has no hyperwedge");
  } else {
    if (ctx->n_edges == 0) return fail(MOCHY_E_INVALID, "the hypergraph has no hyperedge");
    void* t;
    MOCHY_TRY(scratch(ctx, 0, (size_t)(samples + 1) * 8 * 3, &t));
    int64_t* row = (int64_t*)t;
    int64_t* deg = row + (samples + 1);
    int64_t* pre = deg + (samples + 1);
    MOCHY_CUDA(cudaMemsetAsync(deg, 0, (size_t)(samples + 1) * 8, st));
    k_draw_rows<<<ceil_div(samples, 256), 256, 0, st>>>(g, row, deg);
    MOCHY_LAUNCHED();
    MOCHY_TRY(scan_exclusive_i64(ctx, deg, pre, samples + 1));
    MOCHY_CUDA(cudaMemcpyAsync(&n_items, pre + samples, 8, cudaMemcpyDeviceToHost, st));
    MOCHY_CUDA(cudaStreamSynchronize(st));
    g.item_prefix = pre;
    g.sample_row = row;
  }
  if (n_items == 0) return MOCHY_OK;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n_items, kSampWarps),
                                                    (int64_t)ctx->num_sms * 8);
  k_sample_wedges<<<grid, kSampThreads, 0, st>>>(g, n_items);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

// ---------------------------------------------------------------------------
// Sampled counting without any device allocation.
//
// For callers that cannot allocate device memory while they run: a process
// whose memory is handed out by another runtime or pool, a serving loop with
// a fixed memory reservation, code that must not grow the context's footprint
// between calls.  The working memory of this path (the motif histogram, the
// drawn rows of MoCHy-A and their prefix sums) lives in one file-scope
// __device__ array of kNoAllocBytes bytes, which every GPU that loads the
// library holds until the process exits.  The first call on a device looks
// up the array's device address (cudaGetSymbolAddress, with that device
// current); that call should come before any stream capture.  All calls
// share the array: each call clears what must start at zero, and calls whose
// work overlaps on the GPU race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxSamplesA = 65536;   // MoCHy-A draws per call
constexpr size_t kNoAllocHist = 432 * 8;
constexpr size_t kNoAllocBytes = kNoAllocHist + 256 + 3 * (kNoAllocMaxSamplesA + 1) * 8;

__global__ void __launch_bounds__(1024) k_noalloc_scan(const int64_t* __restrict__ in,
                                                       int64_t* __restrict__ out, int64_t n) {
  // exclusive scan of n values by one block, tile by tile
  __shared__ int64_t ws[34];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < n ? in[i] : 0;
    int64_t total;
    const int64_t ex = block_scan_i64(v, ws, &total);
    const int64_t c = carry;
    if (i < n) out[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) k_noalloc_finish(
    const unsigned long long* __restrict__ hist, const uint8_t* __restrict__ t2h,
    const uint8_t* __restrict__ hopen, int method, double numer, double samples,
    int64_t* __restrict__ raw_h, int64_t* __restrict__ raw_3h, double* __restrict__ est_h,
    double* __restrict__ est_3h) {
  __shared__ unsigned long long h[27];
  if (threadIdx.x < 27) h[threadIdx.x] = 0ull;
  __syncthreads();
  for (int t = threadIdx.x + 1; t <= MOCHY_N_3H; t += blockDim.x) {
    raw_3h[t - 1] = (int64_t)hist[t];
    const double w = method == MOCHY_A ? 3.0 : (hopen[t2h[t]] ? 2.0 : 3.0);
    est_3h[t - 1] = __ddiv_rn(__dmul_rn((double)hist[t], numer), __dmul_rn(w, samples));
    atomicAdd(&h[t2h[t]], hist[t]);
  }
  __syncthreads();
  if (threadIdx.x < MOCHY_N_H) {
    const int id = threadIdx.x + 1;
    raw_h[threadIdx.x] = (int64_t)h[id];
    const double w = method == MOCHY_A ? 3.0 : (hopen[id] ? 2.0 : 3.0);
    est_h[threadIdx.x] = __ddiv_rn(__dmul_rn((double)h[id], numer), __dmul_rn(w, samples));
  }
}

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch on the current device, looked up once
// per device and kept for the life of the process.  A device reset
// (cudaDeviceReset) or a new primary context invalidates the kept address;
// callers that reset a device must not use this entry point afterwards.
static int noalloc_scratch(int device, unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[256] = {nullptr};
  if (device < 0 || device >= 256) return fail(MOCHY_E_INVALID, "bad device ordinal");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    addr[device] = (unsigned char*)p;
  }
  *out = addr[device];
  return MOCHY_OK;
}

}  // namespace mochy

extern "C" int mochy_count_sampled_noalloc(mochy_ctx* ctx, int method, int64_t samples,
                                           uint64_t seed, int64_t* d_raw_h, int64_t* d_raw_3h,
                                           double* d_est_h, double* d_est_3h) {
  using namespace mochy;
  if (!ctx) return fail(MOCHY_E_INVALID, "null context");
  if (!d_raw_h || !d_raw_3h || !d_est_h || !d_est_3h) return fail(MOCHY_E_INVALID, "null output");
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  if (method != MOCHY_A && method != MOCHY_A_PLUS) return fail(MOCHY_E_INVALID, "bad method");
  if (samples <= 0) return fail(MOCHY_E_INVALID, "samples must be positive");
  if (method == MOCHY_A && samples > kNoAllocMaxSamplesA)
    return fail(MOCHY_E_UNSUPPORTED, "the allocation-free MoCHy-A takes at most 65536 samples "
                                     "per call (its fixed working memory)");
  if (method == MOCHY_A_PLUS && ctx->n_wedges == 0)
    return fail(MOCHY_E_INVALID, "the hypergraph has no hyperwedge");
  if (method == MOCHY_A && ctx->n_edges == 0)
    return fail(MOCHY_E_INVALID, "the hypergraph has no hyperedge");
  MOCHY_CUDA(cudaSetDevice(ctx->device));
  unsigned char* base = nullptr;
  MOCHY_TRY(noalloc_scratch(ctx->device, &base));
  cudaStream_t st = ctx->stream;
  unsigned long long* hist = (unsigned long long*)base;
  int64_t* row = (int64_t*)(base + kNoAllocHist + 256);
  int64_t* deg = row + (kNoAllocMaxSamplesA + 1);
  int64_t* pre = deg + (kNoAllocMaxSamplesA + 1);
  MOCHY_CUDA(cudaMemsetAsync(hist, 0, kNoAllocHist, st));
  SampleArgs g;
  g.n_edges = ctx->n_edges;
  g.n_wedges = ctx->n_wedges;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.ustart = ctx->ustart;
  g.uprefix = ctx->uprefix;
  g.lut3 = ctx->tables.lut3;
  g.hist = hist;
  g.theta = ctx->theta;
  g.method = method;
  g.seed = seed;
  g.samples = samples;
  g.item_prefix = nullptr;
  g.sample_row = nullptr;
  int64_t n_items = samples;
  if (method == MOCHY_A) {
    MOCHY_CUDA(cudaMemsetAsync(deg, 0, (size_t)(samples + 1) * 8, st));
    k_draw_rows<<<ceil_div(samples, 256), 256, 0, st>>>(g, row, deg);
    MOCHY_LAUNCHED();
    k_noalloc_scan<<<1, 1024, 0, st>>>(deg, pre, samples + 1);
    MOCHY_LAUNCHED();
    MOCHY_CUDA(cudaMemcpyAsync(&n_items, pre + samples, 8, cudaMemcpyDeviceToHost, st));
    MOCHY_CUDA(cudaStreamSynchronize(st));
    g.item_prefix = pre;
    g.sample_row = row;
  }
  if (n_items > 0) {
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n_items, kSampWarps),
                                                      (int64_t)ctx->num_sms * 8);
    k_sample_wedges<<<grid, kSampThreads, 0, st>>>(g, n_items);
    MOCHY_LAUNCHED();
  }
  const double numer = method == MOCHY_A ? (double)ctx->n_edges : (double)ctx->n_wedges;
  k_noalloc_finish<<<1, 512, 0, st>>>(hist, ctx->tables.t2h, ctx->tables.hopen, method, numer,
                                      (double)samples, d_raw_h, d_raw_3h, d_est_h, d_est_3h);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

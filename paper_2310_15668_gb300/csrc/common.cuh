// Internal declarations shared by the libmochy CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/mochy.h"

namespace mochy {

// ---------------------------------------------------------------------------
// Error handling: every CUDA call is checked; the first failure is recorded
// in a thread-local message and turned into a MOCHY_E_* return code.
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define MOCHY_CUDA(call)                                                    \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) return ::mochy::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define MOCHY_TRY(call)          \
  do {                           \
    int rc_ = (call);            \
    if (rc_ < 0) return rc_;     \
  } while (0)

// Kernel launch bookkeeping (the count is exported for accounting).
void note_launch(int n = 1);
#define MOCHY_LAUNCHED() \
  do { ::mochy::note_launch(); MOCHY_CUDA(cudaGetLastError()); } while (0)

// ---------------------------------------------------------------------------
// Line-graph entry layout (8 bytes, rows sorted by neighbour id):
//   w0 bits  0..25  neighbour hyperedge id k
//   w0 bits 26..31  |e_k| (1..63)
//   w1              for a row e_i with |e_i| <= 32: bit p set when the p-th
//                   node of e_i (ascending) lies in e_k, so omega = popc(w1);
//                   for |e_i| > 32: omega itself.
// ---------------------------------------------------------------------------
constexpr uint32_t kIdBits = 26;
constexpr uint32_t kIdMask = (1u << kIdBits) - 1u;
constexpr int kMaskedMax = 32;

// Widest window of dense words the dense-triangle kernel accepts: each lane
// counts its share of a hyperwedge's candidates (at most 32 per word, one
// word in 32 of the window) into 16-bit halves of its bins, which stay below
// 65,536 while the window has at most 65,504 words.
constexpr int64_t kMaxWindowWords = 65504;

__host__ __device__ inline uint32_t ent_id(uint2 e) { return e.x & kIdMask; }
__host__ __device__ inline int ent_size(uint2 e) { return (int)(e.x >> kIdBits); }

// Motif tables on the device.
struct Tables {
  uint16_t* lut3 = nullptr;   // [2187] ternary region code -> 3h id (0 invalid)
  uint8_t* t2h = nullptr;     // [432] 3h id -> h id
  uint8_t* hopen = nullptr;   // [27]  h id -> 1 if open
};

// One hypergraph ("unit") of a batch counted as a disjoint union: where its
// dense rows and heavy nodes sit in the split structures.  Its dense rows are
// the dense indices [dbase, dbase + n); their bitmaps cover only the unit's
// window of words [wlo, wlo + wn) and start at word dboff of dbits (4 wn words
// a row); its heavy nodes are the heavy indices from hbase on, with bitmaps
// of wn words from word nboff of nbits.  A lone hypergraph is one unit with
// wlo = 0 and wn = the number of dense words.
struct SegInfo {
  int64_t dbase, dboff, hbase, nboff, wlo, wn;
};

// Scratch arena: grows on demand, freed with the context.
struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace mochy

struct mochy_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int32_t theta = 1;
  double eps = 1.0;
  int64_t budget = 0;
  int64_t held = 0;          // bytes currently allocated by this context
  int num_sms = 0;
  size_t smem_optin = 0;

  mochy::Tables tables;

  // hypergraph (after duplicate removal)
  int64_t n_nodes = 0, n_edges = 0, n_inc = 0;
  int64_t* eoff = nullptr;     // [E+1]
  int32_t* enode = nullptr;    // [n_inc] node lists, ascending per hyperedge
  uint8_t* esize = nullptr;    // [E]
  int64_t* voff = nullptr;     // [N+1]
  int32_t* vedge = nullptr;    // [n_inc] incidence lists E_v, ascending
  int max_size = 0;

  // line graph
  bool projected = false;
  int64_t n_wedges = 0;
  int32_t max_deg = 0;
  int64_t* noff = nullptr;     // [E+1]
  uint2* nadj = nullptr;       // [2 |wedges|]
  int64_t* ustart = nullptr;   // [E]   first entry of row i with k > i
  int64_t* uprefix = nullptr;  // [E+1] exclusive prefix of upper-row lengths
  int32_t* row_order = nullptr;  // [E] rows by decreasing estimated work

  // exact count, split path (built on first use, released with the line graph):
  // rows of line degree >= dense_thr are "dense" and get bitmaps over the
  // dense-row index space; nodes with >= heavy_thr dense hyperedges get one too.
  int exact_kernel = 0;          // 0 split (default), 1 wedge-scan
  int32_t dense_thr = 0;         // 0 = chosen by the tuner
  int32_t rest_path = 0;         // dense candidates outside the bins: 0 auto, 1 per lane, 2 spread
  int32_t heavy_thr = 32;
  bool split_ready = false;
  int64_t n_dense = 0, n_sparse = 0, n_heavy = 0, wwords = 0;
  int32_t* dense_idx = nullptr;   // [E]  dense index or -1
  int32_t* dense_row = nullptr;   // [n_dense]
  uint32_t* dbits = nullptr;      // per dense row, per word of its window, 4 words: bits 0..2
                                  // of min(omega, 7) and the mask of omega >= 1
  int32_t* heavy_idx = nullptr;   // [N]  heavy index or -1
  uint32_t* nbits = nullptr;      // [n_heavy][wwords]  dense members of E_v
  uint32_t* sbits = nullptr;      // per word 4 words (bits 0..3 of min(|e_k|, 15)),
                                  // then [5][wwords] size classes of dense rows
  int32_t* dense_order = nullptr;   // dense rows by decreasing work
  int32_t* sparse_order = nullptr;  // sparse rows by decreasing work
  int64_t* dvoff = nullptr;         // [N+1] dense members of E_v ...
  int32_t* dvedge = nullptr;        // ... as dense indices, ascending
  uint8_t* dsize = nullptr;         // [n_dense] |e_k| of dense rows
  void* rest_block = nullptr;       // dbits .. dsize in one allocation
  size_t split_bytes = 0, rest_bytes = 0, nbits_bytes = 0, dinc_bytes = 0;
  int32_t dense_thr_used = 0;

  // disjoint union of n_units hypergraphs counted together (a batch): unit u
  // owns the nodes [nseg[u], nseg[u+1]) and the hyperedges [eseg[u],
  // eseg[u+1]); an exact count then fills one histogram per unit.  A lone
  // hypergraph is one unit and keeps no arrays.
  int32_t n_units = 1;
  int64_t* d_nseg = nullptr;           // [n_units+1] on the device (then eseg)
  size_t nseg_bytes = 0;
  std::vector<int64_t> h_nseg, h_eseg; // [n_units+1] on the host
  mochy::SegInfo* d_seg = nullptr;     // [n_units] (split structures)
  int64_t* d_dbase = nullptr;          // [n_units+1] first dense index per unit
  int64_t wmax = 0;                    // widest unit window, words

  // MoCHy-A+ without the line graph (built on first use after a load):
  // membership bitmaps of the most popular nodes, size planes, and the
  // prefix of the number of neighbours after each hyperedge
  bool otf_ready = false;
  void* otf_block = nullptr;
  size_t otf_bytes = 0;
  int32_t* otf_hidx = nullptr;     // [N] bitmap index or -1
  uint32_t* otf_hbits = nullptr;   // [otf_bitmaps][otf_words]
  uint32_t* otf_sbits = nullptr;   // per word 4 words: bits 0..3 of min(|e_k|, 15)
  int64_t* otf_uprefix = nullptr;  // [E+1]
  int64_t otf_wedges = 0, otf_bitmaps = 0, otf_words = 0;

  // kh-motif tables (built on first use): lut over k^7 codes, parent h id
  // and pattern (7 states) of each id
  int kh_k = 0, kh_n = 0;
  void* kh_block = nullptr;
  size_t kh_bytes = 0;
  uint16_t* kh_lut = nullptr;
  uint8_t* kh_to_h = nullptr;
  uint8_t* kh_pattern = nullptr;

  // per-call device scratch
  unsigned long long* hist = nullptr;  // [432] 3h histogram (index = id)
  int32_t* counters = nullptr;         // [16] work-queue counters / flags
  mochy::Buffer scratch[4];

  // pinned host staging
  void* pinned = nullptr;

  // tracing: per-phase durations of the last traced call (CUDA events on the
  // context's stream) and kernel statistics
  int trace = 0;                       // 0 off, 1 phase events, 2 + kernel statistics
  int n_phases = 0;
  char phase_name[8][24];
  double phase_ms[8];
  unsigned long long* stats = nullptr;   // [8] device counters, when tracing
  unsigned long long last_stats[24];
};

namespace mochy {

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (never
// lowers it; safe with several host threads).
int ensure_dynamic_smem(const void* func, size_t bytes);

// Memory (budget-checked, tracked per context).
int dev_alloc(mochy_ctx* ctx, void** p, size_t bytes);
void dev_free(mochy_ctx* ctx, void* p, size_t bytes);
int scratch(mochy_ctx* ctx, int slot, size_t bytes, void** p);
void release_graph(mochy_ctx* ctx);
void release_projection(mochy_ctx* ctx);

// Primitives (primitives.cu).
int scan_exclusive_i64(mochy_ctx* ctx, const int64_t* d_in, int64_t* d_out, int64_t n);
int radix_sort_pairs_u32(mochy_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n,
                         int key_bits);

// Stages.
int build_tables(mochy_ctx* ctx);                                     // tables.cu
int build_kh_tables(mochy_ctx* ctx, int k);                           // tables.cu
int load_graph(mochy_ctx* ctx, int64_t n_nodes, int64_t n_edges,
               const int64_t* d_off, const int32_t* d_nodes, int64_t* n_dup);  // load.cu
int project_graph(mochy_ctx* ctx);                                    // project.cu
int count_exact(mochy_ctx* ctx, const int32_t* d_anchors, int64_t n_anchors,
                unsigned long long* d_hist);                          // count_exact.cu
int count_exact_split(mochy_ctx* ctx, unsigned long long* d_hist);    // count_split.cu
int count_split_rows(mochy_ctx* ctx, const int32_t* d_rows, int64_t n_rows,
                     unsigned long long* d_hist);                     // count_split.cu
int hyperedge_profiles(mochy_ctx* ctx, unsigned long long* d_hp);    // count_exact.cu
int star_node_profiles(mochy_ctx* ctx, unsigned long long* d_np);    // count_exact.cu
int radial_node_profiles(mochy_ctx* ctx, unsigned long long* d_np);  // extensions.cu
int count_kh(mochy_ctx* ctx, int k, int thr1, int thr2, unsigned long long* d_hist);  // extensions.cu
int count_sampled_onthefly(mochy_ctx* ctx, int64_t samples, uint64_t seed, int64_t budget,
                           unsigned long long* d_hist, unsigned long long* d_stats);  // onthefly.cu
void release_onthefly(mochy_ctx* ctx);                                // onthefly.cu
int enumerate_instances(mochy_ctx* ctx, int64_t cap, int32_t* d_out,
                        unsigned long long* d_cursor);                // extensions.cu
int prepare_split(mochy_ctx* ctx);                                    // count_split.cu
int choose_dense_threshold(mochy_ctx* ctx);                           // tune.cu
int tune_dense_threshold(mochy_ctx* ctx, const int32_t* cand, int32_t n_cand, double fraction,
                         uint64_t seed, int32_t* best, int32_t* tried,
                         double* ms);                                 // tune.cu
void release_split(mochy_ctx* ctx);                                   // count_split.cu
int count_sampled(mochy_ctx* ctx, int method, int64_t samples, uint64_t seed,
                  unsigned long long* d_hist);                        // sample.cu
int randomize_graph(mochy_ctx* src, uint64_t seed, uint32_t copy, mochy_ctx* dst);  // nullmodel.cu
int pairs_to_hypergraph(mochy_ctx* work, uint32_t* node, uint32_t* edge, int64_t n_pairs,
                        int64_t n_nodes, int64_t n_edges, mochy_ctx* dst);  // nullmodel.cu
int bits_for(int64_t n);                                              // primitives.cu
int count_split_graph(mochy_ctx* ctx, unsigned long long* d_hist, float* ms);  // count_split.cu
int finish_counts(mochy_ctx* ctx, const unsigned long long* d_hist, int64_t* d_out_h,
                  int64_t* d_out_3h);                                 // profile.cu
int scale_estimates(mochy_ctx* ctx, const int64_t* d_raw_h, const int64_t* d_raw_3h,
                    int method, double numer, int64_t samples, double* d_est_h,
                    double* d_est_3h);                                // profile.cu
int significance_cp(mochy_ctx* ctx, const int64_t* d_counts_h, const int64_t* d_counts_3h,
                    int32_t n_random, double eps, double* d_out /* 4 vectors */,
                    int32_t* d_degenerate);                           // profile.cu

int finish_counts_batch(mochy_ctx* ctx, const unsigned long long* d_hist, int n_hist,
                        int64_t* d_out_h, int64_t* d_out_3h, int32_t* d_bad);  // profile.cu
int significance_cp_batch(mochy_ctx* ctx, const int64_t* d_counts_h, const int64_t* d_counts_3h,
                          int n_graphs, int32_t n_random, double eps, double* d_out,
                          int32_t* d_degenerate);                     // profile.cu

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// largest u in [0, n) with b[u] <= x, for ascending b with b[0] <= x (with
// equal bounds the later, non-empty range wins)
__host__ __device__ __forceinline__ int seg_of(const int64_t* b, int n, int64_t x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (b[m] <= x) lo = m; else hi = m;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Small device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t warp_incl_scan_i64(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// Exclusive scan across the block of one value per thread; `ws` is shared
// scratch of 34 int64.  Ends with a barrier, so `ws` can be reused at once.
__device__ __forceinline__ int64_t block_scan_i64(int64_t v, int64_t* ws, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t inc = warp_incl_scan_i64(v);
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
    const int64_t s = lane < nw ? ws[lane] : 0;
    const int64_t si = warp_incl_scan_i64(s);
    __syncwarp();
    ws[lane] = si - s;
    if (lane == 31) ws[32] = si;
  }
  __syncthreads();
  const int64_t res = ws[warp] + inc - v;
  *total = ws[32];
  __syncthreads();
  return res;
}

}  // namespace mochy

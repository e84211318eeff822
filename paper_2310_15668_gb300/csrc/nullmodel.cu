// Randomized hypergraphs of the paper's null model (Section 3.1 "Randomized
// Hypergraphs"; Appendix "Randomized Hypergraphs").
//
// Chung-Lu on the incidence graph (Algorithm "randomized_hypergraph_alg"):
// |E'| = sum |e| draws of a (node, hyperedge) pair, the node with probability
// d_v / |E'| and the hyperedge with probability |e_j| / |E'|.  Draw d of copy
// c takes two Philox4x32-10 outputs (streams 3 and 4, counter (d, stream, c))
// and maps each 64-bit u to x = floor(u |E'| / 2^64); the node is the v with
// voff[v] <= x < voff[v+1] (voff is the degree prefix) and the hyperedge the j
// with eoff[j] <= x < eoff[j+1].
//
// Transform (Algorithm "transform"): the nodes drawn for e_j form a set;
// empty sets are dropped; repeated hyperedges are dropped keeping the first
// (E is a set, Section 2.1), which the loader does.
#include "classify.cuh"
#include "philox.cuh"

namespace mochy {

namespace {

__device__ __forceinline__ int64_t owner(const int64_t* __restrict__ pre, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int64_t m = (lo + hi) >> 1;
    if (pre[m] <= x) lo = m; else hi = m;
  }
  return lo;
}

__global__ void k_chung_lu(int64_t total, const int64_t* __restrict__ voff, int64_t n_nodes,
                           const int64_t* __restrict__ eoff, int64_t n_edges, uint64_t seed,
                           uint32_t copy, uint32_t* __restrict__ node, uint32_t* __restrict__ edge) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= total) return;
  const uint64_t ua = philox_u64(seed, (uint64_t)d, 3u, copy);
  const uint64_t ub = philox_u64(seed, (uint64_t)d, 4u, copy);
  const int64_t xv = (int64_t)__umul64hi(ua, (uint64_t)total);
  const int64_t xe = (int64_t)__umul64hi(ub, (uint64_t)total);
  node[d] = (uint32_t)owner(voff, n_nodes, xv);
  edge[d] = (uint32_t)owner(eoff, n_edges, xe);
}

// after sorting by (edge, node): first occurrences, and per-edge set sizes
__global__ void k_firsts(int64_t total, const uint32_t* __restrict__ edge,
                         const uint32_t* __restrict__ node, int64_t* __restrict__ first,
                         int64_t* __restrict__ size) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= total) return;
  const bool f = d == 0 || edge[d] != edge[d - 1] || node[d] != node[d - 1];
  first[d] = f ? 1 : 0;
  if (f) atomicAdd((unsigned long long*)&size[edge[d]], 1ull);
}

__global__ void k_gather_nodes(int64_t total, const uint32_t* __restrict__ node,
                               const int64_t* __restrict__ first, const int64_t* __restrict__ pos,
                               int32_t* __restrict__ out) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= total || !first[d]) return;
  out[pos[d]] = (int32_t)node[d];
}

__global__ void k_nonempty(int64_t n_edges, const int64_t* __restrict__ size,
                           int64_t* __restrict__ flag) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_edges) return;
  flag[j] = size[j] > 0 ? 1 : 0;
}

__global__ void k_offsets(int64_t n_edges, const int64_t* __restrict__ size,
                          const int64_t* __restrict__ start, const int64_t* __restrict__ rank,
                          int64_t* __restrict__ off) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_edges || size[j] == 0) return;
  off[rank[j]] = start[j];
}

}  // namespace

// The transform of Algorithm "transform" on (node, hyperedge) pairs: every
// hyperedge becomes the set of its nodes, empty hyperedges are dropped, and
// the result is loaded into dst (which drops repeated hyperedges).  The pairs
// are sorted in place; temporaries come from work's scratch.
int pairs_to_hypergraph(mochy_ctx* work, uint32_t* node, uint32_t* edge, int64_t T, int64_t N,
                        int64_t E, mochy_ctx* dst) {
  cudaStream_t st = work->stream;
  const size_t need = (size_t)T * 20 + (size_t)(E + 1) * 40 + 16 * 256;
  void* base;
  MOCHY_TRY(scratch(work, 0, need, &base));
  char* cur = (char*)base;
  auto carve = [&](size_t b) { void* r = cur; cur += (b + 255) & ~(size_t)255; return r; };
  int64_t* first = (int64_t*)carve((size_t)T * 8);
  int64_t* pos = (int64_t*)carve((size_t)T * 8 + 8);
  int64_t* size = (int64_t*)carve((size_t)(E + 1) * 8);
  int64_t* flag = (int64_t*)carve((size_t)(E + 1) * 8);
  int64_t* rank = (int64_t*)carve((size_t)(E + 1) * 8);
  int64_t* start = (int64_t*)carve((size_t)(E + 1) * 8);
  int32_t* nodes_out = (int32_t*)carve((size_t)T * 4);
  const int B = 256;
  // sort by (edge, node): stable by node, then stable by edge
  MOCHY_TRY(radix_sort_pairs_u32(work, node, edge, T, bits_for(N)));
  MOCHY_TRY(radix_sort_pairs_u32(work, edge, node, T, bits_for(E)));
  MOCHY_CUDA(cudaMemsetAsync(size, 0, (size_t)(E + 1) * 8, st));
  k_firsts<<<ceil_div(T, B), B, 0, st>>>(T, edge, node, first, size);
  MOCHY_LAUNCHED();
  MOCHY_TRY(scan_exclusive_i64(work, first, pos, T));
  k_gather_nodes<<<ceil_div(T, B), B, 0, st>>>(T, node, first, pos, nodes_out);
  MOCHY_LAUNCHED();
  // offsets of the non-empty hyperedges, in hyperedge order
  MOCHY_TRY(scan_exclusive_i64(work, size, start, E + 1));
  k_nonempty<<<ceil_div(E + 1, B), B, 0, st>>>(E, size, flag);
  MOCHY_LAUNCHED();
  MOCHY_CUDA(cudaMemsetAsync(flag + E, 0, 8, st));
  MOCHY_TRY(scan_exclusive_i64(work, flag, rank, E + 1));
  int64_t kept = 0, n_out = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&kept, rank + E, 8, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaMemcpyAsync(&n_out, start + E, 8, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  int64_t* off_out = (int64_t*)carve((size_t)(kept + 1) * 8);
  k_offsets<<<ceil_div(E, B), B, 0, st>>>(E, size, start, rank, off_out);
  MOCHY_LAUNCHED();
  MOCHY_CUDA(cudaMemcpyAsync(off_out + kept, &n_out, 8, cudaMemcpyHostToDevice, st));
  // hand the arrays to the destination context's loader (which copies them)
  MOCHY_CUDA(cudaStreamSynchronize(st));
  return load_graph(dst, N, kept, off_out, nodes_out, nullptr);
}

int randomize_graph(mochy_ctx* src, uint64_t seed, uint32_t copy, mochy_ctx* dst) {
  const int64_t T = src->n_inc, E = src->n_edges, N = src->n_nodes;
  cudaStream_t st = src->stream;
  if (T == 0) {
    return load_graph(dst, N, 0, nullptr, nullptr, nullptr);
  }
  // the draws live in scratch slot 2 (the transform takes slots 0, 1 and 3)
  void* base;
  MOCHY_TRY(scratch(src, 2, (size_t)T * 8 + 512, &base));
  uint32_t* node = (uint32_t*)base;
  uint32_t* edge = node + ((T + 63) & ~(int64_t)63);
  const int B = 256;
  k_chung_lu<<<ceil_div(T, B), B, 0, st>>>(T, src->voff, N, src->eoff, E, seed, copy, node, edge);
  MOCHY_LAUNCHED();
  return pairs_to_hypergraph(src, node, edge, T, N, E, dst);
}

}  // namespace mochy

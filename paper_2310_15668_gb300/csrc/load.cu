// Loading a hypergraph G = (V, E) (Section 2.1): validation, sorted node
// lists, removal of repeated hyperedges (E is a set; the first occurrence is
// kept), and the incidence lists E_v sorted by hyperedge id.
#include "common.cuh"

namespace mochy {
namespace {

enum : int { kErrEmpty = 1, kErrRange = 2, kErrRepeat = 4, kErrTooBig = 8, kErrOffsets = 16 };

__global__ void k_validate_sort(const int64_t* __restrict__ off, const int32_t* __restrict__ nodes,
                                int64_t n_edges, int64_t n_nodes, int32_t* __restrict__ sorted,
                                int32_t* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_edges) return;
  const int64_t b = off[i], e = off[i + 1];
  if (i == 0 && b != 0) atomicOr(err, kErrOffsets);
  const int64_t s = e - b;
  if (s <= 0) { atomicOr(err, s == 0 ? kErrEmpty : kErrOffsets); return; }
  if (s > MOCHY_MAX_EDGE_SIZE) { atomicOr(err, kErrTooBig); return; }
  int32_t v[MOCHY_MAX_EDGE_SIZE];
  for (int q = 0; q < (int)s; ++q) {
    const int32_t x = nodes[b + q];
    if (x < 0 || (int64_t)x >= n_nodes) { atomicOr(err, kErrRange); return; }
    int p = q;
    while (p > 0 && v[p - 1] > x) { v[p] = v[p - 1]; --p; }
    v[p] = x;
  }
  for (int q = 1; q < (int)s; ++q)
    if (v[q] == v[q - 1]) { atomicOr(err, kErrRepeat); return; }
  for (int q = 0; q < (int)s; ++q) sorted[b + q] = v[q];
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 33; z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33; z *= 0xc4ceb9fe1a85ec53ull;
  return z ^ (z >> 33);
}

__device__ uint64_t edge_hash(const int32_t* nodes, int64_t b, int64_t e) {
  uint64_t h = 0x9e3779b97f4a7c15ull ^ (uint64_t)(e - b);
  for (int64_t q = b; q < e; ++q) h = mix64(h ^ (uint64_t)(uint32_t)nodes[q]) + 0x632be59bd9b4e019ull;
  return h;
}

__device__ bool same_edge(const int64_t* off, const int32_t* nodes, int64_t x, int64_t y) {
  const int64_t bx = off[x], ex = off[x + 1], by = off[y], ey = off[y + 1];
  if (ex - bx != ey - by) return false;
  for (int64_t q = 0; q < ex - bx; ++q)
    if (nodes[bx + q] != nodes[by + q]) return false;
  return true;
}

// Open-addressing table keyed by hyperedge content; each group of equal
// hyperedges ends with the smallest member id in its slot.
__global__ void k_dedupe_insert(const int64_t* __restrict__ off, const int32_t* __restrict__ nodes,
                                int64_t n_edges, int32_t* __restrict__ table, uint64_t mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_edges) return;
  uint64_t slot = edge_hash(nodes, off[i], off[i + 1]) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    int32_t cur = table[slot];
    if (cur < 0) {
      cur = atomicCAS(&table[slot], -1, (int32_t)i);
      if (cur < 0) return;
    }
    if (same_edge(off, nodes, cur, i)) {
      atomicMin(&table[slot], (int32_t)i);
      return;
    }
    slot = (slot + 1) & mask;
  }
}

__global__ void k_dedupe_mark(const int64_t* __restrict__ off, const int32_t* __restrict__ nodes,
                              int64_t n_edges, const int32_t* __restrict__ table, uint64_t mask,
                              int64_t* __restrict__ keep) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_edges) return;
  uint64_t slot = edge_hash(nodes, off[i], off[i + 1]) & mask;
  int64_t k = 0;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const int32_t cur = table[slot];
    if (cur < 0) break;
    if (same_edge(off, nodes, cur, i)) { k = cur == (int32_t)i ? 1 : 0; break; }
    slot = (slot + 1) & mask;
  }
  keep[i] = k;
}

__global__ void k_kept_sizes(const int64_t* __restrict__ off, const int64_t* __restrict__ keep,
                             int64_t n_edges, int64_t* __restrict__ size_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_edges) return;
  size_out[i] = keep[i] ? off[i + 1] - off[i] : 0;
}

__global__ void k_compact(const int64_t* __restrict__ off, const int32_t* __restrict__ sorted,
                          const int64_t* __restrict__ keep, const int64_t* __restrict__ newid,
                          const int64_t* __restrict__ newpos, int64_t n_edges,
                          int64_t* __restrict__ eoff, int32_t* __restrict__ enode,
                          uint8_t* __restrict__ esize, int32_t* __restrict__ maxsize) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_edges || !keep[i]) return;
  const int64_t j = newid[i], b = off[i], s = off[i + 1] - b, p = newpos[i];
  eoff[j] = p;
  esize[j] = (uint8_t)s;
  for (int64_t q = 0; q < s; ++q) enode[p + q] = sorted[b + q];
  atomicMax(maxsize, (int32_t)s);
}

__global__ void k_incidence_pairs(const int64_t* __restrict__ eoff, const int32_t* __restrict__ enode,
                                  int64_t n_edges, uint32_t* __restrict__ key,
                                  uint32_t* __restrict__ val, unsigned long long* __restrict__ deg) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_edges) return;
  for (int64_t p = eoff[j]; p < eoff[j + 1]; ++p) {
    key[p] = (uint32_t)enode[p];
    val[p] = (uint32_t)j;
    atomicAdd(&deg[enode[p]], 1ull);
  }
}

__global__ void k_set_last(int64_t* a, int64_t idx, int64_t v) { a[idx] = v; }

}  // namespace

int load_graph(mochy_ctx* ctx, int64_t n_nodes, int64_t n_edges, const int64_t* d_off,
               const int32_t* d_nodes, int64_t* n_dup) {
  if (n_edges < 0 || n_nodes < 0) return fail(MOCHY_E_INVALID, "negative size");
  if (n_edges > MOCHY_MAX_EDGES) return fail(MOCHY_E_UNSUPPORTED, "too many hyperedges");
  if (n_nodes > 0x7fffffffLL) return fail(MOCHY_E_UNSUPPORTED, "too many nodes");
  release_graph(ctx);
  cudaStream_t st = ctx->stream;
  int64_t total = 0;
  if (n_edges > 0) {
    MOCHY_CUDA(cudaMemcpyAsync(&total, d_off + n_edges, 8, cudaMemcpyDeviceToHost, st));
    MOCHY_CUDA(cudaStreamSynchronize(st));
    if (total < 0) return fail(MOCHY_E_INVALID, "bad offsets");
    if (total > (int64_t)n_edges * MOCHY_MAX_EDGE_SIZE)
      return fail(MOCHY_E_UNSUPPORTED, "hyperedge with more than 63 nodes");
  }
  // temporaries in scratch slot 0
  uint64_t tsize = 1;
  while (tsize < (uint64_t)(2 * n_edges + 2)) tsize <<= 1;
  const size_t need = (size_t)total * 4 + (size_t)tsize * 4 + (size_t)n_edges * 8 * 4 + 64 * 4;
  void* base = nullptr;
  MOCHY_TRY(scratch(ctx, 0, need, &base));
  char* cur = (char*)base;
  auto carve = [&](size_t bytes) { void* r = cur; cur += (bytes + 255) & ~(size_t)255; return r; };
  int32_t* sorted = (int32_t*)carve((size_t)total * 4 + 4);
  int32_t* table = (int32_t*)carve((size_t)tsize * 4);
  int64_t* keep = (int64_t*)carve((size_t)n_edges * 8 + 8);
  int64_t* newid = (int64_t*)carve((size_t)n_edges * 8 + 8);
  int64_t* sizes = (int64_t*)carve((size_t)n_edges * 8 + 8);
  int64_t* newpos = (int64_t*)carve((size_t)n_edges * 8 + 8);
  int32_t* err = ctx->counters;
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  const int T = 256;
  const int nb = std::max(1, ceil_div(n_edges, T));
  if (n_edges > 0) {
    k_validate_sort<<<nb, T, 0, st>>>(d_off, d_nodes, n_edges, n_nodes, sorted, err);
    MOCHY_LAUNCHED();
  }
  int32_t herr = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    std::string m = "invalid hypergraph:";
    if (herr & kErrEmpty) m += " empty hyperedge;";
    if (herr & kErrRange) m += " node id out of range;";
    if (herr & kErrRepeat) m += " node listed twice in a hyperedge;";
    if (herr & kErrOffsets) m += " offsets not starting at 0 or decreasing;";
    if (herr & kErrTooBig) return fail(MOCHY_E_UNSUPPORTED, "hyperedge with more than 63 nodes");
    return fail(MOCHY_E_INVALID, m);
  }
  int64_t kept = 0;
  if (n_edges > 0) {
    MOCHY_CUDA(cudaMemsetAsync(table, 0xff, (size_t)tsize * 4, st));
    k_dedupe_insert<<<nb, T, 0, st>>>(d_off, sorted, n_edges, table, tsize - 1);
    MOCHY_LAUNCHED();
    k_dedupe_mark<<<nb, T, 0, st>>>(d_off, sorted, n_edges, table, tsize - 1, keep);
    MOCHY_LAUNCHED();
    MOCHY_TRY(scan_exclusive_i64(ctx, keep, newid, n_edges));
    k_kept_sizes<<<nb, T, 0, st>>>(d_off, keep, n_edges, sizes);
    MOCHY_LAUNCHED();
    MOCHY_TRY(scan_exclusive_i64(ctx, sizes, newpos, n_edges));
    int64_t last[4];
    MOCHY_CUDA(cudaMemcpyAsync(&last[0], newid + n_edges - 1, 8, cudaMemcpyDeviceToHost, st));
    MOCHY_CUDA(cudaMemcpyAsync(&last[1], keep + n_edges - 1, 8, cudaMemcpyDeviceToHost, st));
    MOCHY_CUDA(cudaMemcpyAsync(&last[2], newpos + n_edges - 1, 8, cudaMemcpyDeviceToHost, st));
    MOCHY_CUDA(cudaMemcpyAsync(&last[3], sizes + n_edges - 1, 8, cudaMemcpyDeviceToHost, st));
    MOCHY_CUDA(cudaStreamSynchronize(st));
    kept = last[0] + last[1];
    ctx->n_inc = last[2] + last[3];
  } else {
    ctx->n_inc = 0;
  }
  ctx->n_nodes = n_nodes;
  ctx->n_edges = kept;
  if (n_dup) *n_dup = n_edges - kept;
  void* p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int64_t) * (size_t)(kept + 1)));
  ctx->eoff = (int64_t*)p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int32_t) * (size_t)std::max<int64_t>(ctx->n_inc, 1)));
  ctx->enode = (int32_t*)p;
  MOCHY_TRY(dev_alloc(ctx, &p, (size_t)std::max<int64_t>(kept, 1)));
  ctx->esize = (uint8_t*)p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int64_t) * (size_t)(n_nodes + 1)));
  ctx->voff = (int64_t*)p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int32_t) * (size_t)std::max<int64_t>(ctx->n_inc, 1)));
  ctx->vedge = (int32_t*)p;
  int32_t* maxsize = ctx->counters + 1;
  if (n_edges > 0) {
    k_compact<<<nb, T, 0, st>>>(d_off, sorted, keep, newid, newpos, n_edges, ctx->eoff,
                                ctx->enode, ctx->esize, maxsize);
    MOCHY_LAUNCHED();
  }
  k_set_last<<<1, 1, 0, st>>>(ctx->eoff, kept, ctx->n_inc);
  MOCHY_LAUNCHED();
  // incidence lists: stable sort of (node, hyperedge) pairs by node
  if (ctx->n_inc > 0) {
    void* t2 = nullptr;
    MOCHY_TRY(scratch(ctx, 2, (size_t)ctx->n_inc * 8 + (size_t)(n_nodes + 1) * 16, &t2));
    uint32_t* key = (uint32_t*)t2;
    uint32_t* val = key + ctx->n_inc;
    unsigned long long* deg = (unsigned long long*)((char*)t2 + (size_t)ctx->n_inc * 8);
    MOCHY_CUDA(cudaMemsetAsync(deg, 0, (size_t)(n_nodes + 1) * 8, st));
    k_incidence_pairs<<<std::max(1, ceil_div(kept, T)), T, 0, st>>>(ctx->eoff, ctx->enode, kept,
                                                                    key, val, deg);
    MOCHY_LAUNCHED();
    MOCHY_TRY(radix_sort_pairs_u32(ctx, key, val, ctx->n_inc, bits_for(n_nodes)));
    MOCHY_TRY(scan_exclusive_i64(ctx, (const int64_t*)deg, ctx->voff, n_nodes + 1));
    MOCHY_CUDA(cudaMemcpyAsync(ctx->vedge, val, (size_t)ctx->n_inc * 4, cudaMemcpyDeviceToDevice, st));
  } else {
    MOCHY_CUDA(cudaMemsetAsync(ctx->voff, 0, sizeof(int64_t) * (size_t)(n_nodes + 1), st));
  }
  int32_t ms = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&ms, maxsize, 4, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  ctx->max_size = ms;
  return MOCHY_OK;
}

}  // namespace mochy

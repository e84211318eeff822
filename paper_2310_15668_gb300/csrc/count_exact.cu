// Exact h-motif / 3h-motif counting (MoCHy-E, Algorithm
// "exact_motif_counting", Section 3.2), reorganised around hyperwedges.
//
// Algorithm exact_motif_counting visits, for each e_i, every pair of its
// neighbours and keeps an instance when it is open (counted at its centre)
// or when e_i has the smallest id (closed).  Here the instances are found
// from hyperwedges instead: a CTA stages the neighbourhood of one hyperedge
// e_a as a 2-bit-per-id code of omega(e_a, e_k) (0 = not adjacent, 1, 2,
// 3 = three or more) in shared memory; its warps take the hyperwedges
// (e_a, e_b) of e_a and stream the row of e_b from e_a onwards.  Each
// instance is counted exactly once:
//   * closed {a, b, k} (all pairs adjacent) when a < b < k;
//   * open with centre b and leaves a, k (a and k not adjacent) when a < k.
// An open instance has one centre and two leaves, so it is met once, from
// its smaller leaf; a closed one once, from its smallest member.  The triple
// intersection of a closed instance is popc(mask(b->a) & mask(b->k)): both
// masks mark nodes of e_b, read from the row of e_b.
#include "classify.cuh"

namespace mochy {
namespace {

constexpr int kExactThreads = 512;
constexpr int kExactWarps = kExactThreads / 32;

struct ExactArgs {
  int64_t n_edges;
  const int64_t* eoff;
  const int32_t* enode;
  const int64_t* noff;
  const uint2* nadj;
  const int32_t* rows;      // rows to stage, in work order
  int64_t n_rows;
  int32_t* queue;           // work-queue counter
  const uint16_t* lut3;
  unsigned long long* hist; // [432]
  int theta;
};

// shared-memory layout: hist[432] u64 | lut[2187] u16 | e_a nodes[64] | codes[]
__global__ void __launch_bounds__(kExactThreads)
k_exact_rows(ExactArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hist = (unsigned long long*)smem;
  uint16_t* lut = (uint16_t*)(hist + 432);
  int32_t* anodes = (int32_t*)(lut + 2192);
  uint32_t* codes = (uint32_t*)(anodes + 64);
  __shared__ int64_t row_slot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t code_words = (g.n_edges + 15) / 16;
  for (int q = threadIdx.x; q < 432; q += kExactThreads) hist[q] = 0ull;
  for (int q = threadIdx.x; q < 2187; q += kExactThreads) lut[q] = g.lut3[q];
  RunCache rc;
  while (true) {
    if (threadIdx.x == 0) row_slot = atomicAdd(g.queue, 1);
    __syncthreads();
    const int64_t slot = row_slot;
    if (slot >= g.n_rows) break;
    const int64_t a = g.rows[slot];
    const int64_t ab = g.noff[a], ae = g.noff[a + 1];
    const int A = (int)(g.eoff[a + 1] - g.eoff[a]);
    if (threadIdx.x < A) anodes[threadIdx.x] = g.enode[g.eoff[a] + threadIdx.x];
    for (int64_t q = threadIdx.x; q < code_words; q += kExactThreads) codes[q] = 0u;
    __syncthreads();
    for (int64_t p = ab + threadIdx.x; p < ae; p += kExactThreads) {
      const uint2 e = g.nadj[p];
      const uint32_t k = ent_id(e);
      const uint32_t w = (uint32_t)min(entry_omega(e.y, A), 3);
      atomicOr(&codes[k >> 4], w << (2 * (k & 15)));
    }
    __syncthreads();
    for (int64_t idx = ab + warp; idx < ae; idx += kExactWarps) {
      const uint2 eab = g.nadj[idx];
      const uint32_t b = ent_id(eab);
      const int B = ent_size(eab);
      const int x = entry_omega(eab.y, A);
      const int64_t bb = g.noff[b], be = g.noff[b + 1];
      const int64_t pa = warp_lower_bound(g.nadj, bb, be, (uint32_t)a);
      const uint32_t mask_ba = g.nadj[pa].y;   // nodes of e_b lying in e_a
      const bool b_after_a = (int64_t)b > a;
      for (int64_t q = pa + 1 + lane; q < be; q += 32) {
        const uint2 ebk = g.nadj[q];
        const uint32_t k = ent_id(ebk);
        const int C = ent_size(ebk);
        const int y = entry_omega(ebk.y, B);
        const int za = (int)((codes[k >> 4] >> (2 * (k & 15))) & 3u);
        int code;
        if (za == 0) {
          // open, centre b, leaves a < k
          code = ternary_code(A, B, C, x, y, 0, 0, g.theta);
        } else if (b_after_a && k > b) {
          // closed, a < b < k
          int z = za;
          if (za == 3) {
            const int64_t kb = g.eoff[k];
            z = sorted_overlap(anodes, A, g.enode + kb, (int)(g.eoff[k + 1] - kb));
          }
          int t;
          if (B <= kMaskedMax) {
            t = __popc(mask_ba & ebk.y);
          } else {
            const int64_t kb = g.eoff[k], bb2 = g.eoff[b];
            t = sorted_overlap3(anodes, A, g.enode + bb2, B, g.enode + kb,
                                (int)(g.eoff[k + 1] - kb));
          }
          code = ternary_code(A, B, C, x, y, z, t, g.theta);
        } else {
          continue;
        }
        rc.add(lut[code], hist);
      }
    }
    __syncthreads();
  }
  rc.flush(hist);
  __syncthreads();
  for (int q = threadIdx.x; q < 432; q += kExactThreads)
    if (hist[q]) atomicAdd(&g.hist[q], hist[q]);
}

// Hyperedge profiles (Section 3.1, "Hyperedge Profile (HP)": the t-th
// element of HP(e) is the number of instances of motif t that include e).
// The instances are enumerated exactly as by k_exact_rows (each once, from
// the CTA of its smallest leaf or smallest member e_a) and each is added to
// the profiles of its three hyperedges: e_a's in a shared row flushed once
// per staged row, e_b's through a per-lane run cache flushed per
// hyperwedge, e_k's by a global atomic.  hp is |E| x 432 (index = 3h id).
__global__ void __launch_bounds__(kExactThreads)
k_hyperedge_profile(ExactArgs g, unsigned long long* __restrict__ hp) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hista = (unsigned long long*)smem;
  uint16_t* lut = (uint16_t*)(hista + 432);
  int32_t* anodes = (int32_t*)(lut + 2192);
  uint32_t* codes = (uint32_t*)(anodes + 64);
  __shared__ int64_t row_slot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t code_words = (g.n_edges + 15) / 16;
  for (int q = threadIdx.x; q < 432; q += kExactThreads) hista[q] = 0ull;
  for (int q = threadIdx.x; q < 2187; q += kExactThreads) lut[q] = g.lut3[q];
  while (true) {
    if (threadIdx.x == 0) row_slot = atomicAdd(g.queue, 1);
    __syncthreads();
    const int64_t slot = row_slot;
    if (slot >= g.n_rows) break;
    const int64_t a = g.rows[slot];
    const int64_t ab = g.noff[a], ae = g.noff[a + 1];
    const int A = (int)(g.eoff[a + 1] - g.eoff[a]);
    if (threadIdx.x < A) anodes[threadIdx.x] = g.enode[g.eoff[a] + threadIdx.x];
    for (int64_t q = threadIdx.x; q < code_words; q += kExactThreads) codes[q] = 0u;
    __syncthreads();
    for (int64_t p = ab + threadIdx.x; p < ae; p += kExactThreads) {
      const uint2 e = g.nadj[p];
      const uint32_t k = ent_id(e);
      const uint32_t w = (uint32_t)min(entry_omega(e.y, A), 3);
      atomicOr(&codes[k >> 4], w << (2 * (k & 15)));
    }
    __syncthreads();
    for (int64_t idx = ab + warp; idx < ae; idx += kExactWarps) {
      const uint2 eab = g.nadj[idx];
      const uint32_t b = ent_id(eab);
      const int B = ent_size(eab);
      const int x = entry_omega(eab.y, A);
      const int64_t bb = g.noff[b], be = g.noff[b + 1];
      const int64_t pa = warp_lower_bound(g.nadj, bb, be, (uint32_t)a);
      const uint32_t mask_ba = g.nadj[pa].y;   // nodes of e_b lying in e_a
      const bool b_after_a = (int64_t)b > a;
      unsigned long long* hpb = hp + (int64_t)b * 432;
      RunCacheT<false> rcb;   // rows of e_b's profile in device memory
      for (int64_t q = pa + 1 + lane; q < be; q += 32) {
        const uint2 ebk = g.nadj[q];
        const uint32_t k = ent_id(ebk);
        const int C = ent_size(ebk);
        const int y = entry_omega(ebk.y, B);
        const int za = (int)((codes[k >> 4] >> (2 * (k & 15))) & 3u);
        int code;
        if (za == 0) {
          // open, centre b, leaves a < k
          code = ternary_code(A, B, C, x, y, 0, 0, g.theta);
        } else if (b_after_a && k > b) {
          // closed, a < b < k
          int z = za;
          if (za == 3) {
            const int64_t kb = g.eoff[k];
            z = sorted_overlap(anodes, A, g.enode + kb, (int)(g.eoff[k + 1] - kb));
          }
          int t;
          if (B <= kMaskedMax) {
            t = __popc(mask_ba & ebk.y);
          } else {
            const int64_t kb = g.eoff[k], bb2 = g.eoff[b];
            t = sorted_overlap3(anodes, A, g.enode + bb2, B, g.enode + kb,
                                (int)(g.eoff[k + 1] - kb));
          }
          code = ternary_code(A, B, C, x, y, z, t, g.theta);
        } else {
          continue;
        }
        const int id = lut[code];
        atomicAdd(&hista[id], 1ull);
        rcb.add(id, hpb);
        atomicAdd(&hp[(int64_t)k * 432 + id], 1ull);
      }
      rcb.flush(hpb);
    }
    __syncthreads();
    unsigned long long* hpa = hp + a * 432;
    for (int q = threadIdx.x; q < 432; q += kExactThreads) {
      const unsigned long long v = hista[q];
      if (v) {
        atomicAdd(&hpa[q], v);
        hista[q] = 0ull;
      }
    }
    __syncthreads();
  }
}

// u in an ascending node list in global memory
__device__ __forceinline__ bool in_sorted(const int32_t* __restrict__ s, int n, int32_t u) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (s[m] < u) lo = m + 1; else hi = m;
  }
  return lo < n && s[lo] == u;
}

// Star node profiles (Section 3.1, "Node Profile (NP)" with star
// ego-networks).  The star ego-network of v keeps the hyperedges that contain
// v, so its instances are exactly the closed instances of G whose triple
// intersection holds v: every closed instance (met once, from its smallest
// member e_a, as in k_exact_rows) is added to the row of each node of
// e_a & e_b & e_k.  np is n_nodes x 432 (index = 3h id).
__global__ void __launch_bounds__(kExactThreads)
k_star_profile(ExactArgs g, unsigned long long* __restrict__ np) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* lut = (uint16_t*)(smem + 432 * 8);
  int32_t* anodes = (int32_t*)(lut + 2192);
  uint32_t* codes = (uint32_t*)(anodes + 64);
  __shared__ int64_t row_slot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t code_words = (g.n_edges + 15) / 16;
  for (int q = threadIdx.x; q < 2187; q += kExactThreads) lut[q] = g.lut3[q];
  while (true) {
    if (threadIdx.x == 0) row_slot = atomicAdd(g.queue, 1);
    __syncthreads();
    const int64_t slot = row_slot;
    if (slot >= g.n_rows) break;
    const int64_t a = g.rows[slot];
    const int64_t ab = g.noff[a], ae = g.noff[a + 1];
    const int A = (int)(g.eoff[a + 1] - g.eoff[a]);
    if (threadIdx.x < A) anodes[threadIdx.x] = g.enode[g.eoff[a] + threadIdx.x];
    for (int64_t q = threadIdx.x; q < code_words; q += kExactThreads) codes[q] = 0u;
    __syncthreads();
    for (int64_t p = ab + threadIdx.x; p < ae; p += kExactThreads) {
      const uint2 e = g.nadj[p];
      const uint32_t k = ent_id(e);
      const uint32_t w = (uint32_t)min(entry_omega(e.y, A), 3);
      atomicOr(&codes[k >> 4], w << (2 * (k & 15)));
    }
    __syncthreads();
    for (int64_t idx = ab + warp; idx < ae; idx += kExactWarps) {
      const uint2 eab = g.nadj[idx];
      const uint32_t b = ent_id(eab);
      if ((int64_t)b <= a) continue;                // closed instances: a < b < k
      const int B = ent_size(eab);
      const int x = entry_omega(eab.y, A);
      const int64_t bb = g.noff[b], be = g.noff[b + 1];
      const int64_t pa = warp_lower_bound(g.nadj, bb, be, (uint32_t)a);
      const uint32_t mask_ba = g.nadj[pa].y;   // nodes of e_b lying in e_a
      const int32_t* bnodes = g.enode + g.eoff[b];
      for (int64_t q = pa + 1 + lane; q < be; q += 32) {
        const uint2 ebk = g.nadj[q];
        const uint32_t k = ent_id(ebk);
        const int za = (int)((codes[k >> 4] >> (2 * (k & 15))) & 3u);
        if (za == 0 || k <= b) continue;
        const int C = ent_size(ebk);
        const int y = entry_omega(ebk.y, B);
        const int32_t* knodes = g.enode + g.eoff[k];
        int z = za;
        if (za == 3) z = sorted_overlap(anodes, A, knodes, C);
        int t;
        if (B <= kMaskedMax) {
          t = __popc(mask_ba & ebk.y);
        } else {
          t = sorted_overlap3(anodes, A, bnodes, B, knodes, C);
        }
        if (t == 0) continue;                   // in no star ego-network
        const int id = lut[ternary_code(A, B, C, x, y, z, t, g.theta)];
        if (B <= kMaskedMax) {
          uint32_t tm = mask_ba & ebk.y;        // positions in e_b of the common nodes
          while (tm) {
            const int pos = __ffs(tm) - 1;
            tm &= tm - 1;
            atomicAdd(&np[(int64_t)bnodes[pos] * 432 + id], 1ull);
          }
        } else {
          for (int q2 = 0; q2 < A; ++q2) {
            const int32_t u = anodes[q2];
            if (in_sorted(bnodes, B, u) && in_sorted(knodes, C, u))
              atomicAdd(&np[(int64_t)u * 432 + id], 1ull);
          }
        }
      }
    }
    __syncthreads();
  }
}

// Test hook: the contribution of the outer-loop iterations of the given
// anchors in Algorithm exact_motif_counting.  For anchor e_x, every pair
// {p, q} of its neighbours with p < q is checked: counted when p and q are
// not adjacent (open, centre x) or x < p (closed, x smallest).  omega(p, q)
// comes from a search in the row of e_p.  One warp per neighbour p.
__global__ void __launch_bounds__(kExactThreads)
k_exact_anchor(ExactArgs g, const int32_t* __restrict__ anchors, int64_t n_anchors) {
  __shared__ unsigned long long hist[432];
  __shared__ uint16_t lut[2187];
  __shared__ int32_t xnodes[64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < 432; q += kExactThreads) hist[q] = 0ull;
  for (int q = threadIdx.x; q < 2187; q += kExactThreads) lut[q] = g.lut3[q];
  RunCache rc;
  for (int64_t ai = blockIdx.x; ai < n_anchors; ai += gridDim.x) {
    const int64_t xrow = anchors[ai];
    const int64_t xb = g.noff[xrow], xe = g.noff[xrow + 1];
    const int X = (int)(g.eoff[xrow + 1] - g.eoff[xrow]);
    __syncthreads();
    if (threadIdx.x < X) xnodes[threadIdx.x] = g.enode[g.eoff[xrow] + threadIdx.x];
    __syncthreads();
    for (int64_t ip = xb + warp; ip < xe; ip += kExactWarps) {
      const uint2 exp_ = g.nadj[ip];
      const uint32_t p = ent_id(exp_);
      const int P = ent_size(exp_);
      const int zxp = entry_omega(exp_.y, X);
      const int64_t pb = g.noff[p], pe = g.noff[p + 1];
      for (int64_t iq = ip + 1 + lane; iq < xe; iq += 32) {
        const uint2 exq = g.nadj[iq];
        const uint32_t q = ent_id(exq);
        const int Q = ent_size(exq);
        const int zxq = entry_omega(exq.y, X);
        // omega(p, q) by binary search of q in the row of p
        int64_t lo = pb, hi = pe;
        while (lo < hi) {
          const int64_t m = (lo + hi) >> 1;
          if (ent_id(g.nadj[m]) < q) lo = m + 1; else hi = m;
        }
        int wpq = 0;
        if (lo < pe && ent_id(g.nadj[lo]) == q) wpq = entry_omega(g.nadj[lo].y, P);
        if (!(wpq == 0 || xrow < (int64_t)p)) continue;
        int t = 0;
        if (wpq > 0) {
          if (X <= kMaskedMax) {
            t = __popc(exp_.y & exq.y);
          } else {
            t = sorted_overlap3(xnodes, X, g.enode + g.eoff[p], P, g.enode + g.eoff[q], Q);
          }
        }
        rc.add(lut[ternary_code(X, P, Q, zxp, wpq, zxq, t, g.theta)], hist);
      }
    }
  }
  rc.flush(hist);
  __syncthreads();
  for (int q = threadIdx.x; q < 432; q += kExactThreads)
    if (hist[q]) atomicAdd(&g.hist[q], hist[q]);
}

}  // namespace

size_t exact_smem_bytes(int64_t n_edges) {
  return 432 * 8 + 2192 * 2 + 64 * 4 + (size_t)((n_edges + 15) / 16) * 4;
}

// The hyperedge profiles of the projected hypergraph into d_hp (|E| x 432,
// cleared here).
int hyperedge_profiles(mochy_ctx* ctx, unsigned long long* d_hp) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  cudaStream_t st = ctx->stream;
  const int64_t E = ctx->n_edges;
  if (E == 0) return MOCHY_OK;
  MOCHY_CUDA(cudaMemsetAsync(d_hp, 0, (size_t)E * 432 * 8, st));
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  ExactArgs g;
  g.n_edges = E;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.rows = ctx->row_order;
  g.n_rows = E;
  g.queue = ctx->counters + 4;
  g.lut3 = ctx->tables.lut3;
  g.hist = nullptr;
  g.theta = ctx->theta;
  const size_t smem = exact_smem_bytes(E);
  if (smem + 1024 > ctx->smem_optin)
    return fail(MOCHY_E_UNSUPPORTED, "hyperedge profiles support at most 786432 hyperedges");
  MOCHY_TRY(ensure_dynamic_smem((const void*)k_hyperedge_profile, smem));
  int per_sm = 0;
  MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hyperedge_profile,
                                                           kExactThreads, smem));
  per_sm = std::max(per_sm, 1);
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)ctx->num_sms * per_sm, E);
  k_hyperedge_profile<<<grid, kExactThreads, smem, st>>>(g, d_hp);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

// The star node profiles of the projected hypergraph into d_np (n_nodes x
// 432, cleared here).
int star_node_profiles(mochy_ctx* ctx, unsigned long long* d_np) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  cudaStream_t st = ctx->stream;
  const int64_t E = ctx->n_edges;
  MOCHY_CUDA(cudaMemsetAsync(d_np, 0, (size_t)std::max<int64_t>(ctx->n_nodes, 1) * 432 * 8, st));
  if (E == 0) return MOCHY_OK;
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  ExactArgs g;
  g.n_edges = E;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.rows = ctx->row_order;
  g.n_rows = E;
  g.queue = ctx->counters + 4;
  g.lut3 = ctx->tables.lut3;
  g.hist = nullptr;
  g.theta = ctx->theta;
  const size_t smem = exact_smem_bytes(E);
  if (smem + 1024 > ctx->smem_optin)
    return fail(MOCHY_E_UNSUPPORTED, "node profiles support at most 786432 hyperedges");
  MOCHY_TRY(ensure_dynamic_smem((const void*)k_star_profile, smem));
  int per_sm = 0;
  MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_star_profile,
                                                           kExactThreads, smem));
  per_sm = std::max(per_sm, 1);
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)ctx->num_sms * per_sm, E);
  k_star_profile<<<grid, kExactThreads, smem, st>>>(g, d_np);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

int count_exact(mochy_ctx* ctx, const int32_t* d_anchors, int64_t n_anchors,
                unsigned long long* d_hist) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  cudaStream_t st = ctx->stream;
  MOCHY_CUDA(cudaMemsetAsync(d_hist, 0, 432 * 8, st));
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  if (ctx->n_edges == 0) return MOCHY_OK;
  ExactArgs g;
  g.n_edges = ctx->n_edges;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.rows = ctx->row_order;
  g.n_rows = ctx->n_edges;
  g.queue = ctx->counters + 4;
  g.lut3 = ctx->tables.lut3;
  g.hist = d_hist;
  g.theta = ctx->theta;
  if (d_anchors) {
    if (n_anchors <= 0) return MOCHY_OK;
    const unsigned grid = (unsigned)std::min<int64_t>(n_anchors, (int64_t)ctx->num_sms * 4);
    k_exact_anchor<<<grid, kExactThreads, 0, st>>>(g, d_anchors, n_anchors);
    MOCHY_LAUNCHED();
    return MOCHY_OK;
  }
  const size_t smem = exact_smem_bytes(ctx->n_edges);
  // leave room for the kernel's static shared memory
  if (smem + 1024 > ctx->smem_optin)
    return fail(MOCHY_E_UNSUPPORTED, "exact counting supports at most 786432 hyperedges");
  MOCHY_TRY(ensure_dynamic_smem((const void*)k_exact_rows, smem));
  int per_sm = 0;
  MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exact_rows, kExactThreads,
                                                           smem));
  per_sm = std::max(per_sm, 1);
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)ctx->num_sms * per_sm, ctx->n_edges);
  k_exact_rows<<<grid, kExactThreads, smem, st>>>(g);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

}  // namespace mochy

// Extensions of the exact count: kh-motifs (Section 4.1 "Extensions Beyond
// Ternary"), instance enumeration (MoCHy-E_ENUM, Algorithm "alg:enum") and
// radial node profiles (Section 3.1 "Node Profile (NP)" with radial
// ego-networks).
//
// kh-motifs and enumeration reuse the per-hyperwedge scan of the exact
// count (count_exact.cu): a CTA stages the neighbourhood of one hyperedge
// e_a as 2-bit codes of omega(e_a, e_k) in shared memory, its warps take the
// hyperwedges (e_a, e_b) and stream the row of e_b from e_a onwards; each
// instance is met exactly once (closed {a, b, k} when a < b < k, open with
// centre b when a < k and e_a, e_k are disjoint).  kh-motifs classify it
// with k states per region; enumeration appends it to an output stream.
#include "classify.cuh"

namespace mochy {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanWarps = kScanThreads / 32;

struct ScanArgs {
  int64_t n_edges;
  const int64_t* eoff;
  const int32_t* enode;
  const int64_t* noff;
  const uint2* nadj;
  const int32_t* rows;
  int64_t n_rows;
  int32_t* queue;
};

// k-state code of the seven regions (Lemma "motif:time" for the
// cardinalities; Section 4.1 for the states): a region of cardinality c has
// state 0 when empty, else 1 + the number of thresholds it exceeds.
__device__ __forceinline__ int kh_state(int c, int k, int thr1, int thr2) {
  return c == 0 ? 0 : 1 + (k > 2 && c > thr1 ? 1 : 0) + (k > 3 && c > thr2 ? 1 : 0);
}

__device__ __forceinline__ int kh_code(int A, int B, int C, int x, int y, int z, int t, int k,
                                       int thr1, int thr2) {
  const int r[7] = {A - x - z + t, B - x - y + t, C - y - z + t, x - t, y - t, z - t, t};
  int code = 0, pw = 1;
#pragma unroll
  for (int p = 0; p < 7; ++p) {
    code += kh_state(r[p], k, thr1, thr2) * pw;
    pw *= k;
  }
  return code;
}

// Regions of the instance met at (a, b, k): (x, y, z, t) with
// x = omega(a, b), y = omega(b, k), z = omega(k, a) and t the triple
// intersection; z = 0 for an open instance centred at b.
struct Meet {
  int C, y, z, t;
  bool valid;
};

__device__ __forceinline__ Meet meet(const ScanArgs& g, const uint32_t* codes, int64_t a,
                                     const int32_t* anodes, int A, uint32_t b, int B,
                                     bool b_after_a, uint32_t mask_ba, uint2 ebk) {
  Meet m{0, 0, 0, 0, false};
  const uint32_t k = ent_id(ebk);
  m.C = ent_size(ebk);
  m.y = entry_omega(ebk.y, B);
  const int za = (int)((codes[k >> 4] >> (2 * (k & 15))) & 3u);
  if (za == 0) {
    m.valid = true;   // open, centre b, leaves a < k
    return m;
  }
  if (!(b_after_a && k > b)) return m;
  // closed, a < b < k
  m.z = za;
  const int64_t kb = g.eoff[k];
  if (za == 3) m.z = sorted_overlap(anodes, A, g.enode + kb, m.C);
  if (B <= kMaskedMax) {
    m.t = __popc(mask_ba & ebk.y);
  } else {
    m.t = sorted_overlap3(anodes, A, g.enode + g.eoff[b], B, g.enode + kb, m.C);
  }
  m.valid = true;
  return m;
}

// Stage row a's neighbourhood codes (all threads of the CTA).
__device__ __forceinline__ void stage_row(const ScanArgs& g, int64_t a, int A, int32_t* anodes,
                                          uint32_t* codes, int64_t code_words) {
  if (threadIdx.x < A) anodes[threadIdx.x] = g.enode[g.eoff[a] + threadIdx.x];
  for (int64_t q = threadIdx.x; q < code_words; q += blockDim.x) codes[q] = 0u;
  __syncthreads();
  for (int64_t p = g.noff[a] + threadIdx.x; p < g.noff[a + 1]; p += blockDim.x) {
    const uint2 e = g.nadj[p];
    const uint32_t k = ent_id(e);
    const uint32_t w = (uint32_t)min(entry_omega(e.y, A), 3);
    atomicOr(&codes[k >> 4], w << (2 * (k & 15)));
  }
  __syncthreads();
}

// kh-motif counts.  Shared: hist[n_bins] u64 | lut (k^7 u16) | anodes[64] | codes.
__global__ void __launch_bounds__(kScanThreads)
k_count_kh(ScanArgs g, const uint16_t* __restrict__ glut, int n_codes, int n_bins, int k,
           int thr1, int thr2, unsigned long long* __restrict__ ghist) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hist = (unsigned long long*)smem;
  uint16_t* lut = (uint16_t*)(hist + n_bins);
  int32_t* anodes = (int32_t*)(lut + ((n_codes + 7) & ~7));
  uint32_t* codes = (uint32_t*)(anodes + 64);
  __shared__ int64_t row_slot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t code_words = (g.n_edges + 15) / 16;
  for (int q = threadIdx.x; q < n_bins; q += kScanThreads) hist[q] = 0ull;
  for (int q = threadIdx.x; q < n_codes; q += kScanThreads) lut[q] = glut[q];
  RunCache rc;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) row_slot = atomicAdd(g.queue, 1);
    __syncthreads();
    const int64_t slot = row_slot;
    if (slot >= g.n_rows) break;
    const int64_t a = g.rows[slot];
    const int A = (int)(g.eoff[a + 1] - g.eoff[a]);
    stage_row(g, a, A, anodes, codes, code_words);
    const int64_t ab = g.noff[a], ae = g.noff[a + 1];
    for (int64_t idx = ab + warp; idx < ae; idx += kScanWarps) {
      const uint2 eab = g.nadj[idx];
      const uint32_t b = ent_id(eab);
      const int B = ent_size(eab);
      const int x = entry_omega(eab.y, A);
      const int64_t bb = g.noff[b], be = g.noff[b + 1];
      const int64_t pa = warp_lower_bound(g.nadj, bb, be, (uint32_t)a);
      const uint32_t mask_ba = g.nadj[pa].y;
      const bool b_after_a = (int64_t)b > a;
      for (int64_t q = pa + 1 + lane; q < be; q += 32) {
        const Meet m = meet(g, codes, a, anodes, A, b, B, b_after_a, mask_ba, g.nadj[q]);
        if (!m.valid) continue;
        rc.add(lut[kh_code(A, B, m.C, x, m.y, m.z, m.t, k, thr1, thr2)], hist);
      }
    }
  }
  rc.flush(hist);
  __syncthreads();
  for (int q = threadIdx.x; q < n_bins; q += kScanThreads)
    if (hist[q]) atomicAdd(&ghist[q], hist[q]);
}

// Instance enumeration: every instance appended once as (i, j, k, h, 3h)
// with i < j < k.  A warp takes a slot range per 32 candidates (one atomic
// on the stream's cursor); rows past `cap` are counted but not written.
// Shared: lut (2187 u16) | anodes[64] | codes.
__global__ void __launch_bounds__(kScanThreads)
k_enumerate(ScanArgs g, const uint16_t* __restrict__ glut, const uint8_t* __restrict__ t2h,
            int theta, int64_t cap, int32_t* __restrict__ out,
            unsigned long long* __restrict__ cursor) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* lut = (uint16_t*)smem;
  int32_t* anodes = (int32_t*)(lut + 2192);
  uint32_t* codes = (uint32_t*)(anodes + 64);
  __shared__ int64_t row_slot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t code_words = (g.n_edges + 15) / 16;
  for (int q = threadIdx.x; q < 2187; q += kScanThreads) lut[q] = glut[q];
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) row_slot = atomicAdd(g.queue, 1);
    __syncthreads();
    const int64_t slot = row_slot;
    if (slot >= g.n_rows) break;
    const int64_t a = g.rows[slot];
    const int A = (int)(g.eoff[a + 1] - g.eoff[a]);
    stage_row(g, a, A, anodes, codes, code_words);
    const int64_t ab = g.noff[a], ae = g.noff[a + 1];
    for (int64_t idx = ab + warp; idx < ae; idx += kScanWarps) {
      const uint2 eab = g.nadj[idx];
      const uint32_t b = ent_id(eab);
      const int B = ent_size(eab);
      const int x = entry_omega(eab.y, A);
      const int64_t bb = g.noff[b], be = g.noff[b + 1];
      const int64_t pa = warp_lower_bound(g.nadj, bb, be, (uint32_t)a);
      const uint32_t mask_ba = g.nadj[pa].y;
      const bool b_after_a = (int64_t)b > a;
      // uniform loop: every lane runs every round, so the ballot is whole
      for (int64_t q0 = pa + 1; q0 < be; q0 += 32) {
        const int64_t q = q0 + lane;
        Meet m{0, 0, 0, 0, false};
        uint32_t k = 0;
        if (q < be) {
          const uint2 ebk = g.nadj[q];
          k = ent_id(ebk);
          m = meet(g, codes, a, anodes, A, b, B, b_after_a, mask_ba, ebk);
        }
        const unsigned have = __ballot_sync(0xffffffffu, m.valid);
        if (!have) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)__popc(have));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (m.valid) {
          const unsigned long long at = base + __popc(have & ((1u << lane) - 1u));
          if ((int64_t)at < cap) {
            const int id3 = lut[ternary_code(A, B, m.C, x, m.y, m.z, m.t, theta)];
            // ascending ids: closed a < b < k; open b between its leaves a < k
            int32_t i0 = (int32_t)a, i1 = (int32_t)b, i2 = (int32_t)k;
            if (m.z == 0) {
              i0 = (int32_t)a;
              i1 = (int32_t)min((int64_t)b, (int64_t)k);
              i2 = (int32_t)max((int64_t)b, (int64_t)k);
              if ((int64_t)b < a) { i0 = (int32_t)b; i1 = (int32_t)a; i2 = (int32_t)k; }
            }
            int32_t* o = out + at * 5;
            o[0] = i0;
            o[1] = i1;
            o[2] = i2;
            o[3] = (int32_t)t2h[id3];
            o[4] = id3;
          }
        }
      }
    }
  }
}

// Radial node profiles: one CTA per node v (work queue).  V_v (the nodes of
// the hyperedges that hold v) is marked in a node bitmap, R_v (the
// hyperedges inside V_v: those of E_v and, since each node of such a
// hyperedge lies in a hyperedge of E_v, neighbours of E_v in the line graph
// whose nodes are all marked) in a hyperedge bitmap and a list.  The
// instances among R_v are then counted by Algorithm "exact_motif_counting"
// run over the anchors of R_v with every neighbour outside R_v skipped: for
// anchor e_x and neighbours p < q of it in R_v, counted when p and q are
// disjoint (open, centre x) or x < p (closed, x smallest).  Each CTA has its
// own bitmaps and list in global scratch.  np is n_nodes x 432.
struct RadialArgs {
  int64_t n_nodes, n_edges;
  const int64_t* eoff;
  const int32_t* enode;
  const int64_t* voff;
  const int32_t* vedge;
  const int64_t* noff;
  const uint2* nadj;
  const uint16_t* lut3;
  int theta;
  int32_t* queue;
  uint32_t* vbits;      // [grid][node words]
  uint32_t* ebits;      // [grid][hyperedge words]
  int32_t* rlist;       // [grid][n_edges]
  unsigned long long* np;
};

__device__ __forceinline__ bool bit_of(const uint32_t* b, int64_t i) {
  return (b[i >> 5] >> (i & 31)) & 1u;
}

__global__ void __launch_bounds__(kScanThreads) k_radial_profile(RadialArgs g) {
  __shared__ unsigned long long hist[432];
  __shared__ uint16_t lut[2192];
  __shared__ int32_t xnodes[kScanWarps][64];
  __shared__ int64_t node_slot;
  __shared__ int n_r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t vw = (g.n_nodes + 31) / 32, ew = (g.n_edges + 31) / 32;
  uint32_t* vbits = g.vbits + (int64_t)blockIdx.x * vw;
  uint32_t* ebits = g.ebits + (int64_t)blockIdx.x * ew;
  int32_t* rlist = g.rlist + (int64_t)blockIdx.x * g.n_edges;
  for (int q = threadIdx.x; q < 2187; q += kScanThreads) lut[q] = g.lut3[q];
  for (int q = threadIdx.x; q < 432; q += kScanThreads) hist[q] = 0ull;
  RunCache rc;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      node_slot = atomicAdd(g.queue, 1);
      n_r = 0;
    }
    __syncthreads();
    const int64_t v = node_slot;
    if (v >= g.n_nodes) break;
    const int64_t vb = g.voff[v], ve = g.voff[v + 1];
    if (ve - vb < 1) continue;
    // V_v: the nodes of the hyperedges of E_v
    for (int64_t q = vb + warp; q < ve; q += kScanWarps) {
      const int64_t e = g.vedge[q];
      for (int64_t p = g.eoff[e] + lane; p < g.eoff[e + 1]; p += 32) {
        const int32_t u = g.enode[p];
        atomicOr(&vbits[u >> 5], 1u << (u & 31));
      }
    }
    __syncthreads();
    // R_v: E_v and the neighbours of E_v inside V_v
    for (int64_t q = vb + warp; q < ve; q += kScanWarps) {
      const int64_t f = g.vedge[q];
      for (int64_t p = g.noff[f] - 1 + lane; p < g.noff[f + 1]; p += 32) {
        // p = noff[f] - 1 stands for f itself
        const int64_t e = p < g.noff[f] ? f : (int64_t)ent_id(g.nadj[p]);
        if (p < g.noff[f] && lane != 0) continue;
        bool inside = true;
        for (int64_t s = g.eoff[e]; s < g.eoff[e + 1] && inside; ++s) {
          const int32_t u = g.enode[s];
          inside = bit_of(vbits, u);
        }
        if (!inside) continue;
        const uint32_t old = atomicOr(&ebits[e >> 5], 1u << (e & 31));
        if (!(old & (1u << (e & 31)))) rlist[atomicAdd(&n_r, 1)] = (int32_t)e;
      }
    }
    __syncthreads();
    const int nr = n_r;
    // instances among R_v: warp per anchor
    for (int ai = warp; ai < nr; ai += kScanWarps) {
      const int64_t xr = rlist[ai];
      const int X = (int)(g.eoff[xr + 1] - g.eoff[xr]);
      if (lane < X) xnodes[warp][lane] = g.enode[g.eoff[xr] + lane];
      if (lane + 32 < X) xnodes[warp][lane + 32] = g.enode[g.eoff[xr] + lane + 32];
      __syncwarp();
      const int64_t xb = g.noff[xr], xe = g.noff[xr + 1];
      for (int64_t ip = xb; ip < xe; ++ip) {
        const uint2 exp_ = g.nadj[ip];
        const uint32_t p = ent_id(exp_);
        if (!bit_of(ebits, p)) continue;
        const int P = ent_size(exp_);
        const int zxp = entry_omega(exp_.y, X);
        const int64_t pb = g.noff[p], pe = g.noff[p + 1];
        for (int64_t iq = ip + 1 + lane; iq < xe; iq += 32) {
          const uint2 exq = g.nadj[iq];
          const uint32_t q = ent_id(exq);
          if (!bit_of(ebits, q)) continue;
          const int Q = ent_size(exq);
          const int zxq = entry_omega(exq.y, X);
          int64_t lo = pb, hi = pe;
          while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (ent_id(g.nadj[m]) < q) lo = m + 1; else hi = m;
          }
          int wpq = 0;
          if (lo < pe && ent_id(g.nadj[lo]) == q) wpq = entry_omega(g.nadj[lo].y, P);
          if (!(wpq == 0 || xr < (int64_t)p)) continue;
          int t = 0;
          if (wpq > 0) {
            if (X <= kMaskedMax) {
              t = __popc(exp_.y & exq.y);
            } else {
              t = sorted_overlap3(xnodes[warp], X, g.enode + g.eoff[p], P, g.enode + g.eoff[q],
                                  Q);
            }
          }
          rc.add(lut[ternary_code(X, P, Q, zxp, wpq, zxq, t, g.theta)], hist);
        }
      }
      __syncwarp();
    }
    rc.flush(hist);
    __syncthreads();
    // row v, then clear the shared histogram and both bitmaps
    for (int q = threadIdx.x; q < 432; q += kScanThreads) {
      g.np[v * 432 + q] = hist[q];
      hist[q] = 0ull;
    }
    for (int i = threadIdx.x; i < nr; i += kScanThreads) {
      const int32_t e = rlist[i];
      ebits[e >> 5] = 0u;
    }
    for (int64_t q = vb + warp; q < ve; q += kScanWarps) {
      const int64_t e = g.vedge[q];
      for (int64_t p = g.eoff[e] + lane; p < g.eoff[e + 1]; p += 32) vbits[g.enode[p] >> 5] = 0u;
    }
  }
}

ScanArgs scan_args(mochy_ctx* ctx) {
  ScanArgs g;
  g.n_edges = ctx->n_edges;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.rows = ctx->row_order;
  g.n_rows = ctx->n_edges;
  g.queue = ctx->counters + 4;
  return g;
}

}  // namespace

// kh-motif counts of the projected hypergraph: d_hist (n_bins = X(k) + 1
// entries, index = kh id) is cleared and filled.
int count_kh(mochy_ctx* ctx, int k, int thr1, int thr2, unsigned long long* d_hist) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  MOCHY_TRY(build_kh_tables(ctx, k));
  cudaStream_t st = ctx->stream;
  const int n_bins = ctx->kh_n + 1;
  MOCHY_CUDA(cudaMemsetAsync(d_hist, 0, (size_t)n_bins * 8, st));
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  if (ctx->n_edges == 0) return MOCHY_OK;
  int n_codes = 1;
  for (int r = 0; r < 7; ++r) n_codes *= k;
  const size_t smem = (size_t)n_bins * 8 + (size_t)((n_codes + 7) & ~7) * 2 + 64 * 4 +
                      (size_t)((ctx->n_edges + 15) / 16) * 4;
  if (smem + 1024 > ctx->smem_optin)
    return fail(MOCHY_E_UNSUPPORTED, "too many hyperedges for the kh-motif count");
  MOCHY_TRY(ensure_dynamic_smem((const void*)k_count_kh, smem));
  int per_sm = 0;
  MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_kh, kScanThreads,
                                                           smem));
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1),
                                                    ctx->n_edges);
  k_count_kh<<<grid, kScanThreads, smem, st>>>(scan_args(ctx), ctx->kh_lut, n_codes, n_bins, k,
                                               thr1, thr2, d_hist);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

// Enumeration into d_out (cap x 5 int32); *d_cursor (cleared here) ends as
// the number of instances.
int enumerate_instances(mochy_ctx* ctx, int64_t cap, int32_t* d_out,
                        unsigned long long* d_cursor) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  cudaStream_t st = ctx->stream;
  MOCHY_CUDA(cudaMemsetAsync(d_cursor, 0, 8, st));
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  if (ctx->n_edges == 0) return MOCHY_OK;
  const size_t smem = 2192 * 2 + 64 * 4 + (size_t)((ctx->n_edges + 15) / 16) * 4;
  if (smem + 1024 > ctx->smem_optin)
    return fail(MOCHY_E_UNSUPPORTED, "too many hyperedges for enumeration");
  MOCHY_TRY(ensure_dynamic_smem((const void*)k_enumerate, smem));
  int per_sm = 0;
  MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enumerate, kScanThreads,
                                                           smem));
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1),
                                                    ctx->n_edges);
  k_enumerate<<<grid, kScanThreads, smem, st>>>(scan_args(ctx), ctx->tables.lut3,
                                                ctx->tables.t2h, ctx->theta, cap, d_out,
                                                d_cursor);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

// Radial node profiles into d_np (n_nodes x 432, every row written).
int radial_node_profiles(mochy_ctx* ctx, unsigned long long* d_np) {
  if (!ctx->projected) return fail(MOCHY_E_NOT_PROJECTED, "call mochy_project first");
  cudaStream_t st = ctx->stream;
  const int64_t N = ctx->n_nodes, E = ctx->n_edges;
  MOCHY_CUDA(cudaMemsetAsync(d_np, 0, (size_t)std::max<int64_t>(N, 1) * 432 * 8, st));
  if (E == 0 || N == 0) return MOCHY_OK;
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  int per_sm = 0;
  MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_radial_profile,
                                                           kScanThreads, 0));
  const int64_t grid = std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1), N);
  const int64_t vw = (N + 31) / 32, ew = (E + 31) / 32;
  const size_t bytes = (size_t)grid * (size_t)(vw + ew + E) * 4;
  void* t = nullptr;
  MOCHY_TRY(scratch(ctx, 1, bytes, &t));
  MOCHY_CUDA(cudaMemsetAsync(t, 0, (size_t)grid * (size_t)(vw + ew) * 4, st));
  RadialArgs g;
  g.n_nodes = N;
  g.n_edges = E;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.voff = ctx->voff;
  g.vedge = ctx->vedge;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.lut3 = ctx->tables.lut3;
  g.theta = ctx->theta;
  g.queue = ctx->counters + 4;
  g.vbits = (uint32_t*)t;
  g.ebits = g.vbits + grid * vw;
  g.rlist = (int32_t*)(g.ebits + grid * ew);
  g.np = d_np;
  k_radial_profile<<<(unsigned)grid, kScanThreads, 0, st>>>(g);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

}  // namespace mochy

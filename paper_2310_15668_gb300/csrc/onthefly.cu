// MoCHy-A+ without the line graph (Section 3.4 "Motif Counting without Line
// Graphs"; Appendix "Details of On-the-Fly MoCHy", Algorithms "alg_memdeg"
// and "alg_memdeg_adv").
//
// The paper memoizes whole neighbourhoods N_e in a hash map within a budget.
// Here no neighbourhood is ever materialized: a neighbourhood is the union
// of the incidence lists E_v of a hyperedge's nodes, and the hyperedge-id
// space is scanned 32 words per warp step (32 x 32 ids), with
//   * a membership bitmap over hyperedge ids for each popular node (the
//     memoized part: built once, as many as the budget allows, most popular
//     first), and
//   * the sorted incidence lists E_v of the other nodes, merged into the
//     scan chunk by chunk.
// Three uses of the scan:
//   1. degrees: d_i = |N_{e_i}| and the number of neighbours after i (the
//      ascending (i, j) order of hyperwedges that MoCHy-A+ draws from);
//   2. the draw: hyperwedge n is index floor(u |wedges| / 2^64) of that
//      order, as for the projected MoCHy-A+, so e_j is the o-th neighbour of
//      e_i after i, found by popcounts along the scan;
//   3. classification: for every e_k in N_i u N_j \ {e_i, e_j}, the counts
//      xa = |e_k & (e_i \ e_j)|, xb = |e_k & (e_j \ e_i)|, xt = |e_k & e_i &
//      e_j| are bit-sliced (3 bits and an overflow flag) from the bitmaps and
//      lists of the nodes of each part; omega_ik = xa + xt, omega_jk = xb +
//      xt and the triple intersection xt give the seven regions (Lemma
//      "motif:time").  For theta = 1 the four commonest (xa, xb, xt) are
//      popcounted per size class; other candidates are grouped per warp by
//      (xa, xb, xt, effective size) in a shared table and classified once
//      per group at the end of the hyperwedge, counts of 4 to 7 are
//      classified at once, and only counts of 8 or more (the slices'
//      overflow) from node lists.
// Every classified instance equals the projected MoCHy-A+'s for the same
// draws, so raw counts and estimates are the same bit for bit.
#include "classify.cuh"
#include "philox.cuh"

namespace mochy {
namespace {

constexpr int kOtfThreads = 256;
constexpr int kOtfWarps = kOtfThreads / 32;
constexpr int kOtfNodes = 128;     // nodes of e_i u e_j
constexpr int kOtfCeff = 16;
constexpr int kOtfKeys = 64 * kOtfCeff;

struct OtfArgs {
  int64_t n_edges, W;             // hyperedges; 32-bit words over hyperedge ids
  const int64_t* eoff;
  const int32_t* enode;
  const uint8_t* esize;
  const int64_t* voff;
  const int32_t* vedge;
  const int32_t* hidx;            // [N] bitmap index of a node, or -1
  const uint32_t* hbits;          // [n_bitmaps][W]
  const uint32_t* sbits;          // per word 4 words: bits 0..3 of min(|e_k|, 15)
  const int64_t* uprefix;         // [E+1] exclusive prefix of the neighbours after i
  int64_t n_wedges;
  const uint16_t* lut3;
  unsigned long long* hist;
  int theta;
  uint64_t seed;
  int64_t samples;
  int32_t* queue;
  int64_t* deg;                   // degree pass: d_i and neighbours after i
  int64_t* up;
  unsigned long long* stats;      // [4] candidates, words scanned, list entries, exact
};

__device__ __forceinline__ void slice_add(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& ovf,
                                          uint32_t m) {
  const uint32_t k0 = c0 & m;
  c0 ^= m;
  const uint32_t k1 = c1 & k0;
  c1 ^= k0;
  ovf |= c2 & k1;
  c2 ^= k1;
}

__device__ __forceinline__ int sval(uint32_t c0, uint32_t c1, uint32_t c2, int bit) {
  return (int)((c0 >> bit) & 1u) + 2 * (int)((c1 >> bit) & 1u) + 4 * (int)((c2 >> bit) & 1u);
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t lo,
                                                   int64_t hi, int64_t x) {
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if ((int64_t)a[m] < x) lo = m + 1; else hi = m;
  }
  return lo;
}

// Per-warp state: the nodes of e_i u e_j split by part (0: e_i only, 1: e_j
// only, 2: both) into bitmap nodes and list nodes, the list cursors, and
// the table of grouped candidates.
struct OtfWarp {
  int32_t anodes[64], bnodes[64];
  int32_t hb[kOtfNodes];          // bitmap index
  int32_t hpart[kOtfNodes];
  int32_t ln[kOtfNodes];          // list node
  int32_t lpart[kOtfNodes];
  int64_t lpos[kOtfNodes], lend[kOtfNodes];
  int64_t lnext[kOtfNodes];       // id of the list's next entry (INT64_MAX when done)
  uint32_t lw[32];                // one list's entries of a chunk, as word masks
  int64_t lmin;                   // smallest next entry over the lists
  int32_t nh, nl;
  uint32_t table[kOtfKeys];
  uint32_t dirty[kOtfKeys / 32];
};

// smallest next entry over the warp's lists, into me.lmin (warp-wide)
__device__ __forceinline__ void update_lmin(OtfWarp& me) {
  const int lane = threadIdx.x & 31;
  int64_t best = INT64_MAX;
  for (int q = lane; q < me.nl; q += 32) best = min(best, me.lnext[q]);
  for (int d = 16; d; d >>= 1) best = min(best, (int64_t)__shfl_xor_sync(0xffffffffu, best, d));
  __syncwarp();
  if (lane == 0) me.lmin = best;
  __syncwarp();
}

// Sort the nodes of e (a = 0) or of e_i and e_j (a = 2) into bitmap and list
// nodes with their parts; list cursors start at the first entry >= from.
__device__ void split_nodes(const OtfArgs& g, OtfWarp& me, int A, int B, bool pair, int64_t from) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) me.nh = me.nl = 0;
  __syncwarp();
  for (int side = 0; side < (pair ? 2 : 1); ++side) {
    const int n = side == 0 ? A : B;
    const int32_t* mine = side == 0 ? me.anodes : me.bnodes;
    const int32_t* other = side == 0 ? me.bnodes : me.anodes;
    const int no = pair ? (side == 0 ? B : A) : 0;
    for (int base = 0; base < n; base += 32) {
      const int l = base + lane;
      const int32_t v = l < n ? mine[l] : -1;
      bool in_other = false;
      if (l < n) {
        int lo = 0, hi = no;
        while (lo < hi) {
          const int m = (lo + hi) >> 1;
          if (other[m] < v) lo = m + 1; else hi = m;
        }
        in_other = lo < no && other[lo] == v;
      }
      // e_j's nodes that e_i also has were taken with e_i (part 2)
      const bool take = l < n && !(side == 1 && in_other);
      const int part = side == 0 ? (in_other ? 2 : 0) : 1;
      const int h = take ? g.hidx[v] : -1;
      const bool isb = take && h >= 0, isl = take && h < 0;
      const unsigned bb = __ballot_sync(0xffffffffu, isb), bl = __ballot_sync(0xffffffffu, isl);
      const int nh0 = me.nh, nl0 = me.nl;
      __syncwarp();
      if (isb) {
        const int q = nh0 + __popc(bb & ((1u << lane) - 1u));
        me.hb[q] = h;
        me.hpart[q] = part;
      }
      if (isl) {
        const int q = nl0 + __popc(bl & ((1u << lane) - 1u));
        me.ln[q] = v;
        me.lpart[q] = part;
        const int64_t vb = g.voff[v], ve = g.voff[v + 1];
        const int64_t ps = lower_bound_i32(g.vedge, vb, ve, from);
        me.lpos[q] = ps;
        me.lend[q] = ve;
        me.lnext[q] = ps < ve ? (int64_t)g.vedge[ps] : INT64_MAX;
      }
      __syncwarp();
      if (lane == 0) {
        me.nh = nh0 + __popc(bb);
        me.nl = nl0 + __popc(bl);
      }
      __syncwarp();
    }
  }
  update_lmin(me);
}

// The bit-sliced counters of the 32 words [w0, w0 + 32) of the three parts
// (this lane's word w0 + lane): bitmap nodes OR-ed in word by word, list
// entries below hi (ids) added one by one by the lane that owns their word.
struct Slices {
  uint32_t c[3][4];   // part -> (bit 0, bit 1, bit 2, overflow)
};

__device__ __forceinline__ void gather_chunk(const OtfArgs& g, OtfWarp& me, int64_t w0,
                                             Slices& s, unsigned long long& n_entries) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < 3; ++p) s.c[p][0] = s.c[p][1] = s.c[p][2] = s.c[p][3] = 0u;
  const int64_t w = w0 + lane;
  const bool inr = w < g.W;
  const int nh = me.nh, nl = me.nl;
  // bitmap nodes, eight loads in flight before their words are added
  for (int q0 = 0; q0 < nh; q0 += 8) {
    uint32_t wd[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      wd[u] = (inr && q0 + u < nh) ? __ldg(&g.hbits[(int64_t)me.hb[q0 + u] * g.W + w]) : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = q0 + u < nh ? me.hpart[q0 + u] : 3;   // 3: no node (word 0)
      if (p == 0) slice_add(s.c[0][0], s.c[0][1], s.c[0][2], s.c[0][3], wd[u]);
      else if (p == 1) slice_add(s.c[1][0], s.c[1][1], s.c[1][2], s.c[1][3], wd[u]);
      else if (p == 2) slice_add(s.c[2][0], s.c[2][1], s.c[2][2], s.c[2][3], wd[u]);
    }
  }
  // list nodes: a list's entries are distinct hyperedges, so its entries in
  // this chunk are one mask per word (shared-memory OR), added once per list
  const int64_t hi = (w0 + 32) * 32;
  if (me.lmin >= hi) return;           // uniform: no list has an entry here
  for (int q = 0; q < nl; ++q) {
    if (me.lnext[q] >= hi) continue;   // uniform: nothing of this list here
    const int p = me.lpart[q];
    while (true) {
      const int64_t pos = me.lpos[q], end = me.lend[q];
      const int64_t e = pos + lane < end ? (int64_t)g.vedge[pos + lane] : INT64_MAX;
      const bool in = e < hi;
      const int nin = __popc(__ballot_sync(0xffffffffu, in));
      if (in) atomicOr(&me.lw[(e >> 5) - w0], 1u << (e & 31));
      n_entries += (unsigned long long)nin;
      const int64_t nx = __shfl_sync(0xffffffffu, e, nin & 31);
      __syncwarp();
      if (lane == 0) {
        me.lpos[q] = pos + nin;
        me.lnext[q] = nin < 32 ? nx : INT64_MAX;
      }
      __syncwarp();
      if (nin < 32) break;
      if (me.lpos[q] >= end) {
        if (lane == 0) me.lnext[q] = INT64_MAX;
        __syncwarp();
        break;
      }
    }
    const uint32_t m = me.lw[lane];
    me.lw[lane] = 0u;
    __syncwarp();
    if (p == 0) slice_add(s.c[0][0], s.c[0][1], s.c[0][2], s.c[0][3], m);
    else if (p == 1) slice_add(s.c[1][0], s.c[1][1], s.c[1][2], s.c[1][3], m);
    else slice_add(s.c[2][0], s.c[2][1], s.c[2][2], s.c[2][3], m);
  }
  update_lmin(me);
}

// first word, at or after w0, that holds an entry of a list node (for
// scans without bitmap nodes); W when none is left
__device__ __forceinline__ int64_t next_list_word(const OtfArgs& g, const OtfWarp& me) {
  return me.lmin == INT64_MAX ? g.W : min(g.W, me.lmin >> 5);
}

__device__ __forceinline__ uint32_t any_of(const Slices& s, int p) {
  return s.c[p][0] | s.c[p][1] | s.c[p][2] | s.c[p][3];
}

// Degrees: one warp per hyperedge e_i; its neighbours are the hyperedges
// marked in the union over its nodes, except i itself.
__global__ void __launch_bounds__(kOtfThreads) k_otf_degrees(OtfArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  OtfWarp& me = ((OtfWarp*)smem)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * kOtfWarps;
  me.lw[lane] = 0u;
  __syncwarp();
  for (int64_t i = (int64_t)blockIdx.x * kOtfWarps + (threadIdx.x >> 5); i < g.n_edges;
       i += nwarps) {
    const int A = (int)(g.eoff[i + 1] - g.eoff[i]);
    if (lane < A) me.anodes[lane] = g.enode[g.eoff[i] + lane];
    if (lane + 32 < A) me.anodes[lane + 32] = g.enode[g.eoff[i] + lane + 32];
    __syncwarp();
    split_nodes(g, me, A, 0, false, 0);
    unsigned long long d = 0, u = 0, ent = 0;
    const bool scan_all = me.nh > 0;
    int64_t w0 = scan_all ? 0 : next_list_word(g, me);
    while (w0 < g.W) {
      Slices s;
      gather_chunk(g, me, w0, s, ent);
      const int64_t w = w0 + lane;
      uint32_t m = w < g.W ? any_of(s, 0) : 0u;
      if (w == (i >> 5)) m &= ~(1u << (i & 31));
      d += __popc(m);
      if (w > (i >> 5)) u += __popc(m);
      else if (w == (i >> 5) && (i & 31) != 31) u += __popc(m & (0xffffffffu << ((i & 31) + 1)));
      w0 = scan_all ? w0 + 32 : max(w0 + 32, next_list_word(g, me));
    }
    for (int dd = 16; dd; dd >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, dd);
      u += __shfl_xor_sync(0xffffffffu, u, dd);
    }
    if (lane == 0) {
      g.deg[i] = (int64_t)d;
      g.up[i] = (int64_t)u;
    }
    __syncwarp();
  }
}

__device__ __forceinline__ int64_t upper_row(const int64_t* __restrict__ pre, int64_t n,
                                             int64_t x) {
  int64_t lo = 0, hi = n;   // pre[0] <= x < pre[n]
  while (hi - lo > 1) {
    const int64_t m = (lo + hi) >> 1;
    if (pre[m] <= x) lo = m; else hi = m;
  }
  return lo;
}

// exact overlaps of e_k with e_i (z), e_j (y) and both (t)
__device__ __forceinline__ void exact_overlaps(const int32_t* a, int A, const int32_t* b, int B,
                                               const int32_t* k, int C, int& z, int& y, int& t) {
  z = y = t = 0;
  for (int q = 0; q < C; ++q) {
    const int32_t u = k[q];
    int lo = 0, hi = A;
    while (lo < hi) { const int m = (lo + hi) >> 1; if (a[m] < u) lo = m + 1; else hi = m; }
    const bool ia = lo < A && a[lo] == u;
    lo = 0; hi = B;
    while (lo < hi) { const int m = (lo + hi) >> 1; if (b[m] < u) lo = m + 1; else hi = m; }
    const bool ib = lo < B && b[lo] == u;
    z += ia; y += ib; t += ia && ib;
  }
}

// Popcounted bins for theta = 1: (xa, xb, xt, effective size).  The motif
// depends on |e_k| only through min(|e_k|, xa + xb + 2 xt + 2), so the last
// size class of each combination stands for every larger size.
__constant__ int kPopBin[13][4] = {
    {0, 0, 1, 1}, {0, 0, 1, 2}, {0, 0, 1, 3}, {0, 0, 1, 4},   // closed through e_i & e_j only
    {1, 0, 0, 1}, {1, 0, 0, 2}, {1, 0, 0, 3},                 // open, centre e_i
    {0, 1, 0, 1}, {0, 1, 0, 2}, {0, 1, 0, 3},                 // open, centre e_j
    {1, 1, 0, 2}, {1, 1, 0, 3}, {1, 1, 0, 4}};                // closed, empty triple region

// One warp per drawn hyperwedge (work queue over the samples).
// Shared: hist[432] | lut[2192] | OtfWarp[kOtfWarps]
__global__ void __launch_bounds__(kOtfThreads) k_otf_sample(OtfArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hist = (unsigned long long*)smem;
  uint16_t* lut = (uint16_t*)(hist + 432);
  OtfWarp& me = ((OtfWarp*)(lut + 2192))[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < 432; q += kOtfThreads) hist[q] = 0ull;
  for (int q = threadIdx.x; q < 2187; q += kOtfThreads) lut[q] = g.lut3[q];
  for (int q = lane; q < kOtfKeys; q += 32) me.table[q] = 0u;
  me.dirty[lane] = 0u;
  me.lw[lane] = 0u;
  __syncthreads();
  const int theta = g.theta;
  unsigned long long st_cand = 0, st_words = 0, st_ent = 0, st_exact = 0;
  while (true) {
    int64_t n = 0;
    if (lane == 0) n = atomicAdd((unsigned long long*)g.queue, 1ull);
    n = __shfl_sync(0xffffffffu, n, 0);
    if (n >= g.samples) break;
    // the draw: hyperwedge index w of the ascending (i, j) order
    const uint64_t uu = philox_u64(g.seed, (uint64_t)n, 2u, 0u);
    const int64_t wi = (int64_t)__umul64hi(uu, (uint64_t)g.n_wedges);
    const int64_t i = upper_row(g.uprefix, g.n_edges, wi);
    int64_t o = wi - g.uprefix[i];
    const int A = (int)(g.eoff[i + 1] - g.eoff[i]);
    if (lane < A) me.anodes[lane] = g.enode[g.eoff[i] + lane];
    if (lane + 32 < A) me.anodes[lane + 32] = g.enode[g.eoff[i] + lane + 32];
    __syncwarp();
    // e_j: the o-th neighbour of e_i after i
    split_nodes(g, me, A, 0, false, i + 1);
    int64_t j = -1;
    {
      const bool scan_all = me.nh > 0;
      int64_t w0 = scan_all ? ((i + 1) >> 5) : next_list_word(g, me);
      while (w0 < g.W && j < 0) {
        Slices s;
        gather_chunk(g, me, w0, s, st_ent);
        const int64_t w = w0 + lane;
        uint32_t m = w < g.W ? any_of(s, 0) : 0u;
        if (w < ((i + 1) >> 5)) m = 0u;
        if (w == ((i + 1) >> 5)) m &= 0xffffffffu << ((i + 1) & 31);
        const int c = __popc(m);
        int incl = c;
        for (int d = 1; d < 32; d <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += t;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (o < tot) {
          const unsigned at = __ballot_sync(0xffffffffu, incl > o);
          const int src = __ffs(at) - 1;
          const int before = __shfl_sync(0xffffffffu, incl - c, src);
          const uint32_t ms = __shfl_sync(0xffffffffu, m, src);
          const int64_t ws = __shfl_sync(0xffffffffu, w, src);
          j = ws * 32 + (int64_t)__fns(ms, 0, (int)(o - before) + 1);
        } else {
          o -= tot;
        }
        w0 = scan_all ? w0 + 32 : max(w0 + 32, next_list_word(g, me));
      }
    }
    if (j < 0) {
      // cannot happen when the degrees are consistent: counted as an
      // instance of no motif, which the host reports as an internal error
      if (lane == 0) atomicAdd(&hist[0], 1ull);
      continue;
    }
    const int B = (int)(g.eoff[j + 1] - g.eoff[j]);
    if (lane < B) me.bnodes[lane] = g.enode[g.eoff[j] + lane];
    if (lane + 32 < B) me.bnodes[lane + 32] = g.enode[g.eoff[j] + lane + 32];
    __syncwarp();
    split_nodes(g, me, A, B, true, 0);
    // x = |e_i & e_j|
    int x = 0;
    for (int q = lane; q < A; q += 32) {
      const int32_t v = me.anodes[q];
      int lo = 0, hi = B;
      while (lo < hi) { const int m = (lo + hi) >> 1; if (me.bnodes[m] < v) lo = m + 1; else hi = m; }
      x += lo < B && me.bnodes[lo] == v;
    }
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    // classification of N_i u N_j \ {i, j}
    const bool scan_all = me.nh > 0;
    // theta = 1: per-lane counts of the four commonest (xa, xb, xt) by
    // size class (see kPopBin below); the others go through the table
    uint32_t bins[13];
#pragma unroll
    for (int b = 0; b < 13; ++b) bins[b] = 0u;
    int64_t w0 = scan_all ? 0 : next_list_word(g, me);
    while (w0 < g.W) {
      Slices s;
      gather_chunk(g, me, w0, s, st_ent);
      const int64_t w = w0 + lane;
      const bool inr = w < g.W;
      uint32_t m = inr ? (any_of(s, 0) | any_of(s, 1) | any_of(s, 2)) : 0u;
      if (w == (i >> 5)) m &= ~(1u << (i & 31));
      if (w == (j >> 5)) m &= ~(1u << (j & 31));
      st_words += inr ? 1 : 0;
      st_cand += __popc(m);
      const uint4 ps = inr ? __ldg(&((const uint4*)g.sbits)[w]) : make_uint4(0u, 0u, 0u, 0u);
      const uint32_t p0 = ps.x, p1 = ps.y, p2 = ps.z, p3 = ps.w;
      const uint32_t ovf = s.c[0][3] | s.c[1][3] | s.c[2][3];
      if (theta == 1) {
        const uint32_t az = ~(s.c[0][0] | s.c[0][1] | s.c[0][2] | s.c[0][3]);
        const uint32_t a1 = s.c[0][0] & ~(s.c[0][1] | s.c[0][2] | s.c[0][3]);
        const uint32_t bz = ~(s.c[1][0] | s.c[1][1] | s.c[1][2] | s.c[1][3]);
        const uint32_t b1 = s.c[1][0] & ~(s.c[1][1] | s.c[1][2] | s.c[1][3]);
        const uint32_t tz = ~(s.c[2][0] | s.c[2][1] | s.c[2][2] | s.c[2][3]);
        const uint32_t t1 = s.c[2][0] & ~(s.c[2][1] | s.c[2][2] | s.c[2][3]);
        const uint32_t c001 = m & az & bz & t1, c100 = m & a1 & bz & tz;
        const uint32_t c010 = m & az & b1 & tz, c110 = m & a1 & b1 & tz;
        const uint32_t hi4 = p2 | p3;
        const uint32_t e1 = ~hi4 & ~p1 & p0, e2 = ~hi4 & p1 & ~p0, e3 = ~hi4 & p1 & p0;
        const uint32_t ge3 = e3 | hi4;
        bins[0] += __popc(c001 & e1);
        bins[1] += __popc(c001 & e2);
        bins[2] += __popc(c001 & e3);
        bins[3] += __popc(c001 & hi4);
        bins[4] += __popc(c100 & e1);
        bins[5] += __popc(c100 & e2);
        bins[6] += __popc(c100 & ge3);
        bins[7] += __popc(c010 & e1);
        bins[8] += __popc(c010 & e2);
        bins[9] += __popc(c010 & ge3);
        bins[10] += __popc(c110 & e2);
        bins[11] += __popc(c110 & e3);
        bins[12] += __popc(c110 & hi4);
        m &= ~(c001 | c100 | c010 | c110);
      }
      // remaining candidates, 32 at a time over the whole warp: lane l takes
      // the l-th remaining candidate of this chunk
      const int rc = __popc(m);
      int incl = rc;
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      for (int base = 0; base < total; base += 32) {
        const int item = base + lane;
        int src = 0;
#pragma unroll
        for (int stp = 16; stp; stp >>= 1) {
          const int probe = __shfl_sync(0xffffffffu, incl, src + stp - 1);
          if (probe <= item) src += stp;
        }
        src &= 31;
        const int ex = __shfl_sync(0xffffffffu, incl - rc, src);
        const uint32_t ms = __shfl_sync(0xffffffffu, m, src);
        uint32_t sc[3][4];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int b = 0; b < 4; ++b) sc[p][b] = __shfl_sync(0xffffffffu, s.c[p][b], src);
        const uint32_t so = __shfl_sync(0xffffffffu, ovf, src);
        const uint32_t q0 = __shfl_sync(0xffffffffu, p0, src), q1 = __shfl_sync(0xffffffffu, p1, src);
        const uint32_t q2 = __shfl_sync(0xffffffffu, p2, src), q3 = __shfl_sync(0xffffffffu, p3, src);
        const int64_t sw = __shfl_sync(0xffffffffu, w, src);
        const bool act = item < total;
        int key = -1;
        if (act) {
          const int bit = __fns(ms, 0, item - ex + 1);
          const int64_t k = sw * 32 + bit;
          int C = (int)((q0 >> bit) & 1u) | ((int)((q1 >> bit) & 1u) << 1) |
                  ((int)((q2 >> bit) & 1u) << 2) | ((int)((q3 >> bit) & 1u) << 3);
          if (C >= 15) C = g.esize[k];
          const int xa = sval(sc[0][0], sc[0][1], sc[0][2], bit);
          const int xb = sval(sc[1][0], sc[1][1], sc[1][2], bit);
          const int xt = sval(sc[2][0], sc[2][1], sc[2][2], bit);
          const int ce = min(C, xa + xb + 2 * xt + theta + 1);
          const bool over = (so >> bit) & 1u;   // some count is 8 or more
          if (!over && xa < 4 && xb < 4 && xt < 4 && ce <= kOtfCeff) {
            key = ((xa * 4 + xb) * 4 + xt) * kOtfCeff + ce - 1;
          } else if (!over) {
            // counts below 8 are exact: classified at once
            atomicAdd(&hist[lut[ternary_code(A, B, C, x, xb + xt, xa + xt, xt, theta)]], 1ull);
          } else {
            int z, y, t;
            exact_overlaps(me.anodes, A, me.bnodes, B, g.enode + g.eoff[k], C, z, y, t);
            atomicAdd(&hist[lut[ternary_code(A, B, C, x, y, z, t, theta)]], 1ull);
            ++st_exact;
          }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && (peers & ((1u << lane) - 1u)) == 0) {
          atomicAdd(&me.table[key], (uint32_t)__popc(peers));
          atomicOr(&me.dirty[key >> 5], 1u << (key & 31));
        }
      }
      w0 = scan_all ? w0 + 32 : max(w0 + 32, next_list_word(g, me));
    }
    // the popcounted bins: (xa, xb, xt) and the size they stand for
    if (theta == 1) {
      uint32_t mine = 0u;
#pragma unroll
      for (int b = 0; b < 13; ++b) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, bins[b]);
        if (lane == b) mine = v;
      }
      if (lane < 13 && mine) {
        const int xa = kPopBin[lane][0], xb = kPopBin[lane][1], xt = kPopBin[lane][2];
        const int ce = kPopBin[lane][3];
        atomicAdd(&hist[lut[ternary_code(A, B, ce, x, xb + xt, xa + xt, xt, 1)]],
                  (unsigned long long)mine);
      }
    }
    // the groups of this hyperwedge, classified once each
    __syncwarp();
    uint32_t dw = me.dirty[lane];
    me.dirty[lane] = 0u;
    while (dw) {
      const int q = lane * 32 + __ffs(dw) - 1;
      dw &= dw - 1;
      const uint32_t cnt = me.table[q];
      me.table[q] = 0u;
      if (!cnt) continue;
      const int ce = q % kOtfCeff + 1, combo = q / kOtfCeff;
      const int xt = combo & 3, xb = (combo >> 2) & 3, xa = combo >> 4;
      atomicAdd(&hist[lut[ternary_code(A, B, ce, x, xb + xt, xa + xt, xt, theta)]],
                (unsigned long long)cnt);
    }
    __syncwarp();
  }
  if (g.stats) {
    for (int d = 16; d; d >>= 1) {
      st_cand += __shfl_xor_sync(0xffffffffu, st_cand, d);
      st_words += __shfl_xor_sync(0xffffffffu, st_words, d);
      st_ent += __shfl_xor_sync(0xffffffffu, st_ent, d);
      st_exact += __shfl_xor_sync(0xffffffffu, st_exact, d);
    }
    if (lane == 0) {
      atomicAdd(&g.stats[0], st_cand);
      atomicAdd(&g.stats[1], st_words);
      atomicAdd(&g.stats[2], st_ent);
      atomicAdd(&g.stats[3], st_exact);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 432; q += kOtfThreads)
    if (hist[q]) atomicAdd(&g.hist[q], hist[q]);
}

// membership bitmap of each bitmap node (its incidence list as bits)
__global__ void k_otf_bits(int64_t n_bitmaps, int64_t W, const int32_t* __restrict__ nodes_of,
                           const int64_t* __restrict__ voff, const int32_t* __restrict__ vedge,
                           uint32_t* __restrict__ bits) {
  for (int64_t h = blockIdx.x; h < n_bitmaps; h += gridDim.x) {
    const int32_t v = nodes_of[h];
    uint32_t* b = bits + h * W;
    for (int64_t q = voff[v] + threadIdx.x; q < voff[v + 1]; q += blockDim.x) {
      const int32_t e = vedge[q];
      atomicOr(&b[e >> 5], 1u << (e & 31));
    }
  }
}

__global__ void k_otf_size_bits(int64_t E, int64_t W, const uint8_t* __restrict__ esize,
                                uint32_t* __restrict__ sbits) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= E) return;
  const int c = min((int)esize[k], 15);
  for (int b = 0; b < 4; ++b)
    if (c & (1 << b)) atomicOr(&sbits[4 * (k >> 5) + b], 1u << (k & 31));
}

}  // namespace

size_t otf_smem_bytes() { return 432 * 8 + 2192 * 2 + sizeof(OtfWarp) * kOtfWarps; }

void release_onthefly(mochy_ctx* ctx) {
  if (ctx->otf_block) {
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, ctx->otf_block, ctx->otf_bytes);
  }
  ctx->otf_block = nullptr;
  ctx->otf_bytes = 0;
  ctx->otf_ready = false;
  ctx->otf_hidx = nullptr;
  ctx->otf_hbits = nullptr;
  ctx->otf_sbits = nullptr;
  ctx->otf_uprefix = nullptr;
  ctx->otf_wedges = ctx->otf_bitmaps = ctx->otf_words = 0;
}

// Bitmaps, size planes, degrees and the prefix of the neighbours after each
// hyperedge.  budget: bytes for bitmaps (<= 0: the library's choice).
int prepare_onthefly(mochy_ctx* ctx, int64_t budget) {
  if (ctx->otf_ready) return MOCHY_OK;
  cudaStream_t st = ctx->stream;
  const int64_t E = ctx->n_edges, N = ctx->n_nodes;
  const int64_t W = std::max<int64_t>((E + 31) / 32, 1);
  // bitmap nodes: degree >= W / 32 (a bitmap costs about what a list of
  // that length costs to merge), most popular first, within the budget
  std::vector<int64_t> voff((size_t)N + 1);
  MOCHY_CUDA(cudaMemcpyAsync(voff.data(), ctx->voff, voff.size() * 8, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  const int64_t thr = std::max<int64_t>(W / 32, 16);
  std::vector<std::pair<int64_t, int32_t>> pop;
  for (int64_t v = 0; v < N; ++v)
    if (voff[v + 1] - voff[v] >= thr) pop.push_back({-(voff[v + 1] - voff[v]), (int32_t)v});
  std::sort(pop.begin(), pop.end());
  const int64_t cap_bytes =
      budget > 0 ? budget : (ctx->budget > 0 ? ctx->budget / 4 : ((int64_t)4 << 30));
  const int64_t max_bitmaps = std::min<int64_t>((int64_t)pop.size(), cap_bytes / (W * 4));
  std::vector<int32_t> hidx((size_t)N, -1), nodes_of((size_t)std::max<int64_t>(max_bitmaps, 1), 0);
  for (int64_t h = 0; h < max_bitmaps; ++h) {
    hidx[(size_t)pop[h].second] = (int32_t)h;
    nodes_of[(size_t)h] = pop[h].second;
  }
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_hidx = al((size_t)std::max<int64_t>(N, 1) * 4);
  const size_t b_nodes = al(nodes_of.size() * 4);
  const size_t b_bits = al((size_t)std::max<int64_t>(max_bitmaps, 1) * W * 4);
  const size_t b_sbits = al((size_t)4 * W * 4);
  const size_t b_pre = al((size_t)(E + 1) * 8);
  const size_t b_deg = al((size_t)std::max<int64_t>(E, 1) * 8);
  const size_t bytes = b_hidx + b_nodes + b_bits + b_sbits + b_pre + 2 * b_deg;
  void* p = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &p, bytes));
  char* c = (char*)p;
  ctx->otf_block = p;
  ctx->otf_bytes = bytes;
  ctx->otf_hidx = (int32_t*)c;
  int32_t* d_nodes_of = (int32_t*)(c + b_hidx);
  ctx->otf_hbits = (uint32_t*)(c + b_hidx + b_nodes);
  ctx->otf_sbits = (uint32_t*)(c + b_hidx + b_nodes + b_bits);
  ctx->otf_uprefix = (int64_t*)(c + b_hidx + b_nodes + b_bits + b_sbits);
  int64_t* deg = (int64_t*)(c + b_hidx + b_nodes + b_bits + b_sbits + b_pre);
  int64_t* up = (int64_t*)((char*)deg + b_deg);
  auto bail = [&](int rc) { release_onthefly(ctx); return rc; };
  if (cudaMemcpyAsync(ctx->otf_hidx, hidx.data(), (size_t)N * 4, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(d_nodes_of, nodes_of.data(), nodes_of.size() * 4, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemsetAsync(ctx->otf_hbits, 0, b_bits + b_sbits, st) != cudaSuccess)
    return bail(fail(MOCHY_E_CUDA, "on-the-fly set-up copy failed"));
  if (max_bitmaps > 0) {
    k_otf_bits<<<(unsigned)std::min<int64_t>(max_bitmaps, 4096), 256, 0, st>>>(
        max_bitmaps, W, d_nodes_of, ctx->voff, ctx->vedge, ctx->otf_hbits);
    note_launch();
  }
  if (E > 0) {
    k_otf_size_bits<<<ceil_div(E, 256), 256, 0, st>>>(E, W, ctx->esize, ctx->otf_sbits);
    note_launch();
  }
  OtfArgs g{};
  g.n_edges = E;
  g.W = W;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.esize = ctx->esize;
  g.voff = ctx->voff;
  g.vedge = ctx->vedge;
  g.hidx = ctx->otf_hidx;
  g.hbits = ctx->otf_hbits;
  g.sbits = ctx->otf_sbits;
  g.deg = deg;
  g.up = up;
  const size_t smem = sizeof(OtfWarp) * kOtfWarps;
  {
    const int rc = ensure_dynamic_smem((const void*)k_otf_degrees, smem);
    if (rc < 0) return bail(rc);
  }
  if (E > 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_otf_degrees, kOtfThreads, smem);
    const int64_t grid = std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1),
                                           (E + kOtfWarps - 1) / kOtfWarps);
    k_otf_degrees<<<(unsigned)grid, kOtfThreads, smem, st>>>(g);
    note_launch();
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bail(cuda_fail(e, "on-the-fly degrees", __FILE__, __LINE__));
  {
    const int rc = scan_exclusive_i64(ctx, up, ctx->otf_uprefix, E + 1);
    if (rc < 0) return bail(rc);
  }
  int64_t total = 0;
  if (cudaMemcpyAsync(&total, ctx->otf_uprefix + E, 8, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return bail(fail(MOCHY_E_CUDA, "on-the-fly prefix copy failed"));
  ctx->otf_wedges = total;
  ctx->otf_bitmaps = max_bitmaps;
  ctx->otf_words = W;
  ctx->otf_ready = true;
  return MOCHY_OK;
}

// MoCHy-A+ of `samples` draws without the line graph into d_hist (432,
// cleared here).  stats (may be null): [4] candidates, words, list
// entries, exact classifications.
int count_sampled_onthefly(mochy_ctx* ctx, int64_t samples, uint64_t seed, int64_t budget,
                           unsigned long long* d_hist, unsigned long long* d_stats) {
  if (samples <= 0) return fail(MOCHY_E_INVALID, "samples must be positive");
  MOCHY_TRY(prepare_onthefly(ctx, budget));
  if (ctx->otf_wedges == 0) return fail(MOCHY_E_INVALID, "the hypergraph has no hyperwedge");
  cudaStream_t st = ctx->stream;
  MOCHY_CUDA(cudaMemsetAsync(d_hist, 0, 432 * 8, st));
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  OtfArgs g{};
  g.n_edges = ctx->n_edges;
  g.W = ctx->otf_words;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.esize = ctx->esize;
  g.voff = ctx->voff;
  g.vedge = ctx->vedge;
  g.hidx = ctx->otf_hidx;
  g.hbits = ctx->otf_hbits;
  g.sbits = ctx->otf_sbits;
  g.uprefix = ctx->otf_uprefix;
  g.n_wedges = ctx->otf_wedges;
  g.lut3 = ctx->tables.lut3;
  g.hist = d_hist;
  g.theta = ctx->theta;
  g.seed = seed;
  g.samples = samples;
  g.queue = ctx->counters + 4;   // 64-bit counter over words 4 and 5
  g.stats = d_stats;
  if (d_stats) MOCHY_CUDA(cudaMemsetAsync(d_stats, 0, 4 * 8, st));
  const size_t smem = otf_smem_bytes();
  MOCHY_TRY(ensure_dynamic_smem((const void*)k_otf_sample, smem));
  int per_sm = 0;
  MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_otf_sample, kOtfThreads,
                                                           smem));
  const int64_t grid = std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1),
                                         (samples + kOtfWarps - 1) / kOtfWarps);
  k_otf_sample<<<(unsigned)grid, kOtfThreads, smem, st>>>(g);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

}  // namespace mochy

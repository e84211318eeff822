// Exact counting (MoCHy-E, Algorithm "exact_motif_counting", Section 3.2)
// split into open and closed instances.
//
// Algorithm exact_motif_counting enumerates, for each centre e_c, every pair
// {e_p, e_q} of its neighbours.  Here the same counts are reached in two
// parts.
//
// Open instances.  For a pair of neighbours that are not adjacent the seven
// regions (Lemma "motif:time") are |e_c| - w_p - w_q, |e_p| - w_p,
// |e_q| - w_q, w_p, 0, w_q, 0 (w_x = |e_c & e_x|), so the motif depends only
// on the class (w_x, min(|e_x| - w_x, theta + 1)) of each leaf.  Per centre,
// the pairs of all neighbour classes are counted from a class histogram; the
// pairs that are in fact adjacent (closed triangles through e_c) are then
// taken out again, one "as if open" term per centre of every triangle.  A pair
// whose overlaps with e_c exceed |e_c| cannot be open and is skipped on both
// sides.
//
// Closed instances (triangles of the line graph) are enumerated once each,
// from their smallest member in the order "sparse rows (by id) before dense
// rows (by line degree, then id)", where a row is dense when its line degree
// is at least a threshold.  A triangle of three dense rows is found with bitmaps over the
// dense rows: 32 candidate third hyperedges per word, and when both overlaps
// with the candidate are 1 the triple intersection is whether the candidate
// holds a node of e_a & e_b (node bitmaps), so such candidates are counted by
// popcount per (triple intersection, size class).  Every other candidate is
// classified exactly from node lists.  Triangles with a sparse smallest member
// are enumerated from a staged copy of that member's row.
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "classify.cuh"

namespace mochy {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kOpenThreads = 256;
constexpr int kOpenWarps = kOpenThreads / 32;
constexpr int kTable = 256;   // per-warp class table of the open-pair kernel
constexpr int kClasses = 5;   // size classes of a simple closed candidate
// tracing counters: [0..7] totals and cycles, [8..71] rest combinations,
// [72..79] setup sections and sizes, [80] signature slots evicted, [81]
// slots flushed full, [82] dense rows counted
constexpr int kStatWords = 88;

// Size class of |e_k| for a closed candidate with both overlaps 1: its motif
// and its three "as if open" terms depend on |e_k| only through the states
// of |e_k| - 1 and |e_k| - 2 and whether |e_k| >= 2.
__host__ __device__ inline int size_class(int C, int theta) {
  if (C <= 1) return 0;
  if (C == 2) return 1;
  if (C <= theta + 1) return 2;
  if (C == theta + 2) return 3;
  return 4;
}

__device__ inline int class_rep(int c, int theta) {
  return c == 0 ? 1 : c == 1 ? 2 : c == 2 ? 3 : c == 3 ? theta + 2 : theta + 3;
}

// h[id] += v on a shared 64-bit bin (see shared_bin_add)
__device__ __forceinline__ void hadd(unsigned long long* h, int id, long long v) {
  shared_bin_add(h, id, v);
}

// One closed instance {a, b, k} with sizes A, B, C, omega_ab = x,
// omega_bk = y, omega_ka = z and triple intersection t, counted n times:
// its motif, minus its "as if open" term at each centre (see above).
__device__ __forceinline__ void add_triangle(unsigned long long* hist, const uint16_t* lut, int theta,
                                             int A, int B, int C, int x, int y, int z, int t,
                                             long long n) {
  hadd(hist, lut[ternary_code(A, B, C, x, y, z, t, theta)], n);
  if (x + z <= A) hadd(hist, lut[ternary_code(A, B, C, x, 0, z, 0, theta)], -n);
  if (x + y <= B) hadd(hist, lut[ternary_code(B, A, C, x, 0, y, 0, theta)], -n);
  if (z + y <= C) hadd(hist, lut[ternary_code(C, A, B, z, 0, y, 0, theta)], -n);
}

// n closed instances of one table key of hyperwedge (a, b): A = |e_a|,
// B = |e_b|, omega_ab = x, and a third hyperedge holding xa nodes of
// e_a \ e_b, xb of e_b \ e_a and xt of both, with effective size
// xa + xb + xt + rel.  The same codes as add_triangle with y = xb + xt,
// z = xa + xt, t = xt, written with the regions that involve the third
// hyperedge already reduced.
__device__ __forceinline__ void add_key(unsigned long long* hist, const uint16_t* lut, int theta,
                                        int A, int B, int x, int xa, int xb, int xt, int rel,
                                        long long n) {
  auto st = [theta](int r) { return (r > 0 ? 1 : 0) + (r > theta ? 1 : 0); };
  const int y = xb + xt, z = xa + xt;
  hadd(hist, lut[st(A - x - xa) + 3 * st(B - x - xb) + 9 * st(rel) + 27 * st(x - xt) +
                 81 * st(xb) + 243 * st(xa) + 729 * st(xt)], n);
  if (x + z <= A)
    hadd(hist, lut[st(A - x - z) + 3 * st(B - x) + 9 * st(xb + rel) + 27 * st(x) + 243 * st(z)], -n);
  if (x + y <= B)
    hadd(hist, lut[st(B - x - y) + 3 * st(A - x) + 9 * st(xa + rel) + 27 * st(x) + 243 * st(y)], -n);
  if (xt <= rel)
    hadd(hist, lut[st(rel - xt) + 3 * st(A - z) + 9 * st(B - y) + 27 * st(z) + 243 * st(y)], -n);
}

// binary search of node u in an ascending list in shared memory
__device__ __forceinline__ bool has_node(const int32_t* s, int n, int32_t u) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (s[m] < u) lo = m + 1; else hi = m;
  }
  return lo < n && s[lo] == u;
}

struct SplitArgs {
  int64_t n_edges;
  const int64_t* eoff;
  const int32_t* enode;
  const int64_t* voff;
  const int32_t* vedge;
  const int64_t* noff;
  const uint2* nadj;
  const uint16_t* lut3;
  unsigned long long* hist;
  int theta;
  // split structures
  int64_t n_dense, wwords;
  const int32_t* dense_idx;
  const int32_t* dense_row;
  const uint32_t* dbits;
  const int32_t* heavy_idx;
  const uint32_t* nbits;
  const uint32_t* sbits;
  const int64_t* dvoff;
  const int32_t* dvedge;
  const uint8_t* dsize;
  const uint32_t* cbits;     // [5][W] size classes (theta other than 1)
  unsigned long long* stats; // tracing counters or null
  const int32_t* order;
  int64_t n_order;
  int32_t* queue;
  // open pairs: only these centres when non-null (a subset of the rows)
  const int32_t* centres;
  int64_t n_centres;
  // batch of disjoint hypergraphs: hist holds n_units histograms of 432
  int32_t n_units;
  const int64_t* nseg;       // [n_units+1] node ranges
  const SegInfo* seg;        // [n_units]
};

// unit (hypergraph of a batch) of hyperedge a: the one owning its first node
__device__ __forceinline__ int unit_of_edge(const SplitArgs& g, int64_t a) {
  return seg_of(g.nseg, g.n_units, g.enode[g.eoff[a]]);
}

// Block-wide, between barriers: the shared histogram holds the counts of
// unit `cur`; before rows of unit `next` are counted it is added to cur's
// global histogram and cleared.  Ends with a barrier when it switches.
__device__ __forceinline__ void switch_unit(unsigned long long* hist, unsigned long long* ghist,
                                            int& cur, int next) {
  if (next == cur) return;
  for (int q = threadIdx.x; q < 432; q += blockDim.x) {
    const unsigned long long v = hist[q];
    if (v) {
      atomicAdd(&ghist[(int64_t)cur * 432 + q], v);
      hist[q] = 0ull;
    }
  }
  cur = next;
  __syncthreads();
}

__device__ __forceinline__ void load_lut(uint16_t* lut, const uint16_t* g, unsigned long long* hist) {
  for (int q = threadIdx.x; q < 432; q += blockDim.x) hist[q] = 0ull;
  for (int q = threadIdx.x; q < 2187; q += blockDim.x) lut[q] = g[q];
}

__device__ __forceinline__ void flush_hist(unsigned long long* g, const unsigned long long* h) {
  for (int q = threadIdx.x; q < 432; q += blockDim.x)
    if (h[q]) atomicAdd(&g[q], h[q]);
}

// ---------------------------------------------------------------------------
// Open pairs: one warp per centre row.
// ---------------------------------------------------------------------------
// Open-pair counts of centre c (one warp) into hist.
__device__ __forceinline__ void open_centre(const SplitArgs& g, int64_t c, unsigned long long* hist,
                                            const uint16_t* lut, int32_t* key, int32_t* cnt) {
  const int lane = threadIdx.x & 31;
  constexpr int kPer = kTable / 32;
  const int64_t rb = g.noff[c], re = g.noff[c + 1];
  if (re - rb < 2) return;
  const int A = (int)(g.eoff[c + 1] - g.eoff[c]);
  for (int q = lane; q < kTable; q += 32) { key[q] = -1; cnt[q] = 0; }
  __syncwarp();
  bool overflow = false;
  for (int64_t p = rb + lane; p < re; p += 32) {
    const uint2 e = g.nadj[p];
    const int x = entry_omega(e.y, A);
    const int s = min(ent_size(e) - x, g.theta + 1);
    const int k = (x << 8) | s;
    unsigned h = ((unsigned)k * 2654435761u) >> 24;   // 8 bits
    int probes = 0;
    while (true) {
      const int old = atomicCAS(&key[h], -1, k);
      if (old == -1 || old == k) { atomicAdd(&cnt[h], 1); break; }
      h = (h + 1) & (kTable - 1);
      if (++probes >= kTable) { overflow = true; break; }
    }
  }
  overflow = __any_sync(0xffffffffu, overflow);
  __syncwarp();
  if (overflow) {
    // more distinct classes than the table holds: enumerate the pairs
    for (int64_t p = rb; p < re; ++p) {
      const uint2 ep = g.nadj[p];
      const int x1 = entry_omega(ep.y, A);
      for (int64_t q = p + 1 + lane; q < re; q += 32) {
        const uint2 eq = g.nadj[q];
        const int x2 = entry_omega(eq.y, A);
        if (x1 + x2 > A) continue;
        hadd(hist, lut[ternary_code(A, ent_size(ep), ent_size(eq), x1, 0, x2, 0, g.theta)], 1);
      }
    }
    __syncwarp();
    return;
  }
  // compact the used slots to the front, in place (each lane first reads
  // its kPer consecutive slots)
  int32_t rk[kPer], rc[kPer];
  int mine = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    rk[q] = key[lane * kPer + q];
    rc[q] = cnt[lane * kPer + q];
    mine += rk[q] != -1 ? 1 : 0;
  }
  int incl = mine;
  for (int d = 1; d < 32; d <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  const int P = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  int pos = incl - mine;
#pragma unroll
  for (int q = 0; q < kPer; ++q)
    if (rk[q] != -1) { key[pos] = rk[q]; cnt[pos] = rc[q]; ++pos; }
  __syncwarp();
  for (int i = lane; i < P; i += 32) {
    const int x1 = key[i] >> 8, s1 = key[i] & 255;
    const long long n1 = cnt[i];
    for (int j = i; j < P; ++j) {
      const int x2 = key[j] >> 8, s2 = key[j] & 255;
      if (x1 + x2 > A) continue;
      const long long n2 = cnt[j];
      const long long n = i == j ? n1 * (n1 - 1) / 2 : n1 * n2;
      if (n) hadd(hist, lut[ternary_code(A, x1 + s1, x2 + s2, x1, 0, x2, 0, g.theta)], n);
    }
  }
  __syncwarp();
}

// One warp per centre row.  For a batch (kSeg) the block takes 8 consecutive
// centres at a time and counts into the shared histogram of the unit of the
// first; a centre of another unit (at a unit boundary) adds to its unit's
// global histogram directly.
template <bool kSeg>
__global__ void __launch_bounds__(kOpenThreads) k_open_pairs(SplitArgs g) {
  __shared__ unsigned long long hist[432];
  __shared__ uint16_t lut[2192];
  __shared__ int32_t tkey[kOpenWarps][kTable];
  __shared__ int32_t tcnt[kOpenWarps][kTable];
  load_lut(lut, g.lut3, hist);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  int32_t* key = tkey[warp];
  int32_t* cnt = tcnt[warp];
  const int64_t nw = (int64_t)gridDim.x * kOpenWarps;
  if (!kSeg) {
    const int64_t nc = g.centres ? g.n_centres : g.n_edges;
    for (int64_t q = (int64_t)blockIdx.x * kOpenWarps + warp; q < nc; q += nw)
      open_centre(g, g.centres ? (int64_t)g.centres[q] : q, hist, lut, key, cnt);
    __syncthreads();
    flush_hist(g.hist, hist);
    return;
  }
  int cur = 0;
  for (int64_t c0 = (int64_t)blockIdx.x * kOpenWarps; c0 < g.n_edges; c0 += nw) {
    __syncthreads();
    switch_unit(hist, g.hist, cur, unit_of_edge(g, c0));
    const int64_t c = c0 + warp;
    if (c < g.n_edges) {
      const int u = unit_of_edge(g, c);
      open_centre(g, c, u == cur ? hist : g.hist + (int64_t)u * 432, lut, key, cnt);
    }
  }
  __syncthreads();
  flush_hist(g.hist + (int64_t)cur * 432, hist);
}

// ---------------------------------------------------------------------------
// Triangles with three dense rows: CTA per dense row a, warp per hyperwedge
// (a, b).  Every dense row keeps its overlaps with the other dense rows of
// its hypergraph as bit-planes over the dense index, interleaved so that a
// word of the row is one 16-byte load: bits 0, 1, 2 of min(omega, 7) and the
// mask of adjacent candidates, 32 candidates per word (the four size planes
// are interleaved the same way).  For a candidate e_k
// adjacent to both e_a and e_b, with xa, xb, xt the numbers of nodes of
// e_a \ e_b, e_b \ e_a and e_a & e_b that e_k holds,
//   omega_ak = xa + xt,  omega_bk = xb + xt,
// so only xt = |e_a & e_b & e_k| is counted in the word loop, bit-sliced
// (3 bits and an overflow flag) from the bitmaps of the nodes of e_a & e_b
// ("heavy" nodes) or their short lists of dense hyperedges ("light" ones).
// The usual combinations (xa, xb, xt) are counted by popcount per size bin;
// any other goes to a per-warp table keyed by (xa, xb, xt, effective size),
// each such candidate classified by the lane whose word holds it (large
// windows, where they are rare) or spread over the warp 32 at a time; a
// candidate with an omega of 7 or more, or xt >= 8, is classified from node
// lists.
// Shared layout: hist | lut | anodes[64] | WarpScratch[kDWarps]
// ---------------------------------------------------------------------------
// 4 warps per CTA and 5 CTAs per SM (96 registers, 32 KB of shared memory
// per CTA): 20 resident warps per SM.  Measured on the medium workload: 22.8 s
// against 24.0 s for 8-warp CTAs at 2 per SM (16 warps, 125 registers) and
// 27.3 s at 3 per SM (80 registers, spilling); with later versions of the
// loop, 16.5 s against 18.2 s at 4 per SM (126 registers), and 15.8 s
// against 17.4 s at 6 per SM (80 registers, spilling)
constexpr int kDThreads = 128;
constexpr int kDWarps = kDThreads / 32;
constexpr int kCombo = 64;         // (xa, xb, xt) with each count below 4
// effective sizes per combination kept in the table, as the offset
// ce - (xa + xb + xt) (the effective size lies in [xa + xb + xt,
// xa + xb + 2 xt + theta + 1]: 6 values for theta = 1)
constexpr int kRel = 8;

constexpr int kLight = 256;        // merged light-node entries per hyperwedge (a power of two)
constexpr int kSlots = 8;          // per-warp signature slots of popcounted bins (theta = 1)
constexpr uint32_t kSlotFlush = 1024;   // hyperwedges per slot before it is flushed

struct WarpScratch {
  int64_t lpos[64];      // next unread entry of each light node's dense list
  int64_t lend[64];      // end of that list
  int32_t lnext[64];     // dense index at lpos (INT_MAX when done)
  int32_t lent[kLight];  // merged entries (dense indices), ascending
  int32_t bnodes[64];
  int32_t hidx[64];      // heavy indices of the nodes of e_a & e_b
  int32_t light[64];     // the nodes of e_a & e_b without a bitmap
  int32_t n[2];          // how many of each
  uint32_t table[kCombo * kRel];
  // theta = 1: totals of the popcounted bins summed over the row's
  // hyperwedges that share a signature (their motif codes are equal)
  uint32_t sacc[kSlots][32];
  int32_t skey[kSlots];        // signature, -1 when free
  int32_t srep[kSlots];        // a hyperwedge with that signature: x | B << 8
  uint32_t sn[kSlots];         // hyperwedges summed since the last flush
  int32_t snext;               // next slot to evict
};

// add one bit per lane to a 3-bit sliced counter (c0, c1, c2); a carry out
// of the top bit marks the lane in ovf
__device__ __forceinline__ void slice_add(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& ovf,
                                          uint32_t m) {
  const uint32_t k0 = c0 & m;
  c0 ^= m;
  const uint32_t k1 = c1 & k0;
  c1 ^= k0;
  ovf |= c2 & k1;
  c2 ^= k1;
}

__device__ __forceinline__ int sval3(uint32_t c0, uint32_t c1, uint32_t c2, int bit) {
  return (int)((c0 >> bit) & 1u) + 2 * (int)((c1 >> bit) & 1u) + 4 * (int)((c2 >> bit) & 1u);
}

// exact overlaps of e_k with e_a (z), e_b (y) and both (t)
struct Overlap {
  int z, y, t;
};

__device__ __forceinline__ Overlap overlaps(const int32_t* anodes, int A, const int32_t* bnodes,
                                            int B, const int32_t* knodes, int C) {
  Overlap o{0, 0, 0};
  for (int q = 0; q < C; ++q) {
    const int32_t u = knodes[q];
    const bool ia = has_node(anodes, A, u), ib = has_node(bnodes, B, u);
    o.z += ia; o.y += ib; o.t += ia && ib;
  }
  return o;
}

// Counting of the usual overlap combinations by popcount.  With theta = 1
// the combinations (xa, xb, xt) = (0,0,1), (0,1,1), (1,0,1), (1,1,0) are
// counted per effective size (|e_k| capped where all codes stop changing:
// 4, 5, 5 and 4); with another theta only (0,0,1) and (1,1,0) are, per size
// class.  Bit-planes p0..p3 hold min(|e_k|, 15) of the candidates.
struct SizeMasks {
  uint32_t e1, e2, e3, e4, e5, ge4, ge5, ge6;
  __device__ __forceinline__ SizeMasks(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3) {
    const uint32_t lo = ~p3 & ~p2;
    e1 = lo & ~p1 & p0;
    e2 = lo & p1 & ~p0;
    e3 = lo & p1 & p0;
    e4 = ~p3 & p2 & ~p1 & ~p0;
    e5 = ~p3 & p2 & ~p1 & p0;
    ge4 = p3 | p2;
    ge5 = ge4 & ~e4;
    ge6 = ge5 & ~e5;
  }
};

// Popcounted combinations for theta = 1: (xa, xb, xt), smallest possible
// effective size, number of size bins (the last bin holds every size from
// the bound xa + xb + 2 xt + 2 up, where the codes stop changing).
__constant__ int c_pop[7][5] = {
    {0, 0, 1, 1, 4}, {0, 1, 1, 2, 4}, {1, 0, 1, 2, 4}, {1, 1, 0, 2, 3},
    {0, 2, 1, 3, 4}, {1, 1, 1, 3, 4}, {0, 0, 2, 2, 5}};
constexpr int kPopBins = 28;   // total bins, counted two per register

// Signature of hyperwedge (a, b) for theta = 1: with A = |e_a| fixed, the
// motif code of every popcounted bin and its three "as if open" codes depend
// on omega_ab = x and B = |e_b| only through min(x, 4), min(A - x, 4),
// min(B - x, 5) and min(B, 5).  The bins have xa <= 1, xb <= 2, xt <= 2
// (so z = xa + xt <= 2 and y = xb + xt <= 3), and the regions that involve x
// or B are x - xt, A - x - xa, B - x - xb (closed code), A - x - z, B - x
// and x (centre a), B - x - y, A - x (centre b), B - y (centre k): each is
// exact below its cap and at least 2 (the top state) at or above it, and so
// are the validity tests x + z <= A and x + y <= B.
__device__ __forceinline__ int pop_signature(int A, int x, int B) {
  return min(x, 4) + 5 * min(A - x, 4) + 25 * min(B - x, 5) + 150 * min(B, 5);
}

// Adds slot `q` of the warp's signature slots to the histogram, as the
// closed instances of its representative hyperwedge, and frees it.
template <typename WS>
__device__ __forceinline__ void flush_slot(WS& me, int q, unsigned long long* hist,
                                           const uint16_t* lut, int A) {
  const int lane = threadIdx.x & 31;
  const uint32_t v = me.sacc[q][lane];
  if (v && lane < kPopBins) {
    const int r = me.srep[q];
    const int x = r & 255, B = r >> 8;
    int s2 = 0, base = 0;
    while (base + c_pop[s2][4] <= lane) { base += c_pop[s2][4]; ++s2; }
    const int xa = c_pop[s2][0], xb = c_pop[s2][1], xt = c_pop[s2][2];
    const int ce = c_pop[s2][3] + (lane - base);
    add_triangle(hist, lut, 1, A, B, ce, x, xb + xt, xa + xt, xt, (long long)v);
  }
  me.sacc[q][lane] = 0u;
  __syncwarp();
  if (lane == 0) {
    me.skey[q] = -1;
    me.sn[q] = 0u;
  }
  __syncwarp();
}

// Candidates of word w (bits of e) whose overlap with e_a or e_b is 7 or
// more, or whose triple intersection is 8 or more: classified from node
// lists (e_b's read here).  Kept out of line: rare, and the word loop stays
// small.  Called by the whole warp.
__device__ __noinline__ void exact_candidates(const SplitArgs& g, uint32_t e, int64_t w,
                                              const int32_t* anodes, int A, int32_t* bnodes,
                                              int64_t b, int B, int x, unsigned long long* hist,
                                              const uint16_t* lut, int theta) {
  const int lane = threadIdx.x & 31;
  if (lane < B) bnodes[lane] = g.enode[g.eoff[b] + lane];
  if (lane + 32 < B) bnodes[lane + 32] = g.enode[g.eoff[b] + lane + 32];
  __syncwarp();
  while (__any_sync(0xffffffffu, e != 0u)) {
    if (!e) continue;
    const int bit = __ffs(e) - 1;
    e &= e - 1;
    const int64_t k = g.dense_row[w * 32 + bit];
    const int64_t kb = g.eoff[k];
    const int C = (int)(g.eoff[k + 1] - kb);
    const Overlap o = overlaps(anodes, A, bnodes, B, g.enode + kb, C);
    add_triangle(hist, lut, theta, A, B, C, x, o.y, o.z, o.t, 1);
  }
}

template <bool kTheta1, bool kSeg, bool kStats, bool kLaneRest>
__global__ void __launch_bounds__(kDThreads, 5) k_dense_triangles(SplitArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hist = (unsigned long long*)smem;
  uint16_t* lut = (uint16_t*)(hist + 432);
  int32_t* anodes = (int32_t*)(lut + 2192);
  WarpScratch* ws = (WarpScratch*)(anodes + 64);
  const int64_t W = g.wwords;
  __shared__ int64_t slot_s;
  __shared__ int64_t row_next;
  __shared__ int unit_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpScratch& me = ws[warp];
  int cur = 0;   // unit whose counts the shared histogram holds (kSeg)
  load_lut(lut, g.lut3, hist);
  for (int q = lane; q < kCombo * kRel; q += 32) me.table[q] = 0u;
  for (int q = 0; q < kSlots; ++q) me.sacc[q][lane] = 0u;
  if (lane < kSlots) {
    me.skey[lane] = -1;
    me.sn[lane] = 0u;
  }
  if (lane == 0) me.snext = 0;
  __syncwarp();
  const int theta = g.theta;
  const uint4* PS = (const uint4*)g.sbits;   // size planes, four words per word
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      slot_s = atomicAdd(g.queue, 1);
      if (kSeg && slot_s < g.n_order) unit_s = unit_of_edge(g, g.order[slot_s]);
    }
    __syncthreads();
    const int64_t slot = slot_s;
    if (slot >= g.n_order) break;
    // the window of dense words of this row's hypergraph (all of them when
    // there is one); omega planes are indexed by word - WLO
    int64_t WLO = 0, WHI = W, WN = W, hbase = 0, dboff = 0, dbase = 0;
    const uint32_t* NB = g.nbits;
    if (kSeg) {
      switch_unit(hist, g.hist, cur, unit_s);
      const SegInfo sg = g.seg[cur];
      WLO = sg.wlo;
      WN = sg.wn;
      WHI = sg.wlo + sg.wn;
      hbase = sg.hbase;
      dboff = sg.dboff;
      dbase = sg.dbase;
      NB = g.nbits + sg.nboff;
    }
    const int64_t a = g.order[slot];
    const int ad = g.dense_idx[a];
    const int64_t rb = g.noff[a], re = g.noff[a + 1];
    const int A = (int)(g.eoff[a + 1] - g.eoff[a]);
    if (threadIdx.x < A) anodes[threadIdx.x] = g.enode[g.eoff[a] + threadIdx.x];
    if (kStats && threadIdx.x == 0) atomicAdd(&g.stats[82], 1ull);
    // omega planes of row a (bits 0, 1, 2 of min(omega, 7)), indexed by word - WLO
    const uint4* AR = (const uint4*)(g.dbits + dboff + (int64_t)(ad - dbase) * 4 * WN);
    if (threadIdx.x == 0) row_next = rb;
    __syncthreads();
    while (true) {
      int64_t idx = 0;
      if (lane == 0) idx = atomicAdd((unsigned long long*)&row_next, 1ull);
      idx = __shfl_sync(0xffffffffu, idx, 0);
      if (idx >= re) break;
      const uint2 eab = g.nadj[idx];
      const int64_t b = ent_id(eab);
      const int bd = g.dense_idx[b];
      if (bd <= ad) continue;                       // b must be dense and after a
      const long long t_setup0 = kStats ? clock64() : 0;
      const int B = ent_size(eab);
      const int x = entry_omega(eab.y, A);
      if (A > kMaskedMax) {
        // a wide row's entries hold omega, not node masks: e_b's nodes are
        // needed for the membership tests below
        if (lane < B) me.bnodes[lane] = g.enode[g.eoff[b] + lane];
        if (lane + 32 < B) me.bnodes[lane + 32] = g.enode[g.eoff[b] + lane + 32];
      }
      if (lane < 2) me.n[lane] = 0;
      __syncwarp();
      // the nodes of e_a & e_b (group T): with a bitmap ("heavy") or a short
      // list of dense hyperedges ("light"); for |e_a| <= 32 the entry (a, b)
      // marks them (bit p: the p-th node of e_a lies in e_b)
      for (int base = 0; base < A; base += 32) {
        const int l = base + lane;
        const int32_t u = l < A ? anodes[l] : -1;
        const bool inT = l < A && (A <= kMaskedMax ? ((eab.y >> l) & 1u) != 0u
                                                   : has_node(me.bnodes, B, u));
        const int hv = inT ? g.heavy_idx[u] : -1;
        const bool hvy = inT && hv >= 0, lt = inT && hv < 0;
        const unsigned bh = __ballot_sync(0xffffffffu, hvy);
        const unsigned bl = __ballot_sync(0xffffffffu, lt);
        const int nh0 = me.n[0], nl0 = me.n[1];
        if (hvy) me.hidx[nh0 + __popc(bh & ((1u << lane) - 1u))] = hv - (int)hbase;
        if (lt) me.light[nl0 + __popc(bl & ((1u << lane) - 1u))] = u;
        __syncwarp();
        if (lane == 0) {
          me.n[0] = nh0 + __popc(bh);
          me.n[1] = nl0 + __popc(bl);
        }
        __syncwarp();
      }
      const int nT = me.n[0], nL = me.n[1];
      const uint4* BR = (const uint4*)(g.dbits + dboff + (int64_t)(bd - dbase) * 4 * WN);
      // per-lane counters: 14 pairs of 16-bit bins (theta = 1) or 10 bins
      uint32_t cnt[14];
#pragma unroll
      for (int c = 0; c < 14; ++c) cnt[c] = 0u;
      unsigned long long st_cand = 0, st_table = 0, st_exact = 0;
      const int64_t first = (int64_t)(bd + 1);
      const int64_t fw = first >> 5;
      const long long t_groups = kStats ? clock64() : 0;
      // light T nodes: their dense lists (fewer than 32 entries each) from
      // `first` on, merged into one ascending list when they fit, else read
      // through one cursor per node
      int n_lent = 0;
      for (int l = 0; l < nL; ++l) {
        const int32_t v = me.light[l];
        const int64_t lb = g.dvoff[v], le = g.dvoff[v + 1];
        const int32_t e = lb + lane < le ? g.dvedge[lb + lane] : 0x7fffffff;
        const int before = __popc(__ballot_sync(0xffffffffu, e < first));
        const int32_t nx = __shfl_sync(0xffffffffu, e, before & 31);
        if (lane == 0) {
          me.lpos[l] = lb + before;
          me.lend[l] = le;
          me.lnext[l] = lb + before < le ? nx : 0x7fffffff;
        }
        const bool keep = e != 0x7fffffff && e >= first;
        const unsigned kb = __ballot_sync(0xffffffffu, keep);
        if (keep && n_lent + __popc(kb) <= kLight)
          me.lent[n_lent + __popc(kb & ((1u << lane) - 1u))] = e;
        n_lent += __popc(kb);
      }
      const bool merged = n_lent <= kLight;
      const long long t_light = kStats ? clock64() : 0;
      if (merged && n_lent > 1) {
        // bitonic sort of the merged entries (padded to a power of two)
        int np = 2;
        while (np < n_lent) np <<= 1;
        for (int q = n_lent + lane; q < np; q += 32) me.lent[q] = 0x7fffffff;
        __syncwarp();
        for (int k = 2; k <= np; k <<= 1)
          for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < np; i += 32) {
              const int ixj = i ^ j;
              if (ixj > i) {
                const int32_t u = me.lent[i], v2 = me.lent[ixj];
                const bool up = (i & k) == 0;
                if ((u > v2) == up) { me.lent[i] = v2; me.lent[ixj] = u; }
              }
            }
            __syncwarp();
          }
      }
      __syncwarp();
      int lcur = 0;   // next merged entry
      long long t_words0 = kStats ? clock64() : 0;
      // uniform loop: every lane runs every iteration (lanes past the end see
      // an empty word), so the warp stays converged
      // the overlap planes of the 32 candidates of word w (omega_ak, omega_bk)
      // and their size planes are loaded one iteration ahead, so that a
      // warp has the next chunk's loads in flight while it works on this one
      // (and the bitmap word of the first heavy node of e_a & e_b, if any)
      // The word loop, compiled twice: for the common hyperwedge whose
      // e_a & e_b is one node with a bitmap (no other heavy node, no light
      // node) and for any other; the first leaves out the bit-sliced sum over
      // several T nodes and the merge of light lists, so its loop is shorter.
      uint32_t dmask = 0u;   // groups of 32 table entries this lane touched
      auto word_loop = [&](auto simple) {
        constexpr bool kSimple = decltype(simple)::value;
      const uint32_t* T0 = NB + (nT > 0 ? (int64_t)me.hidx[0] * WN : 0);
      // word indices fit in 32 bits (at most 2^21 words)
      const int iWHI = (int)WHI, iWLO = (int)WLO, ifw = (int)fw;
      uint4 nqa = make_uint4(0u, 0u, 0u, 0u), nqb = nqa, np = nqa;
      uint32_t nt = 0;
      if (ifw < iWHI) {
        const int w = ifw + lane < iWHI ? ifw + lane : iWHI - 1;
        const int wl = w - iWLO;
        nqa = __ldg(&AR[wl]);
        nqb = __ldg(&BR[wl]);
        np = __ldg(&PS[w]);
        if (nT > 0) nt = __ldg(&T0[wl]);
      }
      for (int w0 = ifw; w0 < iWHI; w0 += 32) {
        const bool inr = w0 + lane < iWHI;
        const int w = inr ? w0 + lane : iWHI - 1;
        const int wl = w - iWLO;
        const uint32_t qa0 = nqa.x, qa1 = nqa.y, qa2 = nqa.z, qb0 = nqb.x, qb1 = nqb.y, qb2 = nqb.z;
        const uint32_t anya = nqa.w, anyb = nqb.w;
        const uint32_t p0 = np.x, p1 = np.y, p2 = np.z, p3 = np.w, tb = nt;
        {
          const int w1 = w0 + 32 + lane < iWHI ? w0 + 32 + lane : iWHI - 1;
          const int wl1 = w1 - iWLO;
          nqa = __ldg(&AR[wl1]);
          nqb = __ldg(&BR[wl1]);
          np = __ldg(&PS[w1]);
          if (nT > 0) nt = __ldg(&T0[wl1]);
        }
        uint32_t m = inr ? (anya & anyb) : 0u;
        if (w == ifw) m &= 0xffffffffu << (first & 31);
        // xt = |e_a & e_b & e_k|, bit-sliced (3 bits and an overflow flag)
        uint32_t t0 = tb, t1 = 0, t2 = 0, ovf = 0;   // tb: the first heavy node's word
        if constexpr (!kSimple) {
          for (int h = 1; h < nT; ++h)
            slice_add(t0, t1, t2, ovf, __ldg(&NB[(int64_t)me.hidx[h] * WN + wl]));
        }
        if constexpr (!kSimple) {
        // light T nodes with a dense index in this iteration's 32 words
        const int64_t hi64 = (int64_t)(w0 + 32) * 32;
        const int32_t hi = hi64 < 0x7fffffff ? (int32_t)hi64 : 0x7fffffff;
        if (merged) {
          while (lcur < n_lent) {
            const int32_t e = lcur + lane < n_lent ? me.lent[lcur + lane] : 0x7fffffff;
            const int nin = __popc(__ballot_sync(0xffffffffu, e < hi && e != 0x7fffffff));
            for (int j = 0; j < nin; ++j) {
              const int32_t kd = __shfl_sync(0xffffffffu, e, j);
              if ((kd >> 5) == w && inr) slice_add(t0, t1, t2, ovf, 1u << (kd & 31));
            }
            lcur += nin;
            if (nin < 32) break;
          }
        } else {
          for (int l = 0; l < nL; ++l) {
            if (me.lnext[l] >= hi) continue;              // uniform: same value on all lanes
            const int64_t pos = me.lpos[l], le = me.lend[l];
            const int32_t e = pos + lane < le ? g.dvedge[pos + lane] : 0x7fffffff;
            const int nin = __popc(__ballot_sync(0xffffffffu, e < hi));
            for (int j = 0; j < nin; ++j) {
              const int32_t kd = __shfl_sync(0xffffffffu, e, j);
              if ((kd >> 5) == w && inr) slice_add(t0, t1, t2, ovf, 1u << (kd & 31));
            }
            const int32_t nx = __shfl_sync(0xffffffffu, e, nin & 31);
            __syncwarp();
            if (lane == 0) {
              me.lpos[l] = pos + nin;
              me.lnext[l] = pos + nin < le ? nx : 0x7fffffff;
            }
            __syncwarp();
          }
        }
        }
        // omega >= 7 or xt >= 8: classified from node lists below
        ovf = (ovf | (qa0 & qa1 & qa2) | (qb0 & qb1 & qb2)) & m;
        const uint32_t valid = m & ~ovf;
        // omega = 1, 2, 3 on valid bits
        const uint32_t a1m = qa0 & ~qa1 & ~qa2, a2m = ~qa0 & qa1 & ~qa2;
        const uint32_t b1m = qb0 & ~qb1 & ~qb2, b2m = ~qb0 & qb1 & ~qb2, b3m = qb0 & qb1 & ~qb2;
        const uint32_t zt = t0 | t1 | t2;
        const uint32_t one_t = t0 & ~t1 & ~t2;
        // (xa, xb, xt) = (omega_ak - xt, omega_bk - xt, xt)
        const uint32_t s001 = valid & a1m & b1m & one_t;
        const uint32_t s110 = valid & a1m & b1m & ~zt;
        uint32_t done = s001 | s110;
        const SizeMasks sz(p0, p1, p2, p3);
        if (kTheta1) {
          const uint32_t two_t = ~t0 & t1 & ~t2;
          const uint32_t s011 = valid & a1m & b2m & one_t;
          const uint32_t s101 = valid & a2m & b1m & one_t;
          const uint32_t s021 = valid & a1m & b3m & one_t;
          const uint32_t s111 = valid & a2m & b2m & one_t;
          const uint32_t s002 = valid & a2m & b2m & two_t;
          done |= s011 | s101 | s021 | s111 | s002;
          // bins: (0,0,1) 1,2,3,4+ | (0,1,1) 2,3,4,5+ | (1,0,1) 2,3,4,5+ |
          // (1,1,0) 2,3,4+ | (0,2,1) 3,4,5,6+ | (1,1,1) 3,4,5,6+ | (0,0,2) 2,3,4,5,6+
          cnt[0] += __popc(s001 & sz.e1) | (__popc(s001 & sz.e2) << 16);
          cnt[1] += __popc(s001 & sz.e3) | (__popc(s001 & sz.ge4) << 16);
          cnt[2] += __popc(s011 & sz.e2) | (__popc(s011 & sz.e3) << 16);
          cnt[3] += __popc(s011 & sz.e4) | (__popc(s011 & sz.ge5) << 16);
          cnt[4] += __popc(s101 & sz.e2) | (__popc(s101 & sz.e3) << 16);
          cnt[5] += __popc(s101 & sz.e4) | (__popc(s101 & sz.ge5) << 16);
          cnt[6] += __popc(s110 & sz.e2) | (__popc(s110 & sz.e3) << 16);
          cnt[7] += __popc(s110 & sz.ge4) | (__popc(s021 & sz.e3) << 16);
          cnt[8] += __popc(s021 & sz.e4) | (__popc(s021 & sz.e5) << 16);
          cnt[9] += __popc(s021 & sz.ge6) | (__popc(s111 & sz.e3) << 16);
          cnt[10] += __popc(s111 & sz.e4) | (__popc(s111 & sz.e5) << 16);
          cnt[11] += __popc(s111 & sz.ge6) | (__popc(s002 & sz.e2) << 16);
          cnt[12] += __popc(s002 & sz.e3) | (__popc(s002 & sz.e4) << 16);
          cnt[13] += __popc(s002 & sz.e5) | (__popc(s002 & sz.ge6) << 16);
        } else {
#pragma unroll
          for (int c = 0; c < kClasses; ++c) {
            const uint32_t sc = __ldg(&g.cbits[(int64_t)c * W + w]);
            cnt[c] += __popc(s001 & sc);
            cnt[5 + c] += __popc(s110 & sc);
          }
        }
        if (kStats) {
          st_cand += __popc(m);
          st_table += __popc(valid & ~done);
          st_exact += __popc(ovf);
        }
        // remaining candidates, classified into the table (or straight into
        // the histogram when the combination or the offset is outside it)
        auto classify_rest = [&](uint32_t ra0, uint32_t ra1, uint32_t ra2, uint32_t rb0,
                                 uint32_t rb1, uint32_t rb2, uint32_t rt0, uint32_t rt1,
                                 uint32_t rt2, uint32_t rp0, uint32_t rp1, uint32_t rp2,
                                 uint32_t rp3, int rw, int bit) {
          const int xt = sval3(rt0, rt1, rt2, bit);
          const int xa = sval3(ra0, ra1, ra2, bit) - xt;
          const int xb = sval3(rb0, rb1, rb2, bit) - xt;
          int C = (int)((rp0 >> bit) & 1u) | ((int)((rp1 >> bit) & 1u) << 1) |
                  ((int)((rp2 >> bit) & 1u) << 2) | ((int)((rp3 >> bit) & 1u) << 3);
          if (C >= 15) C = g.dsize[(int64_t)rw * 32 + bit];
          const int ce = min(C, xa + xb + 2 * xt + theta + 1);
          const int rel = ce - (xa + xb + xt);
          if (xa < 4 && xb < 4 && xt < 4 && rel >= 0 && rel < kRel) {
            const int key = ((xa * 4 + xb) * 4 + xt) * kRel + rel;
            atomicAdd(&me.table[key], 1u);
            dmask |= 1u << (key >> 5);
            if (kStats) atomicAdd(&g.stats[8 + key / kRel], 1ull);
          } else {
            add_triangle(hist, lut, theta, A, B, ce, x, xb + xt, xa + xt, xt, 1);
          }
        };
        uint32_t rest = valid & ~done;
        if constexpr (kLaneRest) {
          // few per word (a large hypergraph): each lane takes the remaining
          // candidates of its own word, one at a time
          if (rest) {
            do {
              const int bit = __ffs(rest) - 1;
              rest &= rest - 1u;
              classify_rest(qa0, qa1, qa2, qb0, qb1, qb2, t0, t1, t2, p0, p1, p2, p3, w, bit);
            } while (rest);
          }
        } else {
          // more per word: spread over the warp, 32 per round (lane l takes
          // the l-th remaining candidate of the iteration and reads its
          // word's planes by shuffle)
          if (__any_sync(0xffffffffu, rest != 0u)) {
            const int rc = __popc(rest);
            int incl = rc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
              const int o = __shfl_up_sync(0xffffffffu, incl, d);
              if (lane >= d) incl += o;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int base = 0; base < total; base += 32) {
              const int item = base + lane;
              // source lane: the first lane whose inclusive count exceeds item
              int src = 0;
#pragma unroll
              for (int st = 16; st; st >>= 1) {
                const int probe = __shfl_sync(0xffffffffu, incl, src + st - 1);
                if (probe <= item) src += st;
              }
              src &= 31;
              const int ex = __shfl_sync(0xffffffffu, incl - rc, src);
              uint32_t rs = __shfl_sync(0xffffffffu, rest, src);
              const uint32_t sa0 = __shfl_sync(0xffffffffu, qa0, src), sa1 = __shfl_sync(0xffffffffu, qa1, src),
                             sa2 = __shfl_sync(0xffffffffu, qa2, src);
              const uint32_t sb0 = __shfl_sync(0xffffffffu, qb0, src), sb1 = __shfl_sync(0xffffffffu, qb1, src),
                             sb2 = __shfl_sync(0xffffffffu, qb2, src);
              const uint32_t st0 = __shfl_sync(0xffffffffu, t0, src), st1 = __shfl_sync(0xffffffffu, t1, src),
                             st2 = __shfl_sync(0xffffffffu, t2, src);
              const uint32_t sp0 = __shfl_sync(0xffffffffu, p0, src), sp1 = __shfl_sync(0xffffffffu, p1, src),
                             sp2 = __shfl_sync(0xffffffffu, p2, src), sp3 = __shfl_sync(0xffffffffu, p3, src);
              const int sw = __shfl_sync(0xffffffffu, w, src);
              if (item < total) {
                for (int k = item - ex; k > 0; --k) rs &= rs - 1u;   // its (item - ex)-th bit
                classify_rest(sa0, sa1, sa2, sb0, sb1, sb2, st0, st1, st2, sp0, sp1, sp2, sp3, sw,
                              __ffs(rs) - 1);
              }
            }
          }
        }
        if (__any_sync(0xffffffffu, ovf != 0u))
          exact_candidates(g, ovf, w, anodes, A, me.bnodes, b, B, x, hist, lut, theta);
      }
      };
      if (nT == 1 && nL == 0) word_loop(std::true_type{});
      else word_loop(std::false_type{});
      long long t_words1 = kStats ? clock64() : 0;
      if (kStats) {
        for (int d = 16; d; d >>= 1) {
          st_cand += __shfl_xor_sync(0xffffffffu, st_cand, d);
          st_table += __shfl_xor_sync(0xffffffffu, st_table, d);
          st_exact += __shfl_xor_sync(0xffffffffu, st_exact, d);
        }
        if (lane == 0) {
          atomicAdd(&g.stats[0], (unsigned long long)(WHI - fw));
          atomicAdd(&g.stats[1], st_cand);
          atomicAdd(&g.stats[2], st_table);
          atomicAdd(&g.stats[3], st_exact);
        }
      }
      // flush the per-lane counters: lane c handles counter c (theta = 1:
      // counters are pairs of 16-bit bins)
      uint32_t mine = 0u;
      if (kTheta1) {
#pragma unroll
        for (int c = 0; c < 14; ++c) {
          const uint32_t lo = __reduce_add_sync(0xffffffffu, cnt[c] & 0xffffu);
          const uint32_t hi2 = __reduce_add_sync(0xffffffffu, cnt[c] >> 16);
          if (lane == 2 * c) mine = lo;
          if (lane == 2 * c + 1) mine = hi2;
        }
        // into the slot of this hyperwedge's signature (found, free, or
        // evicted round-robin)
        const int key = pop_signature(A, x, B);
        const int sk = lane < kSlots ? me.skey[lane] : -2;
        const unsigned hit = __ballot_sync(0xffffffffu, sk == key);
        int q;
        if (hit) {
          q = __ffs(hit) - 1;
        } else {
          const unsigned fr = __ballot_sync(0xffffffffu, sk == -1);
          if (fr) {
            q = __ffs(fr) - 1;
          } else {
            q = me.snext;
            __syncwarp();
            if (lane == 0) me.snext = (q + 1) % kSlots;
            if (kStats && lane == 0) atomicAdd(&g.stats[80], 1ull);
            flush_slot(me, q, hist, lut, A);
          }
          if (lane == 0) {
            me.skey[q] = key;
            me.srep[q] = x | (B << 8);
          }
        }
        if (lane < kPopBins) me.sacc[q][lane] += mine;
        __syncwarp();
        const uint32_t nq = me.sn[q] + 1u;
        __syncwarp();
        if (lane == 0) me.sn[q] = nq;
        __syncwarp();
        if (nq >= kSlotFlush) {
          if (kStats && lane == 0) atomicAdd(&g.stats[81], 1ull);
          flush_slot(me, q, hist, lut, A);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 2 * kClasses; ++c) {
          const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[c]);
          if (lane == c) mine = v;
        }
        if (mine && lane < 2 * kClasses) {
          const int C = class_rep(lane % kClasses, theta);
          add_triangle(hist, lut, theta, A, B, C, x, 1, 1, lane < kClasses ? 1 : 0, (long long)mine);
        }
      }
      __syncwarp();
      // the table entries of this hyperwedge, one group of 32 at a time
      for (uint32_t gm = __reduce_or_sync(0xffffffffu, dmask); gm; gm &= gm - 1u) {
        const int q = (__ffs(gm) - 1) * 32 + lane;
        const uint32_t n = me.table[q];
        if (n) {
          me.table[q] = 0u;
          const int combo = q / kRel, rel = q % kRel;
          const int xt = combo & 3, xb = (combo >> 2) & 3, xa = combo >> 4;
          add_key(hist, lut, theta, A, B, x, xa, xb, xt, rel, (long long)n);
        }
      }
      if (kStats && lane == 0) {
        const long long t_end = clock64();
        atomicAdd(&g.stats[5], (unsigned long long)(t_words0 - t_setup0));
        atomicAdd(&g.stats[72], (unsigned long long)(t_groups - t_setup0));
        atomicAdd(&g.stats[73], (unsigned long long)(t_light - t_groups));
        atomicAdd(&g.stats[74], (unsigned long long)(t_words0 - t_light));
        atomicAdd(&g.stats[75], (unsigned long long)n_lent);
        atomicAdd(&g.stats[76], 1ull);
        atomicAdd(&g.stats[77], (unsigned long long)nL);
        atomicAdd(&g.stats[78], (unsigned long long)nT);
        atomicAdd(&g.stats[6], (unsigned long long)(t_words1 - t_words0));
        atomicAdd(&g.stats[7], (unsigned long long)(t_end - t_words1));
      }
      __syncwarp();
    }
    // the row is done for this warp: its signature slots go to the histogram
    // (their codes depend on |e_a|)
    if (kTheta1) {
      for (int q = 0; q < kSlots; ++q)
        if (me.skey[q] >= 0) flush_slot(me, q, hist, lut, A);
    }
  }
  __syncthreads();
  flush_hist(g.hist + (int64_t)cur * 432, hist);
}

// ---------------------------------------------------------------------------
// Triangles whose smallest member (sparse rows first) is a sparse row a:
// CTA per sparse row; the row is staged in shared memory.
// Shared layout: hist | lut | anodes[64] | per-warp bnodes[64] |
// key[D] | w1[D] | size[D] | didx[D]
// ---------------------------------------------------------------------------
template <bool kSeg>
__global__ void __launch_bounds__(kThreads) k_sparse_triangles(SplitArgs g, int max_deg) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hist = (unsigned long long*)smem;
  uint16_t* lut = (uint16_t*)(hist + 432);
  int32_t* anodes = (int32_t*)(lut + 2192);
  int32_t* bnodes_all = anodes + 64;
  uint32_t* skey = (uint32_t*)(bnodes_all + 64 * kWarps);
  uint32_t* sw1 = skey + max_deg;
  int32_t* sdi = (int32_t*)(sw1 + max_deg);
  uint8_t* ssz = (uint8_t*)(sdi + max_deg);
  __shared__ int64_t slot_s;
  __shared__ int unit_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t* bnodes = bnodes_all + 64 * warp;
  const int64_t W = g.wwords;
  int cur = 0;   // unit whose counts the shared histogram holds (kSeg)
  load_lut(lut, g.lut3, hist);
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      slot_s = atomicAdd(g.queue, 1);
      if (kSeg && slot_s < g.n_order) unit_s = unit_of_edge(g, g.order[slot_s]);
    }
    __syncthreads();
    const int64_t slot = slot_s;
    if (slot >= g.n_order) break;
    int64_t WLO = 0, WN = W, dboff = 0, dbase = 0;
    if (kSeg) {
      switch_unit(hist, g.hist, cur, unit_s);
      const SegInfo sg = g.seg[cur];
      WLO = sg.wlo;
      WN = sg.wn;
      dboff = sg.dboff;
      dbase = sg.dbase;
    }
    const int64_t a = g.order[slot];
    const int64_t rb = g.noff[a], re = g.noff[a + 1];
    const int deg = (int)(re - rb);
    if (deg < 2) continue;
    const int A = (int)(g.eoff[a + 1] - g.eoff[a]);
    if (threadIdx.x < A) anodes[threadIdx.x] = g.enode[g.eoff[a] + threadIdx.x];
    for (int q = threadIdx.x; q < deg; q += kThreads) {
      const uint2 e = g.nadj[rb + q];
      skey[q] = ent_id(e);
      sw1[q] = e.y;
      ssz[q] = (uint8_t)ent_size(e);
      sdi[q] = g.dense_idx[ent_id(e)];
    }
    __syncthreads();
    for (int ib = warp; ib < deg; ib += kWarps) {
      const int64_t b = skey[ib];
      const int bd = sdi[ib];
      if (bd < 0 && b < a) continue;                 // b must come after a
      const int B = ssz[ib];
      const uint32_t mab = sw1[ib];
      const int x = entry_omega(mab, A);
      if (lane < B) bnodes[lane] = g.enode[g.eoff[b] + lane];
      if (B > 32 && lane + 32 < B) bnodes[lane + 32] = g.enode[g.eoff[b] + lane + 32];
      __syncwarp();
      if (bd >= 0) {
        // b dense: every k after b is dense with a larger dense index
        // omega planes of row b: omega_bk = bit0 + 2 bit1 + 4 bit2 (7: 7 or more)
        const uint4* Q = (const uint4*)(g.dbits + dboff + (int64_t)(bd - dbase) * 4 * WN);
        for (int q = lane; q < deg; q += 32) {
          const int kd = sdi[q];
          if (kd <= bd) continue;
          const uint32_t bit = 1u << (kd & 31);
          const int64_t wq = (kd >> 5) - WLO;
          const uint4 qw = __ldg(&Q[wq]);
          const uint32_t q0 = qw.x & bit, q1 = qw.y & bit, q2 = qw.z & bit;
          if (!(q0 | q1 | q2)) continue;
          const int64_t k = skey[q];
          const int C = ssz[q];
          int y = (q0 ? 1 : 0) + (q1 ? 2 : 0) + (q2 ? 4 : 0);
          if (y == 7) y = sorted_overlap(bnodes, B, g.enode + g.eoff[k], C);
          const int z = entry_omega(sw1[q], A);
          int t;
          if (A <= kMaskedMax) {
            t = __popc(mab & sw1[q]);
          } else {
            t = sorted_overlap3(anodes, A, bnodes, B, g.enode + g.eoff[k], C);
          }
          add_triangle(hist, lut, g.theta, A, B, C, x, y, z, t, 1);
        }
      } else {
        // b sparse: k in both rows and after b (dense, or sparse with k > b)
        const int64_t bb = g.noff[b], be = g.noff[b + 1];
        for (int64_t p = bb + lane; p < be; p += 32) {
          const uint2 ebk = g.nadj[p];
          const int64_t k = ent_id(ebk);
          if (k == a) continue;
          int lo = 0, hi = deg;
          while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if ((int64_t)skey[m] < k) lo = m + 1; else hi = m;
          }
          if (lo >= deg || (int64_t)skey[lo] != k) continue;
          if (sdi[lo] < 0 && k < b) continue;
          const int C = ent_size(ebk);
          const int y = entry_omega(ebk.y, B);
          const int z = entry_omega(sw1[lo], A);
          int t;
          if (A <= kMaskedMax) {
            t = __popc(mab & sw1[lo]);
          } else {
            t = sorted_overlap3(anodes, A, bnodes, B, g.enode + g.eoff[k], C);
          }
          add_triangle(hist, lut, g.theta, A, B, C, x, y, z, t, 1);
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  flush_hist(g.hist + (int64_t)cur * 432, hist);
}

// ---------------------------------------------------------------------------
// Preparation kernels.
// ---------------------------------------------------------------------------
__global__ void k_dense_flags(int64_t E, const int64_t* __restrict__ noff, int32_t thr,
                              int64_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E) flag[i] = (noff[i + 1] - noff[i]) >= thr ? 1 : 0;
  if (i == E) flag[i] = 0;
}

__global__ void k_dense_index(int64_t E, const int64_t* __restrict__ flag,
                              const int64_t* __restrict__ pos, int32_t* __restrict__ didx,
                              int32_t* __restrict__ drow) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  if (flag[i]) {
    didx[i] = (int32_t)pos[i];
    drow[pos[i]] = (int32_t)i;
  } else {
    didx[i] = -1;
  }
}

__global__ void k_dense_keys(int64_t n_dense, const int32_t* __restrict__ drow,
                             const int64_t* __restrict__ noff, uint32_t* __restrict__ key) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_dense) key[r] = (uint32_t)(noff[drow[r] + 1] - noff[drow[r]]);
}

__global__ void k_dense_reindex(int64_t n_dense, const int32_t* __restrict__ drow,
                                int32_t* __restrict__ didx) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_dense) didx[drow[r]] = (int32_t)r;
}

// unit of each dense row (rows of a batch)
__global__ void k_dense_units(int64_t n_dense, const int32_t* __restrict__ drow,
                              const int64_t* __restrict__ eoff, const int32_t* __restrict__ enode,
                              const int64_t* __restrict__ nseg, int n_units,
                              uint32_t* __restrict__ unit) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_dense) unit[r] = (uint32_t)seg_of(nseg, n_units, enode[eoff[drow[r]]]);
}

// first index of each unit in an array of units sorted ascending: out[u] =
// number of entries below u, u = 0..n_units
__global__ void k_unit_starts(int64_t n, const uint32_t* __restrict__ unit, int n_units,
                              int64_t* __restrict__ out) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u > n_units) return;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if (unit[m] < (uint32_t)u) lo = m + 1; else hi = m;
  }
  out[u] = lo;
}

__global__ void k_gather_at(int n, const int64_t* __restrict__ src, const int64_t* __restrict__ at,
                            int64_t* __restrict__ out) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) out[u] = src[at[u]];
}

__global__ void k_dense_bits(int64_t n_dense, const SegInfo* __restrict__ seg,
                             const int64_t* __restrict__ dbase, int n_units,
                             const int32_t* __restrict__ drow,
                             const int64_t* __restrict__ eoff, const int64_t* __restrict__ noff,
                             const uint2* __restrict__ nadj, const int32_t* __restrict__ didx,
                             uint32_t* __restrict__ dbits) {
  for (int64_t r = blockIdx.x; r < n_dense; r += gridDim.x) {
    const SegInfo sg = seg[seg_of(dbase, n_units, r)];
    const int64_t b = drow[r];
    const int B = (int)(eoff[b + 1] - eoff[b]);
    // word wq of the row is four words: bits 0, 1, 2 of min(omega, 7) and
    // the mask of adjacent candidates (omega >= 1)
    uint32_t* Q = dbits + sg.dboff + (r - sg.dbase) * 4 * sg.wn;
    for (int64_t p = noff[b] + threadIdx.x; p < noff[b + 1]; p += blockDim.x) {
      const uint2 e = nadj[p];
      const int kd = didx[ent_id(e)];
      if (kd < 0) continue;
      const int om = min(entry_omega(e.y, B), 7);   // 7 stands for 7 or more
      const int64_t wq = 4 * ((kd >> 5) - sg.wlo);
      const uint32_t bit = 1u << (kd & 31);
      if (om & 1) atomicOr(&Q[wq], bit);
      if (om & 2) atomicOr(&Q[wq + 1], bit);
      if (om & 4) atomicOr(&Q[wq + 2], bit);
      atomicOr(&Q[wq + 3], bit);
    }
  }
}

__global__ void k_heavy_flags(int64_t N, const int64_t* __restrict__ voff,
                              const int32_t* __restrict__ vedge, const int32_t* __restrict__ didx,
                              int32_t thr, int64_t* __restrict__ flag) {
  const int64_t v = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v > N) return;
  if (v == N) { if (lane == 0) flag[v] = 0; return; }
  int c = 0;
  for (int64_t q = voff[v] + lane; q < voff[v + 1]; q += 32) c += didx[vedge[q]] >= 0 ? 1 : 0;
  for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if (lane == 0) flag[v] = c >= thr ? 1 : 0;
}

__global__ void k_heavy_index(int64_t N, const int64_t* __restrict__ flag,
                              const int64_t* __restrict__ pos, int32_t* __restrict__ hidx) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < N) hidx[v] = flag[v] ? (int32_t)pos[v] : -1;
}

__global__ void k_heavy_bits(int64_t N, const SegInfo* __restrict__ seg,
                             const int64_t* __restrict__ nseg, int n_units,
                             const int64_t* __restrict__ voff,
                             const int32_t* __restrict__ vedge, const int32_t* __restrict__ didx,
                             const int32_t* __restrict__ hidx, uint32_t* __restrict__ nbits) {
  const int64_t v = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= N) return;
  const int h = hidx[v];
  if (h < 0) return;
  const SegInfo sg = seg[seg_of(nseg, n_units, v)];
  uint32_t* bits = nbits + sg.nboff + (h - sg.hbase) * sg.wn;
  for (int64_t q = voff[v] + lane; q < voff[v + 1]; q += 32) {
    const int kd = didx[vedge[q]];
    if (kd >= 0) atomicOr(&bits[(kd >> 5) - sg.wlo], 1u << (kd & 31));
  }
}

// dense members of each E_v, as ascending dense indices (one warp per node)
__global__ void k_dense_count(int64_t N, const int64_t* __restrict__ voff,
                              const int32_t* __restrict__ vedge, const int32_t* __restrict__ didx,
                              int64_t* __restrict__ cnt) {
  const int64_t v = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v > N) return;
  if (v == N) { if (lane == 0) cnt[v] = 0; return; }
  int c = 0;
  for (int64_t q = voff[v] + lane; q < voff[v + 1]; q += 32) c += didx[vedge[q]] >= 0 ? 1 : 0;
  for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if (lane == 0) cnt[v] = c;
}

__global__ void k_dense_fill(int64_t N, const int64_t* __restrict__ voff,
                             const int32_t* __restrict__ vedge, const int32_t* __restrict__ didx,
                             const int64_t* __restrict__ dvoff, int32_t* __restrict__ dvedge) {
  const int64_t v = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= N) return;
  int64_t o = dvoff[v];
  for (int64_t q0 = voff[v]; q0 < voff[v + 1]; q0 += 32) {
    const int64_t q = q0 + lane;
    const int kd = q < voff[v + 1] ? didx[vedge[q]] : -1;
    const unsigned bal = __ballot_sync(0xffffffffu, kd >= 0);
    if (kd >= 0) dvedge[o + __popc(bal & ((1u << lane) - 1u))] = kd;
    o += __popc(bal);
  }
}

// sort each node's dense list of fewer than 32 entries (the light nodes'
// lists, read in ascending dense index by the dense-triangle kernel)
__global__ void k_sort_short_lists(int64_t N, const int64_t* __restrict__ dvoff,
                                   int32_t* __restrict__ dvedge) {
  const int64_t v = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= N) return;
  const int64_t b = dvoff[v], e = dvoff[v + 1];
  if (e - b > 32 || e - b < 2) return;
  int32_t x = b + lane < e ? dvedge[b + lane] : 0x7fffffff;
  for (int k = 2; k <= 32; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      x = (lower == up) ? min(x, y) : max(x, y);
    }
  }
  if (b + lane < e) dvedge[b + lane] = x;
}

__global__ void k_size_bits(int64_t n_dense, int64_t W, const int32_t* __restrict__ drow,
                            const int64_t* __restrict__ eoff, int theta, uint32_t* __restrict__ sbits,
                            uint8_t* __restrict__ dsize) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_dense) return;
  const int64_t k = drow[r];
  const int C = (int)(eoff[k + 1] - eoff[k]);
  dsize[r] = (uint8_t)C;
  const int cc = min(C, 15);
  for (int b = 0; b < 4; ++b)   // word w of the size planes is four words: bits 0..3
    if (cc & (1 << b)) atomicOr(&sbits[4 * (int64_t)(r >> 5) + b], 1u << (r & 31));
  const int c = size_class(C, theta);
  atomicOr(&sbits[(int64_t)(4 + c) * W + (r >> 5)], 1u << (r & 31));
}

// stable split of row_order into dense and sparse work orders
__global__ void k_split_flags(int64_t E, const int32_t* __restrict__ order,
                              const int32_t* __restrict__ didx, int64_t* __restrict__ fd,
                              int64_t* __restrict__ fs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > E) return;
  if (i == E) { fd[i] = 0; fs[i] = 0; return; }
  const bool d = didx[order[i]] >= 0;
  fd[i] = d ? 1 : 0;
  fs[i] = d ? 0 : 1;
}

__global__ void k_split_scatter(int64_t E, const int32_t* __restrict__ order,
                                const int32_t* __restrict__ didx, const int64_t* __restrict__ pd,
                                const int64_t* __restrict__ ps, int32_t* __restrict__ dorder,
                                int32_t* __restrict__ sorder) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  const int32_t r = order[i];
  if (didx[r] >= 0) dorder[pd[i]] = r; else sorder[ps[i]] = r;
}

}  // namespace

void release_split(mochy_ctx* ctx) {
  if (!ctx->split_ready && !ctx->dense_idx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->dense_idx) dev_free(ctx, ctx->dense_idx, ctx->split_bytes);
  if (ctx->rest_block) dev_free(ctx, ctx->rest_block, ctx->rest_bytes);
  if (ctx->nbits) dev_free(ctx, ctx->nbits, ctx->nbits_bytes);
  if (ctx->dvoff) dev_free(ctx, ctx->dvoff, ctx->dinc_bytes);
  ctx->dvoff = nullptr;
  ctx->dvedge = nullptr;
  ctx->nbits_bytes = ctx->dinc_bytes = 0;
  ctx->dense_idx = nullptr;
  ctx->dense_row = nullptr;
  ctx->dbits = nullptr;
  ctx->heavy_idx = nullptr;
  ctx->nbits = nullptr;
  ctx->sbits = nullptr;
  ctx->dense_order = ctx->sparse_order = nullptr;
  ctx->dsize = nullptr;
  ctx->d_seg = nullptr;
  ctx->d_dbase = nullptr;
  ctx->rest_block = nullptr;
  ctx->split_bytes = ctx->rest_bytes = 0;
  ctx->split_ready = false;
  ctx->n_dense = ctx->n_sparse = ctx->n_heavy = ctx->wwords = ctx->wmax = 0;
}

int choose_dense_threshold(mochy_ctx* ctx);   // tune.cu

size_t dense_smem_bytes(int64_t W) {
  (void)W;   // the rows' omega planes are read from global memory
  return 432 * 8 + 2192 * 2 + 64 * 4 + sizeof(WarpScratch) * kDWarps;
}

size_t sparse_smem_bytes(int max_deg) {
  return 432 * 8 + 2192 * 2 + 64 * 4 + 64 * 4 * kWarps + (size_t)max_deg * 13 + 16;
}

int prepare_split(mochy_ctx* ctx) {
  if (ctx->split_ready) return MOCHY_OK;
  const int64_t E = ctx->n_edges, N = ctx->n_nodes;
  const int U = ctx->n_units;
  cudaStream_t st = ctx->stream;
  const int thr = ctx->dense_thr > 0 ? ctx->dense_thr : choose_dense_threshold(ctx);
  if (thr <= 0) return thr < 0 ? thr : fail(MOCHY_E_UNSUPPORTED, "no usable dense threshold");
  // dense rows
  void* t;
  MOCHY_TRY(scratch(ctx, 0, (size_t)(std::max(E, N) + 2) * 8 * 4, &t));
  int64_t* flag = (int64_t*)t;
  int64_t* pos = flag + std::max(E, N) + 2;
  int64_t* flag2 = pos + std::max(E, N) + 2;
  int64_t* pos2 = flag2 + std::max(E, N) + 2;
  k_dense_flags<<<ceil_div(E + 1, 256), 256, 0, st>>>(E, ctx->noff, thr, flag);
  MOCHY_LAUNCHED();
  MOCHY_TRY(scan_exclusive_i64(ctx, flag, pos, E + 1));
  int64_t n_dense = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&n_dense, pos + E, 8, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  const int64_t W = std::max<int64_t>((n_dense + 31) / 32, 1);   // words of the size planes
  // the dense index, dense rows and unit tables first; the bitmaps are sized
  // once the units' dense ranges are known
  const int64_t nd1 = std::max<int64_t>(n_dense, 1);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_didx = al((size_t)std::max<int64_t>(E, 1) * 4);
  const size_t b_drow = al((size_t)nd1 * 4);
  const size_t b_hidx = al((size_t)std::max<int64_t>(N, 1) * 4);
  const size_t b_sbits = al((size_t)(4 + kClasses) * W * 4);
  const size_t b_ord = al((size_t)std::max<int64_t>(E, 1) * 4);
  const size_t b_dsize = al((size_t)nd1);
  const size_t b_seg = al((size_t)U * sizeof(SegInfo));
  const size_t b_dbase = al((size_t)(U + 1) * 8);
  void* p0;
  MOCHY_TRY(dev_alloc(ctx, &p0, b_didx + b_drow + b_seg + b_dbase));
  ctx->dense_idx = (int32_t*)p0;
  ctx->dense_row = (int32_t*)((char*)p0 + b_didx);
  ctx->d_seg = (SegInfo*)((char*)p0 + b_didx + b_drow);
  ctx->d_dbase = (int64_t*)((char*)p0 + b_didx + b_drow + b_seg);
  ctx->split_bytes = b_didx + b_drow + b_seg + b_dbase;
  k_dense_index<<<ceil_div(E, 256), 256, 0, st>>>(E, flag, pos, ctx->dense_idx, ctx->dense_row);
  MOCHY_LAUNCHED();
  // dense indices in ascending line degree (ties by id): triangles among
  // dense rows are then found from their lowest-degree member.  In a batch
  // the rows are grouped by unit first (stable), so each unit's dense rows
  // are one range of indices.
  std::vector<int64_t> hdb((size_t)U + 1, 0);
  hdb[U] = n_dense;
  if (n_dense > 0) {
    void* kt;
    MOCHY_TRY(scratch(ctx, 2, (size_t)n_dense * 4, &kt));
    if (n_dense > 1) {
      k_dense_keys<<<ceil_div(n_dense, 256), 256, 0, st>>>(n_dense, ctx->dense_row, ctx->noff,
                                                           (uint32_t*)kt);
      MOCHY_LAUNCHED();
      MOCHY_TRY(radix_sort_pairs_u32(ctx, (uint32_t*)kt, (uint32_t*)ctx->dense_row, n_dense, 32));
    }
    if (U > 1) {
      k_dense_units<<<ceil_div(n_dense, 256), 256, 0, st>>>(n_dense, ctx->dense_row, ctx->eoff,
                                                            ctx->enode, ctx->d_nseg, U,
                                                            (uint32_t*)kt);
      MOCHY_LAUNCHED();
      MOCHY_TRY(radix_sort_pairs_u32(ctx, (uint32_t*)kt, (uint32_t*)ctx->dense_row, n_dense,
                                     bits_for(U)));
      k_unit_starts<<<ceil_div(U + 1, 256), 256, 0, st>>>(n_dense, (const uint32_t*)kt, U,
                                                           ctx->d_dbase);
      MOCHY_LAUNCHED();
      MOCHY_CUDA(cudaMemcpyAsync(hdb.data(), ctx->d_dbase, (size_t)(U + 1) * 8,
                                 cudaMemcpyDeviceToHost, st));
    }
    k_dense_reindex<<<ceil_div(n_dense, 256), 256, 0, st>>>(n_dense, ctx->dense_row,
                                                            ctx->dense_idx);
    MOCHY_LAUNCHED();
    MOCHY_CUDA(cudaStreamSynchronize(st));
  }
  // each unit's window of dense words and the place of its bitmaps
  std::vector<SegInfo> seg((size_t)U);
  int64_t dwords = 0, wmax = 0;
  for (int u = 0; u < U; ++u) {
    SegInfo& sg = seg[u];
    const int64_t nd = hdb[u + 1] - hdb[u];
    sg.dbase = hdb[u];
    sg.wlo = hdb[u] >> 5;
    sg.wn = nd > 0 ? ((hdb[u + 1] + 31) >> 5) - sg.wlo : 0;
    sg.dboff = dwords;
    dwords += nd * 4 * sg.wn;
    sg.hbase = sg.nboff = 0;
    wmax = std::max(wmax, sg.wn);
  }
  if (dense_smem_bytes(wmax) + 1024 > ctx->smem_optin) {
    release_split(ctx);
    return fail(MOCHY_E_UNSUPPORTED, "too many dense rows for the shared-memory bitmap");
  }
  if (wmax > kMaxWindowWords) {
    // a lane of the dense kernel adds up to 32 per word of its share of the
    // window into 16-bit halves of its bins
    release_split(ctx);
    return fail(MOCHY_E_UNSUPPORTED, "more than " + std::to_string(kMaxWindowWords * 32) +
                                         " dense rows in one hypergraph; raise dense_threshold");
  }
  const size_t b_dbits = al((size_t)std::max<int64_t>(dwords, 1) * 4);
  const size_t rest = b_dbits + b_hidx + b_sbits + 2 * b_ord + b_dsize;
  void* p1;
  {
    const int rc = dev_alloc(ctx, &p1, rest);
    if (rc < 0) {
      release_split(ctx);
      return rc;
    }
  }
  ctx->rest_block = p1;
  ctx->rest_bytes = rest;
  char* base = (char*)p1;
  ctx->dbits = (uint32_t*)base;
  ctx->heavy_idx = (int32_t*)(base + b_dbits);
  ctx->sbits = (uint32_t*)(base + b_dbits + b_hidx);
  ctx->dense_order = (int32_t*)(base + b_dbits + b_hidx + b_sbits);
  ctx->sparse_order = (int32_t*)((char*)ctx->dense_order + b_ord);
  ctx->dsize = (uint8_t*)((char*)ctx->sparse_order + b_ord);
  if (U == 1 || n_dense == 0)
    MOCHY_CUDA(cudaMemcpyAsync(ctx->d_dbase, hdb.data(), (size_t)(U + 1) * 8,
                               cudaMemcpyHostToDevice, st));
  MOCHY_CUDA(cudaMemcpyAsync(ctx->d_seg, seg.data(), (size_t)U * sizeof(SegInfo),
                             cudaMemcpyHostToDevice, st));
  MOCHY_CUDA(cudaMemsetAsync(ctx->dbits, 0, b_dbits, st));
  MOCHY_CUDA(cudaMemsetAsync(ctx->sbits, 0, (size_t)(4 + kClasses) * W * 4, st));
  if (n_dense > 0) {
    k_dense_bits<<<(unsigned)std::min<int64_t>(n_dense, 1 << 16), 256, 0, st>>>(
        n_dense, ctx->d_seg, ctx->d_dbase, U, ctx->dense_row, ctx->eoff, ctx->noff, ctx->nadj,
        ctx->dense_idx, ctx->dbits);
    MOCHY_LAUNCHED();
    k_size_bits<<<ceil_div(n_dense, 256), 256, 0, st>>>(n_dense, W, ctx->dense_row, ctx->eoff,
                                                         ctx->theta, ctx->sbits, ctx->dsize);
    MOCHY_LAUNCHED();
  }
  // heavy nodes (numbered in node order, so each unit's are one range)
  k_heavy_flags<<<ceil_div(N + 1, 8), 256, 0, st>>>(N, ctx->voff, ctx->vedge, ctx->dense_idx,
                                                    ctx->heavy_thr, flag2);
  MOCHY_LAUNCHED();
  MOCHY_TRY(scan_exclusive_i64(ctx, flag2, pos2, N + 1));
  std::vector<int64_t> hhb((size_t)U + 1, 0);
  if (U > 1) {
    // heavy index at each unit's first node (pos is free again; U <= N)
    k_gather_at<<<ceil_div(U + 1, 256), 256, 0, st>>>(U + 1, pos2, ctx->d_nseg, pos);
    MOCHY_LAUNCHED();
    MOCHY_CUDA(cudaMemcpyAsync(hhb.data(), pos, (size_t)(U + 1) * 8, cudaMemcpyDeviceToHost, st));
  } else {
    MOCHY_CUDA(cudaMemcpyAsync(&hhb[1], pos2 + N, 8, cudaMemcpyDeviceToHost, st));
  }
  MOCHY_CUDA(cudaStreamSynchronize(st));
  const int64_t n_heavy = hhb[U];
  if (N > 0) {
    k_heavy_index<<<ceil_div(N, 256), 256, 0, st>>>(N, flag2, pos2, ctx->heavy_idx);
    MOCHY_LAUNCHED();
  }
  int64_t hwords = 0;
  for (int u = 0; u < U; ++u) {
    seg[u].hbase = hhb[u];
    seg[u].nboff = hwords;
    hwords += (hhb[u + 1] - hhb[u]) * seg[u].wn;
  }
  MOCHY_CUDA(cudaMemcpyAsync(ctx->d_seg, seg.data(), (size_t)U * sizeof(SegInfo),
                             cudaMemcpyHostToDevice, st));
  void* nb = nullptr;
  const size_t b_nbits = (size_t)std::max<int64_t>(hwords, 1) * 4;
  int rc = dev_alloc(ctx, &nb, b_nbits);
  if (rc < 0) {
    release_split(ctx);
    return rc;
  }
  ctx->nbits = (uint32_t*)nb;
  ctx->nbits_bytes = b_nbits;
  MOCHY_CUDA(cudaMemsetAsync(nb, 0, b_nbits, st));
  if (n_heavy > 0) {
    k_heavy_bits<<<ceil_div(N, 8), 256, 0, st>>>(N, ctx->d_seg, ctx->d_nseg, U, ctx->voff,
                                                 ctx->vedge, ctx->dense_idx, ctx->heavy_idx,
                                                 ctx->nbits);
    MOCHY_LAUNCHED();
  }
  // dense incidence lists (for the light nodes)
  k_dense_count<<<ceil_div(N + 1, 8), 256, 0, st>>>(N, ctx->voff, ctx->vedge, ctx->dense_idx, flag2);
  MOCHY_LAUNCHED();
  MOCHY_TRY(scan_exclusive_i64(ctx, flag2, pos2, N + 1));
  int64_t n_dinc = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&n_dinc, pos2 + N, 8, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  {
    const size_t b_off = al((size_t)(N + 1) * 8);
    const size_t bytes = b_off + (size_t)std::max<int64_t>(n_dinc, 1) * 4;
    void* q;
    rc = dev_alloc(ctx, &q, bytes);
    if (rc < 0) {
      release_split(ctx);
      return rc;
    }
    ctx->dinc_bytes = bytes;
    ctx->dvoff = (int64_t*)q;
    ctx->dvedge = (int32_t*)((char*)q + b_off);
    MOCHY_CUDA(cudaMemcpyAsync(ctx->dvoff, pos2, (size_t)(N + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if (N > 0) {
      k_dense_fill<<<ceil_div(N, 8), 256, 0, st>>>(N, ctx->voff, ctx->vedge, ctx->dense_idx,
                                                   ctx->dvoff, ctx->dvedge);
      MOCHY_LAUNCHED();
      k_sort_short_lists<<<ceil_div(N, 8), 256, 0, st>>>(N, ctx->dvoff, ctx->dvedge);
      MOCHY_LAUNCHED();
    }
  }
  // work orders
  k_split_flags<<<ceil_div(E + 1, 256), 256, 0, st>>>(E, ctx->row_order, ctx->dense_idx, flag, flag2);
  MOCHY_LAUNCHED();
  MOCHY_TRY(scan_exclusive_i64(ctx, flag, pos, E + 1));
  MOCHY_TRY(scan_exclusive_i64(ctx, flag2, pos2, E + 1));
  k_split_scatter<<<ceil_div(E, 256), 256, 0, st>>>(E, ctx->row_order, ctx->dense_idx, pos, pos2,
                                                    ctx->dense_order, ctx->sparse_order);
  MOCHY_LAUNCHED();
  MOCHY_CUDA(cudaStreamSynchronize(st));
  ctx->n_dense = n_dense;
  ctx->n_sparse = E - n_dense;
  ctx->n_heavy = n_heavy;
  ctx->wwords = W;
  ctx->wmax = wmax;
  ctx->dense_thr_used = thr;
  ctx->split_ready = true;
  return MOCHY_OK;
}

// Phase timing when tracing is on (mochy_trace or MOCHY_TRACE=1): events
// around each kernel on the context's stream, kept in the context and, with
// MOCHY_TRACE set, printed to stderr.
struct PhaseTimer {
  bool on = false, print = false;
  cudaStream_t st;
  cudaEvent_t ev[8];
  const char* name[8];
  int n = 0;
  bool stats = false;
  PhaseTimer(const mochy_ctx* c) : st(c->stream) {
    const char* e = getenv("MOCHY_TRACE");
    print = e && e[0] && e[0] != '0';
    on = c->trace > 0 || print;
    stats = c->trace > 1 || print;
  }
  void mark(const char* what) {
    if (!on || n >= 8) return;
    cudaEventCreate(&ev[n]);
    cudaEventRecord(ev[n], st);
    name[n++] = what;
  }
  void report(mochy_ctx* c) {
    if (!on || n < 2) return;
    if (!stats) memset(c->last_stats, 0, sizeof(c->last_stats));
    cudaEventSynchronize(ev[n - 1]);
    c->n_phases = 0;
    for (int i = 1; i < n; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
      snprintf(c->phase_name[c->n_phases], sizeof(c->phase_name[0]), "%s", name[i]);
      c->phase_ms[c->n_phases++] = ms;
    }
    if (stats)
    {
      cudaMemcpy(c->last_stats, c->stats, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
      cudaMemcpy(c->last_stats + 8, c->stats + 72, 8 * sizeof(unsigned long long),
                 cudaMemcpyDeviceToHost);
      cudaMemcpy(c->last_stats + 16, c->stats + 80, 8 * sizeof(unsigned long long),
                 cudaMemcpyDeviceToHost);
    }
    if (stats && print) {
      unsigned long long combo[64];
      cudaMemcpy(combo, c->stats + 8, sizeof(combo), cudaMemcpyDeviceToHost);
      fprintf(stderr, "[mochy]   rest combinations (xa,xb,xt): ");
      for (int q = 0; q < 64; ++q)
        if (combo[q]) fprintf(stderr, "(%d,%d,%d)=%llu ", q >> 4, (q >> 2) & 3, q & 3, combo[q]);
      fprintf(stderr, "\n");
    }

    if (print) {
      fprintf(stderr, "[mochy] split exact: E=%lld dense=%lld (threshold %d, %lld words) heavy=%lld\n",
              (long long)c->n_edges, (long long)c->n_dense, c->dense_thr_used,
              (long long)c->wwords, (long long)c->n_heavy);
      for (int i = 0; i < c->n_phases; ++i)
        fprintf(stderr, "[mochy]   %-18s %10.3f ms\n", c->phase_name[i], c->phase_ms[i]);
      if (stats)
        fprintf(stderr, "[mochy]   words %llu  candidates %llu  table %llu  exact %llu  light %llu\n",
                c->last_stats[0], c->last_stats[1], c->last_stats[2], c->last_stats[3],
                c->last_stats[4]);
    }
    for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
    n = 0;
  }
};

// Launch configuration of the three counting kernels (host-only calls, so
// that the launches themselves can be captured into a CUDA graph).
struct SplitPlan {
  SplitArgs g;
  unsigned grid_open = 0, grid_sparse = 0, grid_dense = 0;
  size_t smem_sparse = 0, smem_dense = 0;
  int max_deg = 1;
};

// Windows of at least this many dense words take the remaining candidates
// per lane, smaller ones spread them over the warp.  The share of candidates
// outside the popcounted bins falls as hypergraphs grow, and the per-lane
// path wins only when it is small.  Measured with identical counts: 36 to
// 352 words (4 to 10 % of the candidates remaining) spread 19 to 41 % faster,
// 983 words (2.9 %) spread 9 % faster, 4,498 words (1.9 %) per lane 4.5 %
// faster.
constexpr int64_t kLaneRestWords = 2048;

// the dense-triangle kernel for theta = 1 or another theta, with or without
// the tracing counters, remaining candidates per lane or spread (a batch,
// whose units are small, always spreads them)
template <bool kSeg>
static void (*dense_kernel(bool theta1, bool stats, int64_t wmax, int rest_path))(SplitArgs) {
  if constexpr (!kSeg) {
    if (rest_path == 1 || (rest_path == 0 && wmax >= kLaneRestWords)) {
      if (theta1)
        return stats ? k_dense_triangles<true, false, true, true> : k_dense_triangles<true, false, false, true>;
      return stats ? k_dense_triangles<false, false, true, true> : k_dense_triangles<false, false, false, true>;
    }
  }
  if (theta1)
    return stats ? k_dense_triangles<true, kSeg, true, false> : k_dense_triangles<true, kSeg, false, false>;
  return stats ? k_dense_triangles<false, kSeg, true, false> : k_dense_triangles<false, kSeg, false, false>;
}

template <bool kSeg>
static int plan_kernels(mochy_ctx* ctx, SplitPlan* p) {
  if (ctx->n_sparse > 0) {
    const size_t smem = sparse_smem_bytes(p->max_deg);
    if (smem + 1024 > ctx->smem_optin)
      return fail(MOCHY_E_UNSUPPORTED, "sparse rows too long for shared memory");
    MOCHY_TRY(ensure_dynamic_smem((const void*)k_sparse_triangles<kSeg>, smem));
    int per_sm = 0;
    MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sparse_triangles<kSeg>,
                                                             kThreads, smem));
    p->smem_sparse = smem;
    p->grid_sparse = (unsigned)std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1),
                                                 ctx->n_sparse);
  }
  if (ctx->n_dense > 0) {
    const size_t smem = dense_smem_bytes(ctx->wmax);
    auto kern = dense_kernel<kSeg>(ctx->theta == 1, p->g.stats != nullptr, ctx->wmax, ctx->rest_path);
    MOCHY_TRY(ensure_dynamic_smem((const void*)kern, smem));
    int per_sm = 0;
    MOCHY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDThreads, smem));
    p->smem_dense = smem;
    p->grid_dense = (unsigned)std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1),
                                                ctx->n_dense);
  }
  return MOCHY_OK;
}

static int plan_split(mochy_ctx* ctx, unsigned long long* d_hist, bool stats, SplitPlan* p) {
  SplitArgs& g = p->g;
  g.n_edges = ctx->n_edges;
  g.eoff = ctx->eoff;
  g.enode = ctx->enode;
  g.voff = ctx->voff;
  g.vedge = ctx->vedge;
  g.noff = ctx->noff;
  g.nadj = ctx->nadj;
  g.lut3 = ctx->tables.lut3;
  g.hist = d_hist;
  g.theta = ctx->theta;
  g.n_dense = ctx->n_dense;
  g.wwords = ctx->wwords;
  g.dense_idx = ctx->dense_idx;
  g.dense_row = ctx->dense_row;
  g.dbits = ctx->dbits;
  g.heavy_idx = ctx->heavy_idx;
  g.nbits = ctx->nbits;
  g.sbits = ctx->sbits;
  g.dvoff = ctx->dvoff;
  g.dvedge = ctx->dvedge;
  g.dsize = ctx->dsize;
  g.cbits = ctx->sbits + 4 * ctx->wwords;
  g.stats = stats ? ctx->stats : nullptr;
  g.order = nullptr;
  g.n_order = 0;
  g.queue = nullptr;
  g.centres = nullptr;
  g.n_centres = 0;
  g.n_units = ctx->n_units;
  g.nseg = ctx->d_nseg;
  g.seg = ctx->d_seg;
  p->grid_open = (unsigned)std::min<int64_t>(ceil_div(ctx->n_edges, kOpenWarps),
                                             (int64_t)ctx->num_sms * 8);
  p->max_deg = std::max(1, (int)std::min<int64_t>(ctx->max_deg, ctx->dense_thr_used - 1));
  return ctx->n_units > 1 ? plan_kernels<true>(ctx, p) : plan_kernels<false>(ctx, p);
}

// Rows the counting kernels work on: every centre and the split's sparse and
// dense work orders, or a subset of the rows.
struct WorkLists {
  const int32_t* centres = nullptr;   // null: every row is a centre
  int64_t n_centres = 0;
  const int32_t* sparse = nullptr;
  int64_t n_sparse = 0;
  const int32_t* dense = nullptr;
  int64_t n_dense = 0;
};

static WorkLists all_rows(const mochy_ctx* ctx) {
  WorkLists w;
  w.sparse = ctx->sparse_order;
  w.n_sparse = ctx->n_sparse;
  w.dense = ctx->dense_order;
  w.n_dense = ctx->n_dense;
  return w;
}

// The counting kernels: open pairs, triangles from sparse rows, triangles of
// dense rows.  Stream operations only (capturable).
template <bool kSeg>
static int launch_split(mochy_ctx* ctx, SplitPlan p, PhaseTimer* timer, const WorkLists& wl) {
  cudaStream_t st = ctx->stream;
  SplitArgs g = p.g;
  MOCHY_CUDA(cudaMemsetAsync(ctx->counters, 0, 16 * sizeof(int32_t), st));
  g.centres = wl.centres;
  g.n_centres = wl.n_centres;
  if (p.grid_open > 0 && (!wl.centres || wl.n_centres > 0)) {
    k_open_pairs<kSeg><<<p.grid_open, kOpenThreads, 0, st>>>(g);
    MOCHY_LAUNCHED();
  }
  if (timer) timer->mark("open pairs");
  if (p.grid_sparse > 0 && wl.n_sparse > 0) {
    g.order = wl.sparse;
    g.n_order = wl.n_sparse;
    g.queue = ctx->counters + 5;
    k_sparse_triangles<kSeg><<<p.grid_sparse, kThreads, p.smem_sparse, st>>>(g, p.max_deg);
    MOCHY_LAUNCHED();
    if (timer) timer->mark("sparse triangles");
  }
  if (p.grid_dense > 0 && wl.n_dense > 0) {
    g.order = wl.dense;
    g.n_order = wl.n_dense;
    g.queue = ctx->counters + 6;
    auto kern = dense_kernel<kSeg>(ctx->theta == 1, g.stats != nullptr, ctx->wmax, ctx->rest_path);
    kern<<<p.grid_dense, kDThreads, p.smem_dense, st>>>(g);
    MOCHY_LAUNCHED();
    if (timer) timer->mark("dense triangles");
  }
  return MOCHY_OK;
}

int count_exact_split(mochy_ctx* ctx, unsigned long long* d_hist) {
  cudaStream_t st = ctx->stream;
  PhaseTimer timer(ctx);
  if (timer.stats && !ctx->stats) {
    void* p;
    MOCHY_TRY(dev_alloc(ctx, &p, kStatWords * sizeof(unsigned long long)));
    ctx->stats = (unsigned long long*)p;
  }
  if (timer.stats)
    MOCHY_CUDA(cudaMemsetAsync(ctx->stats, 0, kStatWords * sizeof(unsigned long long), st));
  timer.mark("start");
  MOCHY_TRY(prepare_split(ctx));
  timer.mark("prepare");
  SplitPlan plan;
  MOCHY_TRY(plan_split(ctx, d_hist, timer.stats, &plan));
  if (ctx->n_units > 1) {
    MOCHY_TRY(launch_split<true>(ctx, plan, &timer, all_rows(ctx)));
  } else {
    MOCHY_TRY(launch_split<false>(ctx, plan, &timer, all_rows(ctx)));
  }
  timer.report(ctx);
  return MOCHY_OK;
}

namespace {
// rows of a subset split by kind: sparse rows to the front of `sparse`,
// dense rows to the front of `dense` (in any order), counts in cnt[0..1]
__global__ void k_rows_by_kind(int64_t n, const int32_t* __restrict__ rows,
                               const int32_t* __restrict__ didx, int32_t* __restrict__ sparse,
                               int32_t* __restrict__ dense, unsigned long long* __restrict__ cnt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int32_t r = rows[q];
  if (didx[r] >= 0) dense[atomicAdd(&cnt[1], 1ull)] = r;
  else sparse[atomicAdd(&cnt[0], 1ull)] = r;
}
}  // namespace

// The share of a set of rows in the split count: the pairs of each row's
// neighbours as if open (open-pair kernel, centres of the set only), and the
// closed instances whose first member in the split's order (sparse rows by
// id, then dense rows by line degree and id) is in the set, each with its
// as-if-open terms taken off (triangle kernels, rows of the set only).
// Summed over all rows it is the exact count.
int count_split_rows(mochy_ctx* ctx, const int32_t* d_rows, int64_t n_rows,
                     unsigned long long* d_hist) {
  if (ctx->n_units != 1) return fail(MOCHY_E_INVALID, "row subsets need a lone hypergraph");
  cudaStream_t st = ctx->stream;
  PhaseTimer timer(ctx);
  if (timer.stats && !ctx->stats) {
    void* p;
    MOCHY_TRY(dev_alloc(ctx, &p, kStatWords * sizeof(unsigned long long)));
    ctx->stats = (unsigned long long*)p;
  }
  if (timer.stats)
    MOCHY_CUDA(cudaMemsetAsync(ctx->stats, 0, kStatWords * sizeof(unsigned long long), st));
  MOCHY_CUDA(cudaMemsetAsync(d_hist, 0, 432 * 8, st));
  timer.mark("start");
  MOCHY_TRY(prepare_split(ctx));
  timer.mark("prepare");
  if (n_rows == 0) return MOCHY_OK;
  void* t;
  MOCHY_TRY(scratch(ctx, 3, (size_t)n_rows * 8 + 64, &t));
  unsigned long long* cnt = (unsigned long long*)t;
  int32_t* sparse = (int32_t*)((char*)t + 64);
  int32_t* dense = sparse + n_rows;
  MOCHY_CUDA(cudaMemsetAsync(cnt, 0, 16, st));
  k_rows_by_kind<<<ceil_div(n_rows, 256), 256, 0, st>>>(n_rows, d_rows, ctx->dense_idx, sparse,
                                                         dense, cnt);
  MOCHY_LAUNCHED();
  unsigned long long hc[2] = {0, 0};
  MOCHY_CUDA(cudaMemcpyAsync(hc, cnt, 16, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  SplitPlan plan;
  MOCHY_TRY(plan_split(ctx, d_hist, timer.stats, &plan));
  WorkLists wl;
  wl.centres = d_rows;
  wl.n_centres = n_rows;
  wl.sparse = sparse;
  wl.n_sparse = (int64_t)hc[0];
  wl.dense = dense;
  wl.n_dense = (int64_t)hc[1];
  MOCHY_TRY(launch_split<false>(ctx, plan, &timer, wl));
  timer.report(ctx);
  return MOCHY_OK;
}

// The same count with the clearing of the n_units histograms and the three
// counting kernels captured into one CUDA graph and replayed by a single
// launch; *ms receives the device time of that launch.  Preparation (which
// sizes its arrays on the host) runs before the capture.
int count_split_graph(mochy_ctx* ctx, unsigned long long* d_hist, float* ms) {
  cudaStream_t st = ctx->stream;
  MOCHY_TRY(prepare_split(ctx));
  SplitPlan plan;
  MOCHY_TRY(plan_split(ctx, d_hist, false, &plan));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  MOCHY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = MOCHY_OK;
  if (cudaMemsetAsync(d_hist, 0, (size_t)ctx->n_units * 432 * 8, st) != cudaSuccess)
    rc = fail(MOCHY_E_CUDA, "histogram clear failed during capture");
  if (rc == MOCHY_OK)
    rc = ctx->n_units > 1 ? launch_split<true>(ctx, plan, nullptr, all_rows(ctx))
                          : launch_split<false>(ctx, plan, nullptr, all_rows(ctx));
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  if (rc == MOCHY_OK && ec != cudaSuccess)
    rc = cuda_fail(ec, "cudaStreamEndCapture", __FILE__, __LINE__);
  cudaGraphExec_t exec = nullptr;
  if (rc == MOCHY_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    if (ei != cudaSuccess) rc = cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  if (rc == MOCHY_OK) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    const cudaError_t el = cudaGraphLaunch(exec, st);
    if (el != cudaSuccess) rc = cuda_fail(el, "cudaGraphLaunch", __FILE__, __LINE__);
    cudaEventRecord(e1, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (rc == MOCHY_OK && es != cudaSuccess) rc = cuda_fail(es, "batch count", __FILE__, __LINE__);
    float t = 0.f;
    if (rc == MOCHY_OK) cudaEventElapsedTime(&t, e0, e1);
    if (ms) *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  return rc;
}

}  // namespace mochy

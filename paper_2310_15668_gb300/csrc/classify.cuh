// Classification of one instance {e_i, e_j, e_k} (Lemma "motif:time",
// Section 3.2; Lemma "3H-motif:time", Section 4.1).
//
// From the sizes A = |e_i|, B = |e_j|, C = |e_k|, the overlaps x = |e_i & e_j|,
// y = |e_j & e_k|, z = |e_k & e_i| and t = |e_i & e_j & e_k| the seven Venn
// regions are
//   (1) A - x - z + t   (2) B - x - y + t   (3) C - y - z + t
//   (4) x - t           (5) y - t           (6) z - t           (7) t
// and each region takes state 0 (empty), 1 (at most theta nodes) or 2 (more).
// The ternary code sum_p state_p 3^p indexes the 3h-motif table; the h-motif
// is the parent of the 3h-motif.
#pragma once

#include "common.cuh"

namespace mochy {

__device__ __forceinline__ int region_state(int r, int theta) {
  return (r > 0 ? 1 : 0) + (r > theta ? 1 : 0);
}

__device__ __forceinline__ int ternary_code(int A, int B, int C, int x, int y, int z, int t,
                                            int theta) {
  return region_state(A - x - z + t, theta) + 3 * region_state(B - x - y + t, theta) +
         9 * region_state(C - y - z + t, theta) + 27 * region_state(x - t, theta) +
         81 * region_state(y - t, theta) + 243 * region_state(z - t, theta) +
         729 * region_state(t, theta);
}

// h[id] += v on a 64-bit bin in shared memory, as a 32-bit atomic add on its
// low word plus, when that add carries out or v is negative, an add of the
// carry and v's high word to the high word.  The bin is exact once every add
// has completed (it is only read after a barrier).
__device__ __forceinline__ void shared_bin_add(unsigned long long* h, int id, long long v) {
  unsigned int* w = reinterpret_cast<unsigned int*>(h + id);
  const unsigned int u = (unsigned int)v;
  const unsigned int old = atomicAdd(w, u);
  const unsigned int adj = (old + u < old ? 1u : 0u) + (unsigned int)((unsigned long long)v >> 32);
  if (adj) atomicAdd(w + 1, adj);
}

// Per-lane run-length cache in front of a histogram: consecutive instances
// of the same motif on a lane cost one register add.  kShared: the
// histogram is in shared memory, and its 64-bit bins are added through
// shared_bin_add; otherwise (rows in device memory) by 64-bit atomics.
template <bool kShared>
struct RunCacheT {
  int id = -1;
  unsigned long long n = 0;
  __device__ __forceinline__ void put(unsigned long long* hist) {
    if (kShared) shared_bin_add(hist, id, (long long)n);
    else atomicAdd(&hist[id], n);
  }
  __device__ __forceinline__ void add(int new_id, unsigned long long* hist, unsigned long long c = 1) {
    if (new_id != id) {
      if (n) put(hist);
      id = new_id;
      n = 0;
    }
    n += c;
  }
  __device__ __forceinline__ void flush(unsigned long long* hist) {
    if (n) put(hist);
    n = 0;
    id = -1;
  }
};
using RunCache = RunCacheT<true>;

// |X & Y| for two ascending node lists.
__device__ __forceinline__ int sorted_overlap(const int32_t* X, int nx, const int32_t* Y, int ny) {
  int a = 0, b = 0, c = 0;
  while (a < nx && b < ny) {
    const int32_t u = X[a], v = Y[b];
    c += u == v ? 1 : 0;
    a += u <= v ? 1 : 0;
    b += v <= u ? 1 : 0;
  }
  return c;
}

// |X & Y & Z| for three ascending node lists.
__device__ __forceinline__ int sorted_overlap3(const int32_t* X, int nx, const int32_t* Y, int ny,
                                               const int32_t* Z, int nz) {
  int a = 0, b = 0, c = 0, n = 0;
  while (a < nx && b < ny && c < nz) {
    const int32_t u = X[a], v = Y[b], w = Z[c];
    const int32_t m = max(u, max(v, w));
    if (u == m && v == m && w == m) { ++n; ++a; ++b; ++c; continue; }
    a += u < m ? 1 : 0;
    b += v < m ? 1 : 0;
    c += w < m ? 1 : 0;
  }
  return n;
}

// omega stored in an entry of a row whose hyperedge has `row_size` nodes
__device__ __forceinline__ int entry_omega(uint32_t w1, int row_size) {
  return row_size <= kMaskedMax ? __popc(w1) : (int)w1;
}

// Position of key `a` in the ascending row [lo, hi) (first id >= a), found by
// a warp: 32 probes per round.  All lanes return the same value.
__device__ __forceinline__ int64_t warp_lower_bound(const uint2* __restrict__ nadj, int64_t lo,
                                                    int64_t hi, uint32_t a) {
  const int lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t s = lo + (int64_t)lane * step;
    const bool less = s < hi && ent_id(nadj[s]) < a;
    const int c = __popc(__ballot_sync(0xffffffffu, less));
    if (c == 0) return lo;
    const int64_t nlo = lo + (int64_t)(c - 1) * step + 1;
    const int64_t nhi = min(hi, lo + (int64_t)c * step);
    lo = nlo;
    hi = nhi;
  }
  const int64_t s = lo + lane;
  const bool less = s < hi && ent_id(nadj[s]) < a;
  return lo + __popc(__ballot_sync(0xffffffffu, less));
}

}  // namespace mochy

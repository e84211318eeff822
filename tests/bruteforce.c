/* Brute-force pin for the oracle (test infrastructure).
 *
 * Enumerates every unordered triple {e_a, e_b, e_c} of hyperedges, keeps the
 * connected ones (at least two of the three pairs intersect, Section 2.1),
 * computes the seven Venn-region cardinalities directly from node bitsets
 * (no inclusion-exclusion), maps each to states {0, 1, >1} (theta = 1,
 * Section 4.1), and canonicalises by trying all six orders of the three
 * actual hyperedges (re-deriving the regions from the sets each time) and
 * keeping the lexicographically smallest region tuple.  It writes one line
 * per canonical ternary tuple: "<tuple digits> <count>".
 *
 * Input on stdin: n_nodes n_edges, then per hyperedge: size v1 v2 ...
 * Shares no code with the oracle or the CUDA library.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static int W;              /* 64-bit words per node bitset */
static uint64_t* bits;     /* n_edges x W */

static int popc_and3(const uint64_t* x, const uint64_t* y, const uint64_t* z,
                     int nx, int ny, int nz) {
  /* |region| where membership in each set is required (1), forbidden (0) */
  int c = 0;
  for (int w = 0; w < W; ++w) {
    uint64_t a = nx ? x[w] : ~x[w];
    uint64_t b = ny ? y[w] : ~y[w];
    uint64_t d = nz ? z[w] : ~z[w];
    c += __builtin_popcountll(a & b & d & (x[w] | y[w] | z[w]));
  }
  return c;
}

/* region tuple of (x, y, z) in the paper's order, as ternary digits */
static void tuple3(const uint64_t* x, const uint64_t* y, const uint64_t* z, int out[7]) {
  int r[7];
  r[0] = popc_and3(x, y, z, 1, 0, 0);
  r[1] = popc_and3(x, y, z, 0, 1, 0);
  r[2] = popc_and3(x, y, z, 0, 0, 1);
  r[3] = popc_and3(x, y, z, 1, 1, 0);
  r[4] = popc_and3(x, y, z, 0, 1, 1);
  r[5] = popc_and3(x, y, z, 1, 0, 1);
  r[6] = popc_and3(x, y, z, 1, 1, 1);
  for (int p = 0; p < 7; ++p) out[p] = r[p] == 0 ? 0 : (r[p] == 1 ? 1 : 2);
}

static int less7(const int* a, const int* b) {
  for (int p = 0; p < 7; ++p)
    if (a[p] != b[p]) return a[p] < b[p];
  return 0;
}

static int meets(const uint64_t* x, const uint64_t* y) {
  for (int w = 0; w < W; ++w)
    if (x[w] & y[w]) return 1;
  return 0;
}

int main(void) {
  long n_nodes, n_edges;
  if (scanf("%ld %ld", &n_nodes, &n_edges) != 2) return 1;
  W = (int)((n_nodes + 63) / 64);
  bits = (uint64_t*)calloc((size_t)n_edges * W, sizeof(uint64_t));
  for (long e = 0; e < n_edges; ++e) {
    int s;
    if (scanf("%d", &s) != 1) return 1;
    for (int q = 0; q < s; ++q) {
      long v;
      if (scanf("%ld", &v) != 1) return 1;
      bits[e * W + v / 64] |= 1ull << (v % 64);
    }
  }
  /* adjacency matrix */
  unsigned char* adj = (unsigned char*)calloc((size_t)n_edges * n_edges, 1);
  for (long a = 0; a < n_edges; ++a)
    for (long b = a + 1; b < n_edges; ++b)
      adj[a * n_edges + b] = adj[b * n_edges + a] =
          (unsigned char)meets(bits + a * W, bits + b * W);
  long long* count = (long long*)calloc(2187, sizeof(long long));
  for (long a = 0; a < n_edges; ++a)
    for (long b = a + 1; b < n_edges; ++b) {
      const int ab = adj[a * n_edges + b];
      for (long c = b + 1; c < n_edges; ++c) {
        const int n = ab + adj[b * n_edges + c] + adj[a * n_edges + c];
        if (n < 2) continue;
        const uint64_t* S[3] = {bits + a * W, bits + b * W, bits + c * W};
        static const int ord[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
        int best[7], cur[7];
        for (int o = 0; o < 6; ++o) {
          tuple3(S[ord[o][0]], S[ord[o][1]], S[ord[o][2]], cur);
          if (o == 0 || less7(cur, best)) memcpy(best, cur, sizeof(best));
        }
        int code = 0;
        for (int p = 0; p < 7; ++p) code = code * 3 + best[p];
        count[code] += 1;
      }
    }
  for (int code = 0; code < 2187; ++code)
    if (count[code]) {
      int d[7], x = code;
      for (int p = 6; p >= 0; --p) { d[p] = x % 3; x /= 3; }
      for (int p = 0; p < 7; ++p) putchar('0' + d[p]);
      printf(" %lld\n", count[code]);
    }
  return 0;
}

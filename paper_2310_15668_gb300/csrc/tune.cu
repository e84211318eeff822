// Choice of the dense-row threshold of the split exact count.
//
// A row whose line degree is at least the threshold is "dense": its
// neighbourhood becomes a bitmap over the dense rows and triangles among
// dense rows are scanned 32 candidates per word; every other row is staged
// as a list and its triangles are found by probing.  The tuner evaluates a
// cost model on the line-degree distribution for every power-of-two
// threshold the shared-memory limits allow and keeps the cheapest:
//   dense part  ~ (wedge scans between dense rows) x (words per scan)
//               ~ 1/2 S_d f_d x W / 3, with S_d the degree mass of dense
//                 rows, f_d = S_d / S the chance that a neighbour is dense
//                 and W = n_dense / 32 words;
//   sparse part ~ sum over sparse rows of deg^2 (pairs of neighbours probed).
// Measured on GB300 (medium workload, thresholds 512..8192): the words the
// dense kernel scans hardly fall as the threshold rises, because dense rows
// are ordered by degree and most words come from the highest-degree rows,
// while the model's dense term falls steeply; a scanned word costs about as
// much as a probed pair.  A weight of 0.1 on the model's dense term puts the
// minimum where the measured total is smallest.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mochy {

size_t dense_smem_bytes(int64_t W);       // count_split.cu
size_t sparse_smem_bytes(int max_deg);    // count_split.cu

int choose_dense_threshold(mochy_ctx* ctx) {
  const int64_t E = ctx->n_edges;
  std::vector<int64_t> off((size_t)E + 1);
  MOCHY_CUDA(cudaMemcpyAsync(off.data(), ctx->noff, off.size() * 8, cudaMemcpyDeviceToHost,
                             ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  // a batch is a disjoint union: every hypergraph has its own dense index
  // space, so the words per scan are counted per hypergraph
  const int U = ctx->n_units;
  std::vector<int64_t> eseg = U > 1 ? ctx->h_eseg : std::vector<int64_t>{0, E};
  std::vector<int64_t> deg((size_t)E);
  std::vector<double> S((size_t)U, 0.0);
  for (int u = 0; u < U; ++u)
    for (int64_t i = eseg[u]; i < eseg[u + 1]; ++i) {
      deg[i] = off[i + 1] - off[i];
      S[u] += (double)deg[i];
    }
  const double word_weight = 0.1;
  int best = -1;
  double best_cost = 0.0;
  for (int64_t thr = 32; thr <= (int64_t)1 << 20; thr <<= 1) {
    int64_t nd_all = 0, max_sparse = 0, wmax = 1;
    double cost = 0.0;
    for (int u = 0; u < U; ++u) {
      int64_t nd = 0;
      double Sd = 0.0, sparse = 0.0;
      for (int64_t i = eseg[u]; i < eseg[u + 1]; ++i) {
        if (deg[i] >= thr) {
          ++nd;
          Sd += (double)deg[i];
        } else {
          sparse += (double)deg[i] * (double)deg[i];
          max_sparse = std::max(max_sparse, deg[i]);
        }
      }
      const int64_t W = std::max<int64_t>((nd + 31) / 32, 1);
      wmax = std::max(wmax, U > 1 ? W + 1 : W);   // a unit's window may straddle a word
      const double fd = S[u] > 0 ? Sd / S[u] : 0.0;
      cost += word_weight * 0.5 * Sd * fd * (double)W / 3.0 + sparse;
      nd_all += nd;
    }
    if (dense_smem_bytes(wmax) + 1024 > ctx->smem_optin) continue;
    if (wmax > kMaxWindowWords) continue;
    if (sparse_smem_bytes((int)std::max<int64_t>(max_sparse, 1)) + 1024 > ctx->smem_optin) continue;
    if (best < 0 || cost < best_cost) {
      best = (int)thr;
      best_cost = cost;
    }
    if (nd_all == 0) break;   // larger thresholds change nothing
  }
  if (best < 0) return fail(MOCHY_E_UNSUPPORTED, "no dense threshold fits shared memory");
  return best;
}

}  // namespace mochy

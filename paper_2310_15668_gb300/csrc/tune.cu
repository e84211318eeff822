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

namespace mochy {

int count_split_rows(mochy_ctx* ctx, const int32_t* d_rows, int64_t n_rows,
                     unsigned long long* d_hist);   // count_split.cu

// Measured choice of the dense threshold: for each candidate threshold the
// split structures are built and the split count of one seeded sample of
// rows (the same rows for every candidate) is timed with CUDA events on the
// context's stream; the fastest candidate is kept as the context's
// threshold.  A candidate whose structures do not fit the device memory or
// the kernels' limits is skipped (its time is reported as -1).
int tune_dense_threshold(mochy_ctx* ctx, const int32_t* cand, int32_t n_cand, double fraction,
                         uint64_t seed, int32_t* best_out, int32_t* tried_out, double* ms_out) {
  const int64_t E = ctx->n_edges;
  std::vector<int32_t> cs(cand, cand + n_cand);
  if (cs.empty()) {
    ctx->dense_thr = 0;
    const int model = choose_dense_threshold(ctx);
    if (model < 0) return model;
    for (int f : {4, 2}) cs.push_back(std::max(32, model / f));
    cs.push_back(model);
    for (int f : {2, 4}) cs.push_back(model * f);
  }
  // the sample: rows whose 64-bit hash of (seed, row) falls below fraction
  std::vector<int32_t> rows;
  const uint64_t cut = (uint64_t)(std::min(std::max(fraction, 0.0), 1.0) * 18446744073709551615.0);
  for (int64_t r = 0; r < E; ++r) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(r + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    if (z <= cut) rows.push_back((int32_t)r);
  }
  if (rows.empty()) rows.push_back(0);
  void* d = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &d, rows.size() * 4));
  int rc = MOCHY_OK;
  if (cudaMemcpyAsync(d, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, ctx->stream) !=
      cudaSuccess)
    rc = fail(MOCHY_E_CUDA, "tuner row copy failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int32_t saved = ctx->dense_thr;
  int32_t best = -1;
  double best_ms = 0.0;
  for (size_t c = 0; c < cs.size() && rc == MOCHY_OK; ++c) {
    release_split(ctx);
    ctx->dense_thr = cs[c];
    double ms = -1.0;
    if (prepare_split(ctx) == MOCHY_OK) {
      cudaEventRecord(e0, ctx->stream);
      const int r2 = count_split_rows(ctx, (const int32_t*)d, (int64_t)rows.size(), ctx->hist);
      cudaEventRecord(e1, ctx->stream);
      if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        rc = fail(MOCHY_E_CUDA, "tuner count failed");
      } else if (r2 == MOCHY_OK) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms = t;
        if (best < 0 || ms < best_ms) {
          best = cs[c];
          best_ms = ms;
        }
      }
    }
    if (ms_out) ms_out[c] = ms;
    if (tried_out) tried_out[c] = cs[c];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release_split(ctx);
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d, rows.size() * 4);
  if (rc != MOCHY_OK) {
    ctx->dense_thr = saved;
    return rc;
  }
  if (best < 0) {
    ctx->dense_thr = saved;
    return fail(MOCHY_E_UNSUPPORTED, "no candidate threshold fits");
  }
  ctx->dense_thr = best;
  if (best_out) *best_out = best;
  return MOCHY_OK;
}

}  // namespace mochy

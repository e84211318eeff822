// Batched significance and characteristic profiles (Eq. "significance" and
// Eq. "cp", Section 3.1): many input hypergraphs, each with its randomized
// copies (Algorithm "randomized_hypergraph_alg" followed by "transform"),
// generated on the device and counted exactly together.
//
// The inputs and all their copies form one disjoint union of "units" (unit
// g (R+1) is input g, unit g (R+1) + 1 + c its copy c), each with its own node
// and hyperedge ranges.  The union is projected once; the split exact count
// (count_split.cu) keeps a dense index space, bitmap windows and a histogram
// per unit, and its three persistent work-queue kernels run over the rows of
// every unit at once, captured into one CUDA graph and replayed by a single
// launch.  A unit's counts are exactly those of its hypergraph counted alone
// (no triple crosses two units), so every profile equals what mochy_profile
// gives for that input and seed.  When the union would not fit the memory
// budget the inputs are split into waves, each one union and one launch.
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "philox.cuh"

namespace mochy {
namespace {

struct UnitRow {
  int64_t pp;      // first pair of the unit
  int64_t nb;      // first node of the unit in the union
  int64_t eb;      // first hyperedge (before the transform)
  int32_t g;       // input hypergraph (within the wave)
  int32_t copy;    // copy index, -1 for the input itself
};

struct GraphRow {
  int64_t n0, e0, t0;   // first node, hyperedge and incidence in the input union
  int64_t N, E, T;      // nodes, hyperedges (after duplicate removal), incidences
  uint64_t seed;
};

__device__ __forceinline__ int64_t owner(const int64_t* __restrict__ pre, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int64_t m = (lo + hi) >> 1;
    if (pre[m] <= x) lo = m; else hi = m;
  }
  return lo;
}

// (node, hyperedge) pairs of every unit: an input's incidences as they are,
// a copy's Chung-Lu draws (the same Philox counters as randomize_graph, with
// the input's degree prefixes), both relabelled into the unit's ranges
__global__ void k_batch_pairs(int64_t P, const int64_t* __restrict__ pp, int n_units,
                              const UnitRow* __restrict__ units,
                              const GraphRow* __restrict__ graphs,
                              const int64_t* __restrict__ eoff, const int32_t* __restrict__ enode,
                              const int64_t* __restrict__ voff, uint32_t* __restrict__ node,
                              uint32_t* __restrict__ edge) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const UnitRow ur = units[seg_of(pp, n_units, i)];
  const GraphRow gr = graphs[ur.g];
  const int64_t d = i - ur.pp;
  int64_t v, j;
  if (ur.copy < 0) {
    const int64_t q = gr.t0 + d;
    j = owner(eoff + gr.e0, gr.E, q);
    v = enode[q] - gr.n0;
  } else {
    const uint64_t ua = philox_u64(gr.seed, (uint64_t)d, 3u, (uint32_t)ur.copy);
    const uint64_t ub = philox_u64(gr.seed, (uint64_t)d, 4u, (uint32_t)ur.copy);
    v = owner(voff + gr.n0, gr.N, voff[gr.n0] + (int64_t)__umul64hi(ua, (uint64_t)gr.T));
    j = owner(eoff + gr.e0, gr.E, gr.t0 + (int64_t)__umul64hi(ub, (uint64_t)gr.T));
  }
  node[i] = (uint32_t)(ur.nb + v);
  edge[i] = (uint32_t)(ur.eb + j);
}

// first hyperedge of each unit: the first whose smallest node lies at or
// after the unit's first node (hyperedges are grouped by unit)
__global__ void k_unit_edge_starts(int n_units, const int64_t* __restrict__ nseg, int64_t E,
                                   const int64_t* __restrict__ eoff,
                                   const int32_t* __restrict__ enode, int64_t* __restrict__ out) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u > n_units) return;
  int64_t lo = 0, hi = E;
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if ((int64_t)enode[eoff[m]] < nseg[u]) lo = m + 1; else hi = m;
  }
  out[u] = lo;
}

double ms_since(const cudaEvent_t& a, const cudaEvent_t& b) {
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  return (double)t;
}

// Marks the context as a union of units with the given node starts and
// finds the units' hyperedge starts.
int set_units(mochy_ctx* ctx, const std::vector<int64_t>& nseg) {
  const int U = (int)nseg.size() - 1;
  void* p;
  MOCHY_TRY(dev_alloc(ctx, &p, (size_t)(2 * U + 2) * 8));
  ctx->d_nseg = (int64_t*)p;
  ctx->nseg_bytes = (size_t)(2 * U + 2) * 8;
  int64_t* d_eseg = ctx->d_nseg + U + 1;
  MOCHY_CUDA(cudaMemcpyAsync(ctx->d_nseg, nseg.data(), (size_t)(U + 1) * 8,
                             cudaMemcpyHostToDevice, ctx->stream));
  k_unit_edge_starts<<<ceil_div(U + 1, 256), 256, 0, ctx->stream>>>(U, ctx->d_nseg, ctx->n_edges,
                                                                     ctx->eoff, ctx->enode, d_eseg);
  MOCHY_LAUNCHED();
  ctx->h_nseg = nseg;
  ctx->h_eseg.assign((size_t)U + 1, 0);
  MOCHY_CUDA(cudaMemcpyAsync(ctx->h_eseg.data(), d_eseg, (size_t)(U + 1) * 8,
                             cudaMemcpyDeviceToHost, ctx->stream));
  MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->n_units = U;
  return MOCHY_OK;
}

struct Inputs {
  const int64_t* n_nodes;
  const int64_t* n_edges;
  const int64_t* const* off;
  const int32_t* const* nodes;
  const uint64_t* seeds;
};

struct Outputs {
  double *sig_h, *cp_h, *sig_3h, *cp_3h;
  int64_t *counts_h, *counts_3h;
  int32_t* degenerate;
  mochy_batch_info* info;
  bool any_degenerate;
};

// owns a context of a wave
struct Ctx {
  mochy_ctx* c = nullptr;
  ~Ctx() { if (c) mochy_destroy(c); }
};

struct Events {
  cudaEvent_t e[6];
  Events() { for (auto& x : e) cudaEventCreate(&x); }
  ~Events() { for (auto& x : e) cudaEventDestroy(x); }
};

// owns a device block of a context
struct Block {
  mochy_ctx* c;
  void* p = nullptr;
  size_t b = 0;
  ~Block() {
    if (!p) return;
    cudaStreamSynchronize(c->stream);
    dev_free(c, p, b);
  }
};

int run_wave(const mochy_config& cfg, const Inputs& in, int g0, int g1, int R, Outputs& out) {
  const int G = g1 - g0;
  const int R1 = R + 1;
  const int U = G * R1;
  // 1. the inputs as one union
  Ctx cin;
  MOCHY_TRY(mochy_create(&cin.c, &cfg));
  mochy_ctx* ci = cin.c;
  cudaStream_t st = ci->stream;
  Events ev;
  cudaEventRecord(ev.e[0], st);
  std::vector<int64_t> nseg_in((size_t)G + 1, 0);
  int64_t E_in = 0, T_in = 0;
  for (int g = 0; g < G; ++g) {
    const int64_t Eg = in.n_edges[g0 + g];
    if (Eg > 0 && in.off[g0 + g][0] != 0) return fail(MOCHY_E_INVALID, "offsets must start at 0");
    const int64_t Tg = Eg > 0 ? in.off[g0 + g][Eg] : 0;
    if (Tg < 0) return fail(MOCHY_E_INVALID, "bad offsets");
    nseg_in[g + 1] = nseg_in[g] + in.n_nodes[g0 + g];
    E_in += Eg;
    T_in += Tg;
  }
  if (nseg_in[G] > 0x7fffffffLL) return fail(MOCHY_E_UNSUPPORTED, "too many nodes in a batch");
  if (E_in > MOCHY_MAX_EDGES) return fail(MOCHY_E_UNSUPPORTED, "too many hyperedges in a batch");
  std::vector<int64_t> off((size_t)E_in + 1);
  std::vector<int32_t> nodes((size_t)std::max<int64_t>(T_in, 1));
  {
    int64_t e = 0, t = 0;
    for (int g = 0; g < G; ++g) {
      const int64_t Eg = in.n_edges[g0 + g], Ng = in.n_nodes[g0 + g];
      const int64_t* o = in.off[g0 + g];
      const int32_t* nd = in.nodes[g0 + g];
      if (Eg == 0) continue;
      for (int64_t k = 0; k < Eg; ++k) {
        if (o[k + 1] < o[k]) return fail(MOCHY_E_INVALID, "offsets decrease");
        off[e + k] = t + o[k];
      }
      for (int64_t q = 0; q < o[Eg]; ++q) {
        if (nd[q] < 0 || nd[q] >= Ng) return fail(MOCHY_E_INVALID, "node id out of range");
        nodes[t + q] = (int32_t)(nd[q] + nseg_in[g]);
      }
      e += Eg;
      t += o[Eg];
    }
    off[E_in] = t;
  }
  MOCHY_TRY(mochy_load(ci, nseg_in[G], E_in, off.data(), nodes.data(), nullptr));
  MOCHY_TRY(set_units(ci, nseg_in));
  // 2. every unit's pairs
  std::vector<int64_t> eoff_in((size_t)ci->n_edges + 1);
  MOCHY_CUDA(cudaMemcpyAsync(eoff_in.data(), ci->eoff, eoff_in.size() * 8, cudaMemcpyDeviceToHost,
                             st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  std::vector<GraphRow> graphs((size_t)G);
  for (int g = 0; g < G; ++g) {
    GraphRow& r = graphs[g];
    r.n0 = nseg_in[g];
    r.N = nseg_in[g + 1] - nseg_in[g];
    r.e0 = ci->h_eseg[g];
    r.E = ci->h_eseg[g + 1] - ci->h_eseg[g];
    r.t0 = eoff_in[r.e0];
    r.T = eoff_in[r.e0 + r.E] - r.t0;
    r.seed = in.seeds[g0 + g];
  }
  std::vector<UnitRow> units((size_t)U);
  std::vector<int64_t> pp((size_t)U + 1, 0), nseg((size_t)U + 1, 0);
  int64_t eb = 0;
  for (int u = 0; u < U; ++u) {
    const GraphRow& r = graphs[u / R1];
    units[u] = UnitRow{pp[u], nseg[u], eb, (int32_t)(u / R1), (int32_t)(u % R1) - 1};
    pp[u + 1] = pp[u] + r.T;
    nseg[u + 1] = nseg[u] + r.N;
    eb += r.E;
  }
  const int64_t P = pp[U];
  if (nseg[U] > 0x7fffffffLL) return fail(MOCHY_E_UNSUPPORTED, "too many nodes in a batch");
  if (eb > MOCHY_MAX_EDGES) return fail(MOCHY_E_UNSUPPORTED, "too many hyperedges in a batch");
  Ctx cu;
  MOCHY_TRY(mochy_create(&cu.c, &cfg));
  mochy_ctx* cx = cu.c;
  {
    // tables and pairs in the input context's scratch slot 2 (the transform
    // takes slots 0, 1 and 3)
    const size_t b_units = ((size_t)U * sizeof(UnitRow) + 255) & ~(size_t)255;
    const size_t b_graphs = ((size_t)G * sizeof(GraphRow) + 255) & ~(size_t)255;
    const size_t b_pp = ((size_t)(U + 1) * 8 + 255) & ~(size_t)255;
    const size_t b_pair = ((size_t)std::max<int64_t>(P, 1) * 4 + 255) & ~(size_t)255;
    void* sp;
    MOCHY_TRY(scratch(ci, 2, b_units + b_graphs + b_pp + 2 * b_pair, &sp));
    char* c = (char*)sp;
    UnitRow* d_units = (UnitRow*)c;
    GraphRow* d_graphs = (GraphRow*)(c + b_units);
    int64_t* d_pp = (int64_t*)(c + b_units + b_graphs);
    uint32_t* d_node = (uint32_t*)(c + b_units + b_graphs + b_pp);
    uint32_t* d_edge = (uint32_t*)(c + b_units + b_graphs + b_pp + b_pair);
    MOCHY_CUDA(cudaMemcpyAsync(d_units, units.data(), (size_t)U * sizeof(UnitRow),
                               cudaMemcpyHostToDevice, st));
    MOCHY_CUDA(cudaMemcpyAsync(d_graphs, graphs.data(), (size_t)G * sizeof(GraphRow),
                               cudaMemcpyHostToDevice, st));
    MOCHY_CUDA(cudaMemcpyAsync(d_pp, pp.data(), (size_t)(U + 1) * 8, cudaMemcpyHostToDevice, st));
    if (P > 0) {
      k_batch_pairs<<<ceil_div(P, 256), 256, 0, st>>>(P, d_pp, U, d_units, d_graphs, ci->eoff,
                                                      ci->enode, ci->voff, d_node, d_edge);
      MOCHY_LAUNCHED();
      // 3. sets per hyperedge, empty ones dropped, loaded (repeats dropped)
      MOCHY_TRY(pairs_to_hypergraph(ci, d_node, d_edge, P, nseg[U], eb, cx));
    } else {
      MOCHY_TRY(load_graph(cx, nseg[U], 0, nullptr, nullptr, nullptr));
    }
  }
  MOCHY_TRY(set_units(cx, nseg));
  cudaEventRecord(ev.e[1], cx->stream);
  // 4. the union's line graph and split structures
  MOCHY_TRY(project_graph(cx));
  cudaEventRecord(ev.e[2], cx->stream);
  MOCHY_TRY(prepare_split(cx));
  cudaEventRecord(ev.e[3], cx->stream);
  // 5. one graph launch counts every unit
  const size_t b_hist = (size_t)U * 432 * 8;
  const size_t b_cnt = (size_t)U * 457 * 8;
  const size_t b_out = (size_t)G * 2 * 457 * 8;
  Block blk{cx};
  blk.b = b_hist + b_cnt + b_out + (size_t)G * 8 + 64;
  MOCHY_TRY(dev_alloc(cx, &blk.p, blk.b));
  char* hb = (char*)blk.p;
  unsigned long long* d_hist = (unsigned long long*)hb;
  int64_t* d_ch = (int64_t*)(hb + b_hist);
  int64_t* d_c3 = d_ch + (size_t)U * MOCHY_N_H;
  double* d_out = (double*)(hb + b_hist + b_cnt);
  int32_t* d_deg = (int32_t*)(hb + b_hist + b_cnt + b_out);
  int32_t* d_bad = d_deg + 2 * G;
  float count_ms = 0.f;
  MOCHY_TRY(count_split_graph(cx, d_hist, &count_ms));
  cudaEventRecord(ev.e[4], cx->stream);
  // 6. per-unit counts, then each input's significance and CP
  MOCHY_CUDA(cudaMemsetAsync(d_bad, 0, 4, cx->stream));
  MOCHY_TRY(finish_counts_batch(cx, d_hist, U, d_ch, d_c3, d_bad));
  MOCHY_TRY(significance_cp_batch(cx, d_ch, d_c3, G, R, cx->eps, d_out, d_deg));
  std::vector<int64_t> hc((size_t)U * 457);
  std::vector<double> ho((size_t)G * 2 * 457);
  std::vector<int32_t> hd((size_t)2 * G + 1);
  MOCHY_CUDA(cudaMemcpyAsync(hc.data(), d_ch, b_cnt, cudaMemcpyDeviceToHost, cx->stream));
  MOCHY_CUDA(cudaMemcpyAsync(ho.data(), d_out, b_out, cudaMemcpyDeviceToHost, cx->stream));
  MOCHY_CUDA(cudaMemcpyAsync(hd.data(), d_deg, (size_t)(2 * G + 1) * 4, cudaMemcpyDeviceToHost,
                             cx->stream));
  cudaEventRecord(ev.e[5], cx->stream);
  MOCHY_CUDA(cudaStreamSynchronize(cx->stream));
  if (hd[2 * G]) return fail(MOCHY_E_CUDA, "internal error: an instance mapped to no motif");
  const int64_t* ch = hc.data();
  const int64_t* c3 = ch + (size_t)U * MOCHY_N_H;
  int64_t instances = 0;
  for (size_t q = 0; q < (size_t)U * MOCHY_N_H; ++q) instances += ch[q];
  for (int g = 0; g < G; ++g) {
    const size_t gg = (size_t)(g0 + g);
    const double* o = ho.data() + (size_t)g * 2 * 457;
    if (out.sig_h) memcpy(out.sig_h + gg * MOCHY_N_H, o, MOCHY_N_H * 8);
    if (out.cp_h) memcpy(out.cp_h + gg * MOCHY_N_H, o + MOCHY_N_H, MOCHY_N_H * 8);
    if (out.sig_3h) memcpy(out.sig_3h + gg * MOCHY_N_3H, o + 2 * MOCHY_N_H, MOCHY_N_3H * 8);
    if (out.cp_3h)
      memcpy(out.cp_3h + gg * MOCHY_N_3H, o + 2 * MOCHY_N_H + MOCHY_N_3H, MOCHY_N_3H * 8);
    if (out.counts_h)
      memcpy(out.counts_h + gg * R1 * MOCHY_N_H, ch + (size_t)g * R1 * MOCHY_N_H,
             (size_t)R1 * MOCHY_N_H * 8);
    if (out.counts_3h)
      memcpy(out.counts_3h + gg * R1 * MOCHY_N_3H, c3 + (size_t)g * R1 * MOCHY_N_3H,
             (size_t)R1 * MOCHY_N_3H * 8);
    const bool dg = hd[2 * g] || hd[2 * g + 1];
    if (out.degenerate) out.degenerate[gg] = dg ? 1 : 0;
    out.any_degenerate = out.any_degenerate || dg;
  }
  if (out.info) {
    mochy_batch_info& b = *out.info;
    b.ms_generate += ms_since(ev.e[0], ev.e[1]);
    b.ms_project += ms_since(ev.e[1], ev.e[2]);
    b.ms_prepare += ms_since(ev.e[2], ev.e[3]);
    b.ms_count += (double)count_ms;
    b.ms_finish += ms_since(ev.e[4], ev.e[5]);
    b.n_waves += 1;
    b.n_units += U;
    b.max_units_per_wave = std::max<int64_t>(b.max_units_per_wave, U);
    b.n_edges += cx->n_edges;
    b.n_wedges += cx->n_wedges;
    b.instances += instances;
    b.dense_threshold = cx->dense_thr_used;
  }
  return MOCHY_OK;
}

}  // namespace

// Upper estimate of the device memory one hypergraph needs while it is
// counted: its line graph has at most sum_v C(d_v, 2) hyperwedges (16 bytes
// each), plus per-hyperedge, per-incidence and per-node arrays.
int64_t estimate_graph_bytes(int64_t n_nodes, int64_t n_edges, const int64_t* off,
                             const int32_t* nodes) {
  std::vector<int64_t> deg((size_t)std::max<int64_t>(n_nodes, 0), 0);
  const int64_t T = n_edges > 0 ? off[n_edges] : 0;
  for (int64_t q = 0; q < T; ++q) {
    const int32_t v = nodes[q];
    if (v >= 0 && v < n_nodes) ++deg[(size_t)v];
  }
  double w = 0.0;
  for (int64_t d : deg) w += 0.5 * (double)d * (double)(d - 1);
  return (int64_t)(16.0 * w + 96.0 * (double)n_edges + 48.0 * (double)T +
                   16.0 * (double)n_nodes) + (1 << 20);
}

}  // namespace mochy

using namespace mochy;

extern "C" int mochy_profile_batch(const mochy_config* cfg_in, int32_t n_graphs,
                                   const int64_t* n_nodes, const int64_t* n_edges,
                                   const int64_t* const* edge_offsets,
                                   const int32_t* const* edge_nodes, int32_t n_random,
                                   const uint64_t* seeds, double* sig_h, double* cp_h,
                                   double* sig_3h, double* cp_3h, int64_t* counts_h,
                                   int64_t* counts_3h, int32_t* degenerate,
                                   mochy_batch_info* info) {
  if (n_graphs <= 0) return fail(MOCHY_E_INVALID, "n_graphs must be positive");
  if (n_random <= 0) return fail(MOCHY_E_INVALID, "n_random must be positive");
  if (!n_nodes || !n_edges || !edge_offsets || !edge_nodes || !seeds)
    return fail(MOCHY_E_INVALID, "null argument");
  mochy_config cfg;
  mochy_config_default(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.exact_kernel != 0) return fail(MOCHY_E_UNSUPPORTED, "batches use the split exact count");
  cfg.stream = nullptr;   // the batch's contexts own their streams
  for (int32_t g = 0; g < n_graphs; ++g) {
    if (n_nodes[g] < 1 || n_edges[g] < 0) return fail(MOCHY_E_INVALID, "bad hypergraph size");
    if (n_edges[g] > 0 && (!edge_offsets[g] || !edge_nodes[g]))
      return fail(MOCHY_E_INVALID, "null array");
  }
  if (info) memset(info, 0, sizeof(*info));
  // waves: inputs in order, as many per wave as the memory estimate allows
  // (estimate_graph_bytes per hypergraph and copy); the budget is the
  // configured one, else 70% of the device memory free now.
  int64_t budget = cfg.hbm_budget_bytes;
  if (budget <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(cfg.device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      return fail(MOCHY_E_CUDA, "cannot query device memory");
    }
    budget = (int64_t)((double)fr * 0.7);
  }
  std::vector<int64_t> est((size_t)n_graphs);
  for (int32_t g = 0; g < n_graphs; ++g)
    est[g] = (int64_t)(n_random + 1) *
             estimate_graph_bytes(n_nodes[g], n_edges[g], edge_offsets[g], edge_nodes[g]);
  // MOCHY_BATCH_MAX_GRAPHS caps the inputs per wave (smaller unions)
  int32_t cap = n_graphs;
  if (const char* e = getenv("MOCHY_BATCH_MAX_GRAPHS")) {
    const long v = strtol(e, nullptr, 10);
    if (v > 0) cap = (int32_t)std::min<long>(v, n_graphs);
  }
  Inputs in{n_nodes, n_edges, edge_offsets, edge_nodes, seeds};
  Outputs out{sig_h, cp_h, sig_3h, cp_3h, counts_h, counts_3h, degenerate, info, false};
  int32_t g0 = 0;
  while (g0 < n_graphs) {
    int32_t g1 = g0 + 1;
    int64_t bytes = est[g0], edges = (int64_t)(n_random + 1) * n_edges[g0];
    while (g1 < n_graphs && g1 - g0 < cap && bytes + est[g1] <= budget &&
           edges + (int64_t)(n_random + 1) * n_edges[g1] <= MOCHY_MAX_EDGES) {
      bytes += est[g1];
      edges += (int64_t)(n_random + 1) * n_edges[g1];
      ++g1;
    }
    MOCHY_TRY(run_wave(cfg, in, g0, g1, n_random, out));
    g0 = g1;
  }
  return out.any_degenerate ? MOCHY_W_DEGENERATE_CP : MOCHY_OK;
}

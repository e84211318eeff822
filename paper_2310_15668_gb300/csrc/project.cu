// Line-graph construction (Section 2.1 "Line Graph"; Algorithm
// "hyperwedge_counting", Section 3.1).
//
// The paper visits, for each e_i and each v in e_i, every e_j in E_v and
// increments omega(e_i, e_j) in a hash map.  Here one CTA builds row e_i of
// the line graph: it walks the incidence lists E_v of the nodes of e_i in
// windows of neighbour ids, ORs bit p into a shared word per neighbour when
// the p-th node of e_i lies in it (so omega = popc of the word), and compacts
// the non-zero words in id order.  Two passes: sizes, then entries.
#include "common.cuh"

namespace mochy {
namespace {

constexpr int kProjThreads = 256;
constexpr int kProjWarps = kProjThreads / 32;
constexpr int kWin = 8192;                       // neighbour ids per window
constexpr int kPerThread = kWin / kProjThreads;  // words scanned per thread

template <bool FILL>
__global__ void __launch_bounds__(kProjThreads)
k_project_rows(int64_t n_edges, const int64_t* __restrict__ eoff,
               const int32_t* __restrict__ enode, const int64_t* __restrict__ voff,
               const int32_t* __restrict__ vedge, const uint8_t* __restrict__ esize,
               int64_t* __restrict__ deg_out, int64_t* __restrict__ below_out,
               const int64_t* __restrict__ noff, uint2* __restrict__ nadj) {
  __shared__ uint32_t word[kWin];
  __shared__ int64_t cur[MOCHY_MAX_EDGE_SIZE], endp[MOCHY_MAX_EDGE_SIZE];
  __shared__ int64_t ws[34];
  __shared__ int next_id;
  __shared__ unsigned long long below_acc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t i = blockIdx.x; i < n_edges; i += gridDim.x) {
    const int64_t eb = eoff[i];
    const int s = (int)(eoff[i + 1] - eb);
    const bool masked = s <= kMaskedMax;
    if (threadIdx.x < s) {
      const int32_t v = enode[eb + threadIdx.x];
      cur[threadIdx.x] = voff[v];
      endp[threadIdx.x] = voff[v + 1];
    }
    if (threadIdx.x == 0) below_acc = 0ull;
    int64_t count = 0;
    const int64_t out_base = FILL ? noff[i] : 0;
    __syncthreads();
    while (true) {
      if (threadIdx.x == 0) next_id = 0x7fffffff;
      __syncthreads();
      if (threadIdx.x < s && cur[threadIdx.x] < endp[threadIdx.x])
        atomicMin(&next_id, vedge[cur[threadIdx.x]]);
      __syncthreads();
      const int nid = next_id;
      if (nid == 0x7fffffff) break;
      const int64_t w0 = ((int64_t)nid / kWin) * kWin;
      for (int q = threadIdx.x; q < kWin; q += kProjThreads) word[q] = 0u;
      __syncthreads();
      // accumulate the window: warp w walks the lists of nodes w, w+8, ...
      for (int p = warp; p < s; p += kProjWarps) {
        int64_t c = cur[p];
        const int64_t e = endp[p];
        while (true) {
          const int64_t q = c + lane;
          const int32_t k = q < e ? vedge[q] : 0x7fffffff;
          const bool in = (int64_t)k < w0 + kWin;
          if (in && (int64_t)k != i) {
            if (masked) atomicOr(&word[k - w0], 1u << p);
            else atomicAdd(&word[k - w0], 1u);
          }
          const int n = __popc(__ballot_sync(0xffffffffu, in));
          c += n;
          if (n < 32) break;
        }
        if (lane == 0) cur[p] = c;
      }
      __syncthreads();
      // compact non-zero words in id order
      const int base = threadIdx.x * kPerThread;
      int cnt = 0, blo = 0;
#pragma unroll 4
      for (int q = 0; q < kPerThread; ++q) {
        if (word[base + q]) {
          ++cnt;
          if (w0 + base + q < i) ++blo;
        }
      }
      int64_t total;
      const int64_t pre = block_scan_i64(cnt, ws, &total);
      if (blo) atomicAdd(&below_acc, (unsigned long long)blo);
      if (FILL) {
        int64_t o = out_base + count + pre;
        for (int q = 0; q < kPerThread; ++q) {
          const uint32_t w = word[base + q];
          if (w) {
            const int64_t k = w0 + base + q;
            nadj[o++] = make_uint2((uint32_t)k | ((uint32_t)esize[k] << kIdBits), w);
          }
        }
      }
      count += total;
      __syncthreads();
    }
    if (!FILL && threadIdx.x == 0) {
      deg_out[i] = count;
      below_out[i] = (int64_t)below_acc;
    }
    __syncthreads();
  }
}

__global__ void k_upper(int64_t n_edges, const int64_t* __restrict__ noff,
                        const int64_t* __restrict__ deg, const int64_t* __restrict__ below,
                        int64_t* __restrict__ ustart, int64_t* __restrict__ uplen,
                        int* __restrict__ maxdeg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_edges) return;
  ustart[i] = noff[i] + below[i];
  uplen[i] = deg[i] - below[i];
  atomicMax(maxdeg, (int)deg[i]);
}

// Estimated work of staging row a in the exact count: the neighbours' row
// lengths it will scan.  Keys sort rows by decreasing work.
__global__ void k_row_cost(int64_t n_edges, const int64_t* __restrict__ noff,
                           const uint2* __restrict__ nadj, uint32_t* __restrict__ key,
                           uint32_t* __restrict__ val) {
  const int64_t a = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= n_edges) return;
  double c = 0.0;
  for (int64_t p = noff[a] + lane; p < noff[a + 1]; p += 32) {
    const uint32_t b = ent_id(nadj[p]);
    c += (double)(noff[b + 1] - noff[b]);
  }
  for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  c += (double)(noff[a + 1] - noff[a]);
  if (lane == 0) {
    key[a] = ~__float_as_uint((float)c);
    val[a] = (uint32_t)a;
  }
}

// unit of each row of an order (rows of a batch)
__global__ void k_row_units(int64_t n, const uint32_t* __restrict__ row,
                            const int64_t* __restrict__ eoff, const int32_t* __restrict__ enode,
                            const int64_t* __restrict__ nseg, int n_units,
                            uint32_t* __restrict__ unit) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) unit[i] = (uint32_t)seg_of(nseg, n_units, enode[eoff[row[i]]]);
}

}  // namespace

int project_graph(mochy_ctx* ctx) {
  release_projection(ctx);
  const int64_t E = ctx->n_edges;
  cudaStream_t st = ctx->stream;
  void* p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int64_t) * (size_t)(E + 1)));
  ctx->noff = (int64_t*)p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int64_t) * (size_t)std::max<int64_t>(E, 1)));
  ctx->ustart = (int64_t*)p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int64_t) * (size_t)(E + 1)));
  ctx->uprefix = (int64_t*)p;
  MOCHY_TRY(dev_alloc(ctx, &p, sizeof(int32_t) * (size_t)std::max<int64_t>(E, 1)));
  ctx->row_order = (int32_t*)p;
  if (E == 0) {
    MOCHY_CUDA(cudaMemsetAsync(ctx->noff, 0, 8, st));
    MOCHY_CUDA(cudaMemsetAsync(ctx->uprefix, 0, 8, st));
    ctx->n_wedges = 0;
    ctx->max_deg = 0;
    ctx->projected = true;
    return MOCHY_OK;
  }
  void* t;
  MOCHY_TRY(scratch(ctx, 0, (size_t)(E + 1) * 8 * 3, &t));
  int64_t* deg = (int64_t*)t;
  int64_t* below = deg + (E + 1);
  int64_t* uplen = below + (E + 1);
  MOCHY_CUDA(cudaMemsetAsync(deg, 0, (size_t)(E + 1) * 8 * 3, st));
  const unsigned grid = (unsigned)std::min<int64_t>(E, 1 << 20);
  k_project_rows<false><<<grid, kProjThreads, 0, st>>>(E, ctx->eoff, ctx->enode, ctx->voff,
                                                       ctx->vedge, ctx->esize, deg, below,
                                                       nullptr, nullptr);
  MOCHY_LAUNCHED();
  MOCHY_TRY(scan_exclusive_i64(ctx, deg, ctx->noff, E + 1));
  int64_t total = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&total, ctx->noff + E, 8, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  const size_t bytes = (size_t)std::max<int64_t>(total, 1) * sizeof(uint2);
  int rc = dev_alloc(ctx, &p, bytes);
  if (rc < 0) {
    release_projection(ctx);
    return fail(MOCHY_E_NOMEM, "line graph needs " + std::to_string(bytes) +
                                   " bytes of device memory");
  }
  ctx->nadj = (uint2*)p;
  k_project_rows<true><<<grid, kProjThreads, 0, st>>>(E, ctx->eoff, ctx->enode, ctx->voff,
                                                      ctx->vedge, ctx->esize, nullptr, nullptr,
                                                      ctx->noff, ctx->nadj);
  MOCHY_LAUNCHED();
  int* maxdeg = ctx->counters + 2;
  MOCHY_CUDA(cudaMemsetAsync(maxdeg, 0, 4, st));
  k_upper<<<ceil_div(E, 256), 256, 0, st>>>(E, ctx->noff, deg, below, ctx->ustart, uplen, maxdeg);
  MOCHY_LAUNCHED();
  MOCHY_TRY(scan_exclusive_i64(ctx, uplen, ctx->uprefix, E + 1));
  // rows by decreasing estimated work, for the exact count's work queue
  void* t2;
  MOCHY_TRY(scratch(ctx, 2, (size_t)E * 8, &t2));
  uint32_t* key = (uint32_t*)t2;
  uint32_t* val = key + E;
  k_row_cost<<<ceil_div(E, 8), 256, 0, st>>>(E, ctx->noff, ctx->nadj, key, val);
  MOCHY_LAUNCHED();
  MOCHY_TRY(radix_sort_pairs_u32(ctx, key, val, E, 32));
  if (ctx->n_units > 1) {
    // a batch: rows grouped by hypergraph (stable), so that a block's
    // consecutive rows mostly belong to one of them
    k_row_units<<<ceil_div(E, 256), 256, 0, st>>>(E, val, ctx->eoff, ctx->enode, ctx->d_nseg,
                                                  ctx->n_units, key);
    MOCHY_LAUNCHED();
    MOCHY_TRY(radix_sort_pairs_u32(ctx, key, val, E, bits_for(ctx->n_units)));
  }
  MOCHY_CUDA(cudaMemcpyAsync(ctx->row_order, val, (size_t)E * 4, cudaMemcpyDeviceToDevice, st));
  int32_t md = 0;
  MOCHY_CUDA(cudaMemcpyAsync(&md, maxdeg, 4, cudaMemcpyDeviceToHost, st));
  MOCHY_CUDA(cudaStreamSynchronize(st));
  ctx->n_wedges = total / 2;
  ctx->max_deg = md;
  ctx->projected = true;
  return MOCHY_OK;
}

}  // namespace mochy

// Device-wide building blocks: exclusive scan of int64 and a stable LSD
// radix sort of (uint32 key, uint32 value) pairs.  Both are plain multi-pass
// kernels on the context's stream.
#include "common.cuh"

namespace mochy {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x a multiple
// of 32, at most 1024); the block total is returned through *total.
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t warp_base[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
    const int64_t s = lane < nw ? warp_sums[lane] : 0;
    const int64_t si = warp_incl_scan(s);
    warp_base[lane] = si - s;
    if (lane == 31) warp_base[32] = si;
  }
  __syncthreads();
  const int64_t res = warp_base[warp] + inc - v;
  *total = warp_base[32];
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(const int64_t* __restrict__ in, int64_t n,
                                int64_t* __restrict__ partial) {
  const int64_t tile = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = tile + (int64_t)threadIdx.x * kScanItems + r;
    if (i < n) s += in[i];
  }
  int64_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// One block scans the partial sums in place (exclusive), tile by tile.
__global__ void __launch_bounds__(kScanThreads) k_scan_partials_scan(int64_t* partial, int64_t nb) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? partial[i] : 0;
    int64_t total;
    int64_t ex = block_excl_scan(v, &total);
    int64_t c = carry;
    if (i < nb) partial[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int64_t* __restrict__ in, int64_t n,
                             const int64_t* __restrict__ partial, int64_t* __restrict__ out) {
  const int64_t tile = (int64_t)blockIdx.x * kScanTile;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = tile + (int64_t)threadIdx.x * kScanItems + r;
    v[r] = i < n ? in[i] : 0;
    s += v[r];
  }
  int64_t total;
  int64_t ex = block_excl_scan(s, &total) + partial[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = tile + (int64_t)threadIdx.x * kScanItems + r;
    if (i < n) out[i] = ex;
    ex += v[r];
  }
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, tiles of 256 threads x 8 items in striped order
// (item r*256 + t), ranks made stable by per-round warp counts.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                            int64_t* __restrict__ hist, int nblocks) {
  __shared__ unsigned int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t tile = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = tile + (int64_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                               int64_t n, int shift, const int64_t* __restrict__ offs,
                               int nblocks) {
  __shared__ unsigned int running[256];
  __shared__ unsigned int wcnt[kSortWarps][257];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  running[threadIdx.x] = 0;
  for (int d = threadIdx.x; d < kSortWarps * 257; d += kSortThreads)
    (&wcnt[0][0])[d] = 0xffffffffu;
  __syncthreads();
  const int64_t tile = (int64_t)blockIdx.x * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = tile + (int64_t)r * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    uint32_t val = valid ? vin[i] : 0u;
    const unsigned d = valid ? ((key >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lt);
    const bool leader = (peers & lt) == 0;
    if (leader) wcnt[warp][d] = ((unsigned)r << 16) | (unsigned)__popc(peers);
    __syncthreads();
    if (valid) {
      unsigned before = 0;
      for (int w = 0; w < warp; ++w) {
        unsigned c = wcnt[w][d];
        if ((c >> 16) == (unsigned)r) before += c & 0xffffu;
      }
      const int64_t pos = offs[(int64_t)d * nblocks + blockIdx.x] + running[d] + before + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    if (valid && leader) atomicAdd(&running[d], (unsigned)__popc(peers));
    __syncthreads();
  }
}

}  // namespace

// bits needed for keys below n
int bits_for(int64_t n) {
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) < n) ++b;
  return b;
}

int scan_exclusive_i64(mochy_ctx* ctx, const int64_t* d_in, int64_t* d_out, int64_t n) {
  if (n <= 0) return MOCHY_OK;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  void* part = nullptr;
  MOCHY_TRY(scratch(ctx, 3, sizeof(int64_t) * (size_t)nb, &part));
  int64_t* partial = (int64_t*)part;
  k_scan_partials<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(d_in, n, partial);
  MOCHY_LAUNCHED();
  k_scan_partials_scan<<<1, kScanThreads, 0, ctx->stream>>>(partial, nb);
  MOCHY_LAUNCHED();
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(d_in, n, partial, d_out);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

int radix_sort_pairs_u32(mochy_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n,
                         int key_bits) {
  if (n <= 1) return MOCHY_OK;
  const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
  const int64_t nh = (int64_t)256 * nblocks;
  // scratch slot 3 is used by the scan, so this function takes slots 1 and 2
  void* tmp = nullptr;
  MOCHY_TRY(scratch(ctx, 1, (size_t)n * 8 + (size_t)nh * 16, &tmp));
  uint32_t* k2 = (uint32_t*)tmp;
  uint32_t* v2 = k2 + n;
  int64_t* hist = (int64_t*)((char*)tmp + (size_t)n * 8);
  int64_t* offs = hist + nh;
  uint32_t *kin = keys, *vin = vals, *kout = k2, *vout = v2;
  const int passes = (key_bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_sort_hist<<<nblocks, kSortThreads, 0, ctx->stream>>>(kin, n, shift, hist, nblocks);
    MOCHY_LAUNCHED();
    MOCHY_TRY(scan_exclusive_i64(ctx, hist, offs, nh));
    k_sort_scatter<<<nblocks, kSortThreads, 0, ctx->stream>>>(kin, vin, kout, vout, n, shift,
                                                              offs, nblocks);
    MOCHY_LAUNCHED();
    uint32_t* t;
    t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
  }
  if (kin != keys) {
    MOCHY_CUDA(cudaMemcpyAsync(keys, kin, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    MOCHY_CUDA(cudaMemcpyAsync(vals, vin, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return MOCHY_OK;
}

}  // namespace mochy

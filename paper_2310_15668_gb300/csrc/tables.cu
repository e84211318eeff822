// Motif lookup tables, built on the device once per context.
//
// A pattern assigns a state to each of the seven Venn regions of three
// hyperedges (Section 2.2; regions (1) i only, (2) j only, (3) k only,
// (4) i&j, (5) j&k, (6) k&i, (7) i&j&k).  h-motifs use states {0, 1}
// (empty / not), 3h-motifs {0, 1, 2} (empty / at most theta / more,
// Section 4.1).  Patterns equal up to a re-labelling of the three hyperedges
// are one motif; the representative is the lexicographically smallest state
// tuple (the P_1 rule of the appendix on motifs of k hyperedges).  Patterns of
// disconnected or non-distinct hyperedges are no motif.
//
// Numbering (the figures that fix it are lost): h-motifs 1-16 closed with a
// non-empty triple region, 17-22 open, 23-26 closed with an empty triple
// region, each in ascending tuple order; 3h-motifs in ascending (h-motif id,
// tuple) order.
#include "common.cuh"

namespace mochy {
namespace {

// membership bits (i = 1, j = 2, k = 4) of regions (1)..(7)
__constant__ int c_member[7] = {1, 2, 4, 3, 6, 5, 7};

__device__ int region_of_member(int m) {
  switch (m) {
    case 1: return 0; case 2: return 1; case 4: return 2; case 3: return 3;
    case 6: return 4; case 5: return 5; default: return 6;
  }
}

// state of region r in the little-endian code (digit r has weight base^r)
__device__ int digit(int code, int base, int r) {
  for (int q = 0; q < r; ++q) code /= base;
  return code % base;
}

// lexicographic key: region (1) most significant
__device__ int lex_key(const int* st, int base) {
  int k = 0;
  for (int r = 0; r < 7; ++r) k = k * base + st[r];
  return k;
}

__device__ void permute_roles(const int* st, int perm_id, int* out) {
  // images of the roles i, j, k under the six permutations
  const int img[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int r = 0; r < 7; ++r) {
    int m = c_member[r], m2 = 0;
    for (int b = 0; b < 3; ++b)
      if (m & (1 << b)) m2 |= 1 << img[perm_id][b];
    out[region_of_member(m2)] = st[r];
  }
}

__device__ int canonical_key(int code, int base) {
  int st[7], q[7];
  for (int r = 0; r < 7; ++r) st[r] = digit(code, base, r);
  int best = 0x7fffffff;
  for (int p = 0; p < 6; ++p) {
    permute_roles(st, p, q);
    int k = lex_key(q, base);
    best = k < best ? k : best;
  }
  return best;
}

// does some non-empty region contain both roles of `pair`?
__device__ bool meets(const int* st, int pair_bits) {
  for (int r = 0; r < 7; ++r)
    if (st[r] && (c_member[r] & pair_bits) == pair_bits) return true;
  return false;
}

__device__ int classify_pattern(int code, int base, int* group) {
  int st[7];
  for (int r = 0; r < 7; ++r) st[r] = digit(code, base, r);
  const bool ij = meets(st, 3), jk = meets(st, 6), ki = meets(st, 5);
  const int npairs = (int)ij + (int)jk + (int)ki;
  bool valid = npairs >= 2;
  // e_x == e_y exactly when every region holding one of x, y but not both is empty
  const int pairs[3] = {3, 6, 5};
  for (int q = 0; q < 3 && valid; ++q) {
    bool same = true;
    for (int r = 0; r < 7; ++r) {
      const int m = c_member[r] & pairs[q];
      if (st[r] && (m == 1 || m == 2 || m == 4)) same = false;
    }
    if (same) valid = false;
  }
  *group = npairs == 3 ? (st[6] ? 0 : 2) : 1;
  return valid ? 1 : 0;
}

// One block of 512 threads builds everything.
__global__ void __launch_bounds__(512) k_build_tables(uint16_t* lut3, uint8_t* t2h, uint8_t* hopen,
                               uint8_t* pat2, uint8_t* pat3) {
  __shared__ int key2[128], ok2[128], grp2[128], hid2[128];
  __shared__ int key3[2187];
  __shared__ unsigned char ok3[2187];
  __shared__ int hid3[2187];
  const int t = threadIdx.x;
  for (int c = t; c < 128; c += blockDim.x) {
    key2[c] = canonical_key(c, 2);
    int g;
    ok2[c] = classify_pattern(c, 2, &g);
    grp2[c] = g;
  }
  for (int c = t; c < 2187; c += blockDim.x) {
    key3[c] = canonical_key(c, 3);
    int g;
    ok3[c] = (unsigned char)classify_pattern(c, 3, &g);
  }
  __syncthreads();
  // h ids: rank of (group, key) among valid canonical representatives
  for (int c = t; c < 128; c += blockDim.x) {
    int id = 0;
    if (ok2[c]) {
      id = 1;
      for (int d = 0; d < 128; ++d) {
        if (!ok2[d]) continue;
        int st[7];
        for (int r = 0; r < 7; ++r) st[r] = digit(d, 2, r);
        if (lex_key(st, 2) != key2[d]) continue;  // not a representative
        if (grp2[d] < grp2[c] || (grp2[d] == grp2[c] && key2[d] < key2[c])) ++id;
      }
    }
    hid2[c] = id;
  }
  __syncthreads();
  // 3h: parent h id of each ternary code
  for (int c = t; c < 2187; c += blockDim.x) {
    int b = 0;
    for (int r = 0; r < 7; ++r) b |= (digit(c, 3, r) > 0 ? 1 : 0) << r;
    hid3[c] = ok3[c] ? hid2[b] : 0;
  }
  __syncthreads();
  for (int c = t; c < 2187; c += blockDim.x) {
    int id = 0;
    if (ok3[c]) {
      id = 1;
      for (int d = 0; d < 2187; ++d) {
        if (!ok3[d]) continue;
        int st[7];
        for (int r = 0; r < 7; ++r) st[r] = digit(d, 3, r);
        if (lex_key(st, 3) != key3[d]) continue;
        if (hid3[d] < hid3[c] || (hid3[d] == hid3[c] && key3[d] < key3[c])) ++id;
      }
    }
    lut3[c] = (uint16_t)id;
    if (id) {
      t2h[id] = (uint8_t)hid3[c];
      // the representative writes the pattern
      int st[7];
      for (int r = 0; r < 7; ++r) st[r] = digit(c, 3, r);
      if (lex_key(st, 3) == key3[c])
        for (int r = 0; r < 7; ++r) pat3[id * 7 + r] = (uint8_t)st[r];
    }
  }
  for (int c = t; c < 128; c += blockDim.x) {
    const int id = hid2[c];
    if (!id) continue;
    int st[7];
    for (int r = 0; r < 7; ++r) st[r] = digit(c, 2, r);
    if (lex_key(st, 2) == key2[c]) {
      for (int r = 0; r < 7; ++r) pat2[id * 7 + r] = (uint8_t)st[r];
      hopen[id] = grp2[c] == 1 ? 1 : 0;
    }
  }
}

// kh-motif tables (Section 4.1 "Extensions Beyond Ternary"), k states per
// region, k^7 <= 16384 codes; numbered like the 3h-motifs: ascending
// (parent h-motif id, canonical tuple).  Three passes over the codes.
// Pass 1: canonical key, validity, representative flag and parent h id (the
// h id of a binary pattern is read through the 3h tables: its 0/1 digits
// are a ternary code whose 3h-motif refines exactly that h-motif).
__global__ void k_kh_keys(int base, int n_codes, const uint16_t* __restrict__ lut3,
                          const uint8_t* __restrict__ t2h, int* __restrict__ key,
                          int* __restrict__ hid, unsigned char* __restrict__ rep) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_codes) return;
  int st[7];
  for (int r = 0; r < 7; ++r) st[r] = digit(c, base, r);
  key[c] = canonical_key(c, base);
  int g;
  const bool ok = classify_pattern(c, base, &g) != 0;
  int tc = 0, pw = 1;
  for (int r = 0; r < 7; ++r) {
    tc += (st[r] > 0 ? 1 : 0) * pw;
    pw *= 3;
  }
  hid[c] = ok ? (int)t2h[lut3[tc]] : 0;
  rep[c] = (unsigned char)(ok && lex_key(st, base) == key[c]);
}

// Pass 2: each representative's id is one plus the number of
// representatives before it in (h id, key) order.
__global__ void k_kh_rank(int base, int n_codes, const int* __restrict__ key,
                          const int* __restrict__ hid, const unsigned char* __restrict__ rep,
                          int* __restrict__ id_of_key, uint8_t* __restrict__ to_h,
                          uint8_t* __restrict__ pattern) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_codes || !rep[c]) return;
  int id = 1;
  for (int d = 0; d < n_codes; ++d)
    if (rep[d] && (hid[d] < hid[c] || (hid[d] == hid[c] && key[d] < key[c]))) ++id;
  id_of_key[key[c]] = id;
  to_h[id] = (uint8_t)hid[c];
  for (int r = 0; r < 7; ++r) pattern[id * 7 + r] = (uint8_t)digit(c, base, r);
}

// Pass 3: the id of every code is its representative's.
__global__ void k_kh_lut(int n_codes, const int* __restrict__ key, const int* __restrict__ hid,
                         const int* __restrict__ id_of_key, uint16_t* __restrict__ lut) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_codes) return;
  lut[c] = hid[c] ? (uint16_t)id_of_key[key[c]] : (uint16_t)0;
}

}  // namespace

// The kh-motif tables for k states (2 <= k <= 4) into ctx (built once per k
// and kept with the context).
int build_kh_tables(mochy_ctx* ctx, int k) {
  if (k < 2 || k > 4) return fail(MOCHY_E_UNSUPPORTED, "kh-motifs are provided for k = 2..4");
  if (ctx->kh_k == k) return MOCHY_OK;
  if (ctx->kh_block) {
    dev_free(ctx, ctx->kh_block, ctx->kh_bytes);
    ctx->kh_block = nullptr;
    ctx->kh_k = 0;
  }
  int n_codes = 1;
  for (int r = 0; r < 7; ++r) n_codes *= k;
  cudaStream_t st = ctx->stream;
  const size_t b_lut = ((size_t)n_codes * 2 + 255) & ~(size_t)255;
  const size_t b_toh = 4096, b_pat = 4096 * 7;
  const size_t bytes = b_lut + b_toh + b_pat;
  void* p = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &p, bytes));
  void* t = nullptr;
  const size_t b_tmp = (size_t)n_codes * (4 + 4 + 4 + 1) + 64;
  const int rc0 = dev_alloc(ctx, &t, b_tmp);
  if (rc0 < 0) {
    dev_free(ctx, p, bytes);
    return rc0;
  }
  int* key = (int*)t;
  int* hid = key + n_codes;
  int* id_of_key = hid + n_codes;
  unsigned char* rep = (unsigned char*)(id_of_key + n_codes);
  uint16_t* lut = (uint16_t*)p;
  uint8_t* to_h = (uint8_t*)p + b_lut;
  uint8_t* pat = to_h + b_toh;
  int rc = MOCHY_OK;
  if (cudaMemsetAsync(p, 0, bytes, st) != cudaSuccess ||
      cudaMemsetAsync(id_of_key, 0, (size_t)n_codes * 4, st) != cudaSuccess)
    rc = fail(MOCHY_E_CUDA, "kh table clear failed");
  const int nb = (n_codes + 255) / 256;
  if (rc == MOCHY_OK) {
    k_kh_keys<<<nb, 256, 0, st>>>(k, n_codes, ctx->tables.lut3, ctx->tables.t2h, key, hid, rep);
    note_launch();
    k_kh_rank<<<nb, 256, 0, st>>>(k, n_codes, key, hid, rep, id_of_key, to_h, pat);
    note_launch();
    k_kh_lut<<<nb, 256, 0, st>>>(n_codes, key, hid, id_of_key, lut);
    note_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "kh table kernels", __FILE__, __LINE__);
  }
  int n_motifs = 0;
  if (rc == MOCHY_OK) {
    // the number of motifs is the largest id, found on the host
    std::vector<uint16_t> h((size_t)n_codes);
    if (cudaMemcpyAsync(h.data(), lut, (size_t)n_codes * 2, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(MOCHY_E_CUDA, "kh table copy failed");
    } else {
      for (uint16_t v : h) n_motifs = std::max(n_motifs, (int)v);
    }
  }
  dev_free(ctx, t, b_tmp);
  if (rc != MOCHY_OK) {
    dev_free(ctx, p, bytes);
    return rc;
  }
  ctx->kh_block = p;
  ctx->kh_bytes = bytes;
  ctx->kh_lut = lut;
  ctx->kh_to_h = to_h;
  ctx->kh_pattern = pat;
  ctx->kh_k = k;
  ctx->kh_n = n_motifs;
  return MOCHY_OK;
}

// Process-wide host copy of the patterns (for mochy_motif_pattern).
static uint8_t g_pat2[27 * 7], g_pat3[432 * 7];
static bool g_have_patterns = false;

bool host_patterns(int kind, int32_t id, uint8_t* out) {
  if (!g_have_patterns) return false;
  if (kind == 2 && id >= 1 && id <= 26) {
    for (int r = 0; r < 7; ++r) out[r] = g_pat2[id * 7 + r];
    return true;
  }
  if (kind == 3 && id >= 1 && id <= 431) {
    for (int r = 0; r < 7; ++r) out[r] = g_pat3[id * 7 + r];
    return true;
  }
  return false;
}

int build_tables(mochy_ctx* ctx) {
  const size_t bytes = 2187 * 2 + 432 + 27 + 27 * 7 + 432 * 7;
  void* p = nullptr;
  MOCHY_TRY(dev_alloc(ctx, &p, bytes));
  MOCHY_CUDA(cudaMemsetAsync(p, 0, bytes, ctx->stream));
  uint8_t* b = (uint8_t*)p;
  ctx->tables.lut3 = (uint16_t*)b;
  ctx->tables.t2h = b + 2187 * 2;
  ctx->tables.hopen = ctx->tables.t2h + 432;
  uint8_t* pat2 = ctx->tables.hopen + 27;
  uint8_t* pat3 = pat2 + 27 * 7;
  k_build_tables<<<1, 512, 0, ctx->stream>>>(ctx->tables.lut3, ctx->tables.t2h,
                                              ctx->tables.hopen, pat2, pat3);
  MOCHY_LAUNCHED();
  if (!g_have_patterns) {
    MOCHY_CUDA(cudaMemcpyAsync(g_pat2, pat2, sizeof(g_pat2), cudaMemcpyDeviceToHost, ctx->stream));
    MOCHY_CUDA(cudaMemcpyAsync(g_pat3, pat3, sizeof(g_pat3), cudaMemcpyDeviceToHost, ctx->stream));
    MOCHY_CUDA(cudaStreamSynchronize(ctx->stream));
    g_have_patterns = true;
  }
  return MOCHY_OK;
}

}  // namespace mochy

// Final per-motif arithmetic on the device:
//  * h-motif counts as sums of their 3h-motif subdivisions (every 3h-motif
//    refines exactly one h-motif, Section 4.1);
//  * the rescaling of sampled counts (Algorithm "sampling_ver1": |E| / (3s);
//    Algorithm "sampling_ver2" and Eq. "mht:scale": |wedges| / (w[t] r) with
//    w = 2 for open and 3 for closed h-motifs, Eq. "wt");
//  * significance and characteristic profile (Eq. "significance", Eq. "cp",
//    Section 3.1) in FP64.
// Products and quotients use explicit round-to-nearest intrinsics, so no
// multiply-add is fused and the results do not depend on compiler contraction.
#include "common.cuh"

namespace mochy {
namespace {

__global__ void __launch_bounds__(512) k_finish(const unsigned long long* __restrict__ hist, const uint8_t* __restrict__ t2h,
                         int64_t* __restrict__ out_h, int64_t* __restrict__ out_3h,
                         int32_t* __restrict__ bad) {
  __shared__ unsigned long long h[27];
  if (threadIdx.x < 27) h[threadIdx.x] = 0ull;
  __syncthreads();
  for (int t = threadIdx.x + 1; t <= MOCHY_N_3H; t += blockDim.x) {
    out_3h[t - 1] = (int64_t)hist[t];
    atomicAdd(&h[t2h[t]], hist[t]);
  }
  __syncthreads();
  if (threadIdx.x < MOCHY_N_H) out_h[threadIdx.x] = (int64_t)h[threadIdx.x + 1];
  if (threadIdx.x == 0 && hist[0] != 0ull) *bad = 1;   // an instance with no motif id
}

__global__ void __launch_bounds__(512) k_scale(const int64_t* __restrict__ raw_h, const int64_t* __restrict__ raw_3h,
                        const uint8_t* __restrict__ t2h, const uint8_t* __restrict__ hopen,
                        int method, double numer, double samples, double* __restrict__ est_h,
                        double* __restrict__ est_3h) {
  const int t = threadIdx.x + blockIdx.x * blockDim.x;
  if (t < MOCHY_N_3H) {
    const double w = method == MOCHY_A ? 3.0 : (hopen[t2h[t + 1]] ? 2.0 : 3.0);
    est_3h[t] = __ddiv_rn(__dmul_rn((double)raw_3h[t], numer), __dmul_rn(w, samples));
  }
  if (t < MOCHY_N_H) {
    const double w = method == MOCHY_A ? 3.0 : (hopen[t + 1] ? 2.0 : 3.0);
    est_h[t] = __ddiv_rn(__dmul_rn((double)raw_h[t], numer), __dmul_rn(w, samples));
  }
}

// One block.  counts: (1 + R) rows of n values; out: sig[n] then cp[n].
__device__ void sig_cp(const int64_t* __restrict__ counts, int n, int R, double eps,
                       double* __restrict__ sig, double* __restrict__ cp, int32_t* degenerate,
                       double* red) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int64_t s = 0;
    for (int c = 1; c <= R; ++c) s += counts[(int64_t)c * n + t];
    const double mr = __ddiv_rn((double)s, (double)R);
    const double m = (double)counts[t];
    sig[t] = __ddiv_rn(__dsub_rn(m, mr), __dadd_rn(__dadd_rn(m, mr), eps));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ss = 0.0;
    for (int t = 0; t < n; ++t) ss = __dadd_rn(ss, __dmul_rn(sig[t], sig[t]));
    red[0] = sqrt(ss);
    *degenerate = ss == 0.0 ? 1 : 0;
  }
  __syncthreads();
  const double norm = red[0];
  for (int t = threadIdx.x; t < n; t += blockDim.x)
    cp[t] = norm == 0.0 ? 0.0 : __ddiv_rn(sig[t], norm);
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_sig_cp(const int64_t* __restrict__ counts_h, const int64_t* __restrict__ counts_3h,
                         int R, double eps, double* __restrict__ out, int32_t* __restrict__ deg) {
  __shared__ double red[1];
  sig_cp(counts_h, MOCHY_N_H, R, eps, out, out + MOCHY_N_H, deg, red);
  sig_cp(counts_3h, MOCHY_N_3H, R, eps, out + 2 * MOCHY_N_H, out + 2 * MOCHY_N_H + MOCHY_N_3H,
         deg + 1, red);
}

// A batch: block b finishes histogram b / computes the profile of graph b.
__global__ void __launch_bounds__(512) k_finish_batch(const unsigned long long* __restrict__ hist,
                                                      const uint8_t* __restrict__ t2h,
                                                      int64_t* __restrict__ out_h,
                                                      int64_t* __restrict__ out_3h,
                                                      int32_t* __restrict__ bad) {
  __shared__ unsigned long long h[27];
  const unsigned long long* hb = hist + (int64_t)blockIdx.x * 432;
  if (threadIdx.x < 27) h[threadIdx.x] = 0ull;
  __syncthreads();
  for (int t = threadIdx.x + 1; t <= MOCHY_N_3H; t += blockDim.x) {
    out_3h[(int64_t)blockIdx.x * MOCHY_N_3H + t - 1] = (int64_t)hb[t];
    atomicAdd(&h[t2h[t]], hb[t]);
  }
  __syncthreads();
  if (threadIdx.x < MOCHY_N_H)
    out_h[(int64_t)blockIdx.x * MOCHY_N_H + threadIdx.x] = (int64_t)h[threadIdx.x + 1];
  if (threadIdx.x == 0 && hb[0] != 0ull) *bad = 1;
}

// counts: per graph (1 + R) rows; out: per graph sig_h, cp_h, sig_3h, cp_3h
__global__ void __launch_bounds__(256) k_sig_cp_batch(const int64_t* __restrict__ counts_h,
                                                      const int64_t* __restrict__ counts_3h,
                                                      int R, double eps, double* __restrict__ out,
                                                      int32_t* __restrict__ deg) {
  __shared__ double red[1];
  const int64_t b = blockIdx.x;
  double* o = out + b * 2 * 457;
  sig_cp(counts_h + b * (R + 1) * MOCHY_N_H, MOCHY_N_H, R, eps, o, o + MOCHY_N_H, deg + 2 * b, red);
  sig_cp(counts_3h + b * (R + 1) * MOCHY_N_3H, MOCHY_N_3H, R, eps, o + 2 * MOCHY_N_H,
         o + 2 * MOCHY_N_H + MOCHY_N_3H, deg + 2 * b + 1, red);
}

}  // namespace

int finish_counts_batch(mochy_ctx* ctx, const unsigned long long* d_hist, int n_hist,
                        int64_t* d_out_h, int64_t* d_out_3h, int32_t* d_bad) {
  k_finish_batch<<<n_hist, 512, 0, ctx->stream>>>(d_hist, ctx->tables.t2h, d_out_h, d_out_3h,
                                                  d_bad);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

int significance_cp_batch(mochy_ctx* ctx, const int64_t* d_counts_h, const int64_t* d_counts_3h,
                          int n_graphs, int32_t n_random, double eps, double* d_out,
                          int32_t* d_degenerate) {
  k_sig_cp_batch<<<n_graphs, 256, 0, ctx->stream>>>(d_counts_h, d_counts_3h, n_random, eps, d_out,
                                                    d_degenerate);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

int finish_counts(mochy_ctx* ctx, const unsigned long long* d_hist, int64_t* d_out_h,
                  int64_t* d_out_3h) {
  k_finish<<<1, 512, 0, ctx->stream>>>(d_hist, ctx->tables.t2h, d_out_h, d_out_3h,
                                       ctx->counters + 8);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

int scale_estimates(mochy_ctx* ctx, const int64_t* d_raw_h, const int64_t* d_raw_3h, int method,
                    double numer, int64_t samples, double* d_est_h, double* d_est_3h) {
  k_scale<<<1, 512, 0, ctx->stream>>>(d_raw_h, d_raw_3h, ctx->tables.t2h, ctx->tables.hopen,
                                      method, numer, (double)samples, d_est_h, d_est_3h);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

int significance_cp(mochy_ctx* ctx, const int64_t* d_counts_h, const int64_t* d_counts_3h,
                    int32_t n_random, double eps, double* d_out, int32_t* d_degenerate) {
  k_sig_cp<<<1, 256, 0, ctx->stream>>>(d_counts_h, d_counts_3h, n_random, eps, d_out,
                                       d_degenerate);
  MOCHY_LAUNCHED();
  return MOCHY_OK;
}

}  // namespace mochy

// Detection-quality metrics of Sec. IV-B on the GPU: ROC AUC, AUC_TPR,tau,
// AUC_FPR,tau, AUC_TD and AUC_BS of a score map against anomaly labels.
//
//  1. one pass: min, max, and per class the count and the FP64 sum of the
//     scores (per-CTA partials, combined in CTA order: deterministic);
//  2. the scores min-max normalised in FP64, v = (s - min) / (max - min),
//     quantised to q = min(floor(v * bins), bins - 1), counted per class
//     (shared-memory histograms flushed with integer atomics: exact);
//  3. one CTA: 2U = sum_q pos[q] (2 * background below q + background at q),
//     the Mann-Whitney statistic of the quantised map (ties count one half).
// AUC = 2U / (2 n_p n_n); AUC_TPR,tau (AUC_FPR,tau), the area under TPR (FPR)
// against tau over [0, 1], is the mean normalised score of the anomalies (of
// the background).
#include <algorithm>
#include <cmath>

#include "../../include/erx.h"
#include "erx_internal.cuh"

namespace erx {
namespace {

constexpr int kRT = 256;
constexpr int kShBins = 16384;   // per-class shared histogram up to this many levels

struct RocPart {
  double mn, mx, sp, sn;
  unsigned long long np, nn;
};

template <typename ST>
__global__ void __launch_bounds__(kRT) roc_reduce_kernel(const ST* __restrict__ s,
                                                         const uint8_t* __restrict__ y, int64_t n,
                                                         RocPart* __restrict__ parts) {
  double mn = INFINITY, mx = -INFINITY, sp = 0.0, sn = 0.0;
  unsigned long long np = 0, nn = 0;
  for (int64_t i = (int64_t)blockIdx.x * kRT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRT) {
    const double v = (double)s[i];
    mn = fmin(mn, v);
    mx = fmax(mx, v);
    if (y[i]) sp += v, ++np;
    else sn += v, ++nn;
  }
  __shared__ RocPart sh[kRT];
  sh[threadIdx.x] = {mn, mx, sp, sn, np, nn};
  __syncthreads();
  for (int h = kRT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      RocPart& a = sh[threadIdx.x];
      const RocPart& b = sh[threadIdx.x + h];
      a.mn = fmin(a.mn, b.mn);
      a.mx = fmax(a.mx, b.mx);
      a.sp += b.sp;
      a.sn += b.sn;
      a.np += b.np;
      a.nn += b.nn;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[blockIdx.x] = sh[0];
}

__global__ void roc_final_kernel(const RocPart* __restrict__ parts, int nparts,
                                 RocPart* __restrict__ tot) {
  RocPart a{INFINITY, -INFINITY, 0.0, 0.0, 0ull, 0ull};
  for (int i = 0; i < nparts; ++i) {
    a.mn = fmin(a.mn, parts[i].mn);
    a.mx = fmax(a.mx, parts[i].mx);
    a.sp += parts[i].sp;
    a.sn += parts[i].sn;
    a.np += parts[i].np;
    a.nn += parts[i].nn;
  }
  *tot = a;
}

template <typename ST, bool SHARED>
__global__ void __launch_bounds__(kRT) roc_hist_kernel(const ST* __restrict__ s,
                                                       const uint8_t* __restrict__ y, int64_t n,
                                                       const RocPart* __restrict__ tot, int bins,
                                                       unsigned long long* __restrict__ hist) {
  extern __shared__ unsigned int hsh[];   // [2][bins] when SHARED: anomalies, background
  if (SHARED) {
    for (int i = threadIdx.x; i < 2 * bins; i += kRT) hsh[i] = 0u;
    __syncthreads();
  }
  const double mn = tot->mn, rng = tot->mx - tot->mn;
  for (int64_t i = (int64_t)blockIdx.x * kRT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRT) {
    const double v = rng > 0.0 ? ((double)s[i] - mn) / rng : 0.0;
    // v in [0, 1]; a non-finite score (or range) counts in level 0
    const int q = v > 0.0 ? min((int)floor(v * (double)bins), bins - 1) : 0;
    const int c = y[i] ? 0 : 1;
    if (SHARED) atomicAdd(&hsh[c * bins + q], 1u);
    else atomicAdd(&hist[(int64_t)c * bins + q], 1ull);
  }
  if (SHARED) {
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * bins; i += kRT)
      if (hsh[i]) atomicAdd(&hist[i], (unsigned long long)hsh[i]);
  }
}

// one CTA of 1024 threads; thread t takes levels [t*c, (t+1)*c)
__global__ void __launch_bounds__(1024) roc_auc_kernel(const unsigned long long* __restrict__ hist,
                                                       int bins, unsigned long long* __restrict__ u2) {
  __shared__ unsigned long long scan[1024];
  const unsigned long long* pos = hist;
  const unsigned long long* neg = hist + bins;
  const int c = (bins + 1023) / 1024;
  const int b0 = min(bins, (int)threadIdx.x * c), b1 = min(bins, b0 + c);
  unsigned long long tneg = 0;
  for (int b = b0; b < b1; ++b) tneg += neg[b];
  scan[threadIdx.x] = tneg;
  __syncthreads();
  // inclusive scan of the chunks' background counts (Hillis-Steele)
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned long long v = threadIdx.x >= (unsigned)o ? scan[threadIdx.x - o] : 0ull;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long below = scan[threadIdx.x] - tneg;   // background below this chunk
  unsigned long long acc = 0;
  for (int b = b0; b < b1; ++b) {
    acc += pos[b] * (2ull * below + neg[b]);
    below += neg[b];
  }
  __syncthreads();
  scan[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if (threadIdx.x < (unsigned)h) scan[threadIdx.x] += scan[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *u2 = scan[0];
}

}  // namespace
}  // namespace erx

using namespace erx;

extern "C" erx_status erx_roc_metrics(const void* scores_dev, int32_t score_dtype,
                                      const uint8_t* labels_dev, int64_t n, int32_t bins,
                                      void* cuda_stream, erx_roc* out) {
  if (!scores_dev || !labels_dev || !out || n <= 0 || bins < 2 || bins > (1 << 24) ||
      (score_dtype != ERX_F32 && score_dtype != ERX_F64))
    return ERX_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, n_sm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ECUDA;
  }
  const int nblk = (int)std::min<int64_t>((n + kRT - 1) / kRT, 4 * (int64_t)n_sm);
  const size_t hist_bytes = sizeof(unsigned long long) * 2 * (size_t)bins;
  const size_t bytes = sizeof(RocPart) * (nblk + 1) + hist_bytes + sizeof(unsigned long long);
  char* scratch = nullptr;
  if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ENOMEM;
  }
  RocPart* parts = (RocPart*)scratch;
  RocPart* tot = parts + nblk;
  unsigned long long* hist = (unsigned long long*)(tot + 1);
  unsigned long long* u2 = hist + 2 * (size_t)bins;
  const bool shared = bins <= kShBins;
  const size_t shb = shared ? sizeof(unsigned int) * 2 * (size_t)bins : 0;
  cudaError_t e = cudaMemsetAsync(hist, 0, hist_bytes, st);
  if (e == cudaSuccess && shared) {
    e = cudaFuncSetAttribute(roc_hist_kernel<float, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(roc_hist_kernel<double, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb);
  }
  if (e == cudaSuccess) {
#define ERX_ROC(ST)                                                                             \
  roc_reduce_kernel<ST><<<nblk, kRT, 0, st>>>((const ST*)scores_dev, labels_dev, n, parts);     \
  roc_final_kernel<<<1, 1, 0, st>>>(parts, nblk, tot);                                          \
  if (shared)                                                                                   \
    roc_hist_kernel<ST, true><<<nblk, kRT, shb, st>>>((const ST*)scores_dev, labels_dev, n, tot, \
                                                      bins, hist);                              \
  else                                                                                          \
    roc_hist_kernel<ST, false><<<nblk, kRT, 0, st>>>((const ST*)scores_dev, labels_dev, n, tot,  \
                                                     bins, hist);
    if (score_dtype == ERX_F32) {
      ERX_ROC(float)
    } else {
      ERX_ROC(double)
    }
#undef ERX_ROC
    roc_auc_kernel<<<1, 1024, 0, st>>>(hist, bins, u2);
    e = cudaGetLastError();
  }
  RocPart h{};
  unsigned long long hu2 = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hu2, u2, sizeof(hu2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ERX_ECUDA;
  }
  if (h.np == 0 || h.nn == 0) return ERX_EINVAL;
  const double np = (double)h.np, nn = (double)h.nn, rng = h.mx - h.mn;
  out->positives = (int64_t)h.np;
  out->negatives = (int64_t)h.nn;
  out->u2 = hu2;
  out->auc = (double)hu2 / (2.0 * np * nn);
  out->auc_tpr_tau = rng > 0.0 ? (h.sp / np - h.mn) / rng : 0.0;
  out->auc_fpr_tau = rng > 0.0 ? (h.sn / nn - h.mn) / rng : 0.0;
  out->auc_td = (out->auc + out->auc_tpr_tau) / 2.0;
  out->auc_bs = (out->auc - out->auc_fpr_tau + 1.0) / 2.0;
  return ERX_OK;
}

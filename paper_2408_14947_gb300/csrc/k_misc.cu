// S1 projection, S3 EMA scan and S6 normalisation kernels.
#include <cfloat>
#include <cmath>

#include "erx_internal.cuh"

namespace erx {
namespace {

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }

// ---- S3: exponential moving averages (Sec. III-C) ------------------------
//
// One thread per state element (the P entries of the packed lower triangle
// of K, then the d entries of mu), walking the T lines of the block in order:
//   line statistics -> (t == 0 ? init : (1-a) state + a stats) -> state.
// The recursion is a d^2-wide elementwise scan; the values a line is scored
// with (after the update, or before it for score-then-update) are written
// to mu_t / K_t.
// The per-line loads do not depend on the recursion, so they are issued
// kEmaBatch lines ahead of it to keep enough memory requests in flight; the
// recursion itself stays strictly sequential, so results do not depend on how
// lines are grouped into blocks.
constexpr int kEmaBatch = 8;

__global__ void __launch_bounds__(128) ema_scan_kernel(
    bool int_stats, const uint64_t* __restrict__ S1i, const uint64_t* __restrict__ S2i,
    const double* __restrict__ mu_hat, const double* __restrict__ shift,
    const double* __restrict__ S2f, int T, int d, int W, double alpha, int64_t t0, int order,
    double* __restrict__ mu_state, double* __restrict__ K_state, double* __restrict__ mu_t,
    double* __restrict__ K_t) {
  const int64_t P = packed_size(d);
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P + d) return;
  const double beta = 1.0 - alpha;
  const double Wd = (double)W;
  const double inv_pp = 1.0 / (Wd * (Wd - 1.0));
  const double inv_p1 = 1.0 / (Wd - 1.0);
  const int64_t dd = (int64_t)d * d;
  if (q < P) {
    int a = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while ((int64_t)a * (a + 1) / 2 > q) --a;
    while ((int64_t)(a + 1) * (a + 2) / 2 <= q) ++a;
    const int b = (int)(q - (int64_t)a * (a + 1) / 2);
    const int64_t ab = (int64_t)a * d + b;
    double s = K_state[q];
    for (int t0b = 0; t0b < T; t0b += kEmaBatch) {
      double kh[kEmaBatch];
      const int nb = min(kEmaBatch, T - t0b);
      if (int_stats) {
        int64_t s1a[kEmaBatch], s1b[kEmaBatch], s2[kEmaBatch];
#pragma unroll
        for (int u = 0; u < kEmaBatch; ++u) {
          if (u < nb) {
            const int64_t t = t0b + u;
            s1a[u] = (int64_t)__ldg(S1i + t * d + a);
            s1b[u] = (int64_t)__ldg(S1i + t * d + b);
            s2[u] = (int64_t)__ldg(S2i + t * dd + ab);
          }
        }
#pragma unroll
        for (int u = 0; u < kEmaBatch; ++u)
          if (u < nb) kh[u] = (double)((int64_t)W * s2[u] - s1a[u] * s1b[u]) * inv_pp;
      } else {
        double ea[kEmaBatch], eb[kEmaBatch], sv[kEmaBatch];
#pragma unroll
        for (int u = 0; u < kEmaBatch; ++u) {
          if (u < nb) {
            const int64_t t = t0b + u;
            ea[u] = __ldg(mu_hat + t * d + a) - __ldg(shift + t * d + a);
            eb[u] = __ldg(mu_hat + t * d + b) - __ldg(shift + t * d + b);
            sv[u] = __ldg(S2f + t * dd + ab);
          }
        }
#pragma unroll
        for (int u = 0; u < kEmaBatch; ++u)
          if (u < nb) kh[u] = (sv[u] - Wd * ea[u] * eb[u]) * inv_p1;
      }
#pragma unroll
      for (int u = 0; u < kEmaBatch; ++u) {
        if (u < nb) {
          const int64_t t = t0b + u;
          const bool first = (t0 + t == 0);
          const double post = first ? kh[u] : beta * s + alpha * kh[u];
          K_t[t * P + q] = (order == 0 || first) ? post : s;
          s = post;
        }
      }
    }
    K_state[q] = s;
  } else {
    const int a = (int)(q - P);
    double s = mu_state[a];
    for (int t = 0; t < T; ++t) {
      const double mh = int_stats ? (double)__ldg(S1i + (int64_t)t * d + a) / Wd
                                  : __ldg(mu_hat + (int64_t)t * d + a);
      const bool first = (t0 + t == 0);
      const double post = first ? mh : beta * s + alpha * mh;
      mu_t[(int64_t)t * d + a] = (order == 0 || first) ? post : s;
      s = post;
    }
    mu_state[a] = s;
  }
}

// ---- S6: line-by-line normalisation (Sec. III-E) -------------------------
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double tot = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) tot += sh[i];
  return tot;
}

template <typename ST>
__global__ void __launch_bounds__(256) normalise_kernel(const ST* __restrict__ delta, int W,
                                                        double threshold, int64_t t0,
                                                        int64_t warmup, ST* __restrict__ dn,
                                                        uint8_t* __restrict__ mask,
                                                        uint8_t* __restrict__ detecting) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const ST* dl = delta + (int64_t)t * W;
  double s = 0.0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) s += to_d(dl[i]);
  const double mean = block_sum(s, sh) / (double)W;
  double v = 0.0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double e = to_d(dl[i]) - mean;
    v += e * e;
  }
  const double sd = sqrt(block_sum(v, sh) / (double)W);
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double z = sd > 0.0 ? (to_d(dl[i]) - mean) / sd : 0.0;
    if (dn) dn[(int64_t)t * W + i] = (ST)z;
    if (mask) mask[(int64_t)t * W + i] = (uint8_t)(z >= threshold);
  }
  if (detecting && threadIdx.x == 0) detecting[t] = (uint8_t)(t0 + t >= warmup);
}

// ---- S1: sparse random projection Z = X W (Sec. III-B) --------------------
// One thread per (pixel, output dim); W held as per-column lists of
// (band, weight).  Accumulates in double.
template <typename InT, typename OutT>
__global__ void __launch_bounds__(256) project_kernel(const InT* __restrict__ X,
                                                      int64_t line_stride, int B, int W, int d,
                                                      const int* __restrict__ colptr,
                                                      const int* __restrict__ rows,
                                                      const double* __restrict__ vals,
                                                      OutT* __restrict__ Z) {
  const int t = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)W * d) return;
  const int i = (int)(e / d), j = (int)(e % d);
  const InT* xp = X + (int64_t)t * line_stride + (int64_t)i * B;
  double s = 0.0;
  for (int q = colptr[j]; q < colptr[j + 1]; ++q) s = fma(vals[q], to_d(xp[rows[q]]), s);
  Z[((int64_t)t * W + i) * d + j] = (OutT)s;
}

}  // namespace

void launch_ema_scan(bool int_stats, const uint64_t* S1i, const uint64_t* S2i,
                     const double* mu_hat, const double* shift, const double* S2f, int T, int d,
                     int W, double alpha, int64_t t0, int order, double* mu_state,
                     double* K_state, double* mu_t, double* K_t, cudaStream_t st) {
  const int64_t n = packed_size(d) + d;
  const int blocks = (int)((n + 127) / 128);
  ema_scan_kernel<<<blocks, 128, 0, st>>>(int_stats, S1i, S2i, mu_hat, shift, S2f, T, d, W,
                                          alpha, t0, order, mu_state, K_state, mu_t, K_t);
}

void launch_normalise(bool fp64, const void* delta, int W, int T, double threshold, int64_t t0,
                      int64_t warmup, void* delta_n, uint8_t* mask, uint8_t* detecting,
                      cudaStream_t st) {
  if (fp64)
    normalise_kernel<double><<<T, 256, 0, st>>>((const double*)delta, W, threshold, t0, warmup,
                                                (double*)delta_n, mask, detecting);
  else
    normalise_kernel<float><<<T, 256, 0, st>>>((const float*)delta, W, threshold, t0, warmup,
                                               (float*)delta_n, mask, detecting);
}

void launch_project(int in_type, const void* x, int64_t line_stride, int B, int W, int d, int T,
                    const int* colptr, const int* rows, const double* vals, bool out_fp64,
                    void* z, cudaStream_t st) {
  const int64_t n = (int64_t)W * d;
  dim3 grid((unsigned)((n + 255) / 256), T);
#define ERX_PRJ(IT, OT)                                                                       \
  project_kernel<IT, OT><<<grid, 256, 0, st>>>((const IT*)x, line_stride, B, W, d, colptr, \
                                               rows, vals, (OT*)z)
  if (out_fp64) {
    if (in_type == 0) ERX_PRJ(uint16_t, double);
    else if (in_type == 1) ERX_PRJ(float, double);
    else ERX_PRJ(double, double);
  } else {
    if (in_type == 0) ERX_PRJ(uint16_t, float);
    else if (in_type == 1) ERX_PRJ(float, float);
    else ERX_PRJ(double, float);
  }
#undef ERX_PRJ
}

}  // namespace erx

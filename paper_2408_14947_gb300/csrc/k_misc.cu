// S1 projection, S3 EMA scan and S6 normalisation kernels.
#include <cfloat>
#include <cmath>

#include "erx_batch.cuh"
#include "erx_internal.cuh"

namespace erx {
namespace {

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }

// ---- S3: exponential moving averages (Sec. III-C) ------------------------
//
// Per state element (the P entries of the packed lower triangle of K, then the
// d entries of mu) the recursion s_t = (1-a) s_{t-1} + a khat_t runs over the
// T lines of a block; line 0 of the stream sets s_0 = khat_0.  The values a
// line is scored with (after the update, or before it for score-then-update)
// go to mu_t / K_t.
//
// The recursion is linear, so a block is cut into chunks of kEmaChunk lines:
//   pass A  each (element, chunk) forms the value the recursion reaches from 0
//           over its chunk, as the sum of the chunk's statistics with their
//           weights a (1-a)^k (a weighted sum, not the recursion step by step);
//   pass B  each element chains the chunk results sequentially:
//           s_end = (1-a)^len s_start + u_chunk  (or u_chunk if the chunk holds line 0);
//   pass C  each (element, chunk) reruns its chunk from the carried-in state
//           and writes the per-line values.
// Within a chunk the arithmetic is the sequential recursion; across chunk
// boundaries the carried value is formed in closed form (passes A and B), which
// differs from the sequential recursion only by rounding.  Blocks of at most kEmaChunk lines
// run pass C alone on the state (purely sequential).
constexpr int kEmaChunk = 32;
constexpr int kEmaPre = 8;     // line statistics in flight per thread

struct EmaSrc {
  bool int_stats;
  bool small_ints;   // |W s2 - s1a s1b| <= (W maxv)^2 < 2^51: the exact short conversion applies
  const uint64_t* S1i;
  const uint64_t* S2i;
  const double* mu_hat;
  const double* shift;
  const double* S2f;
  int d, W;
  int64_t P;
  double rw1;    // 1 / (W - 1), correctly rounded
  double rw12;   // 1 / (W (W - 1)), correctly rounded
};

// v as a double, exactly, for |v| < 2^51: v added to the bits of 1.5 * 2^52 (whose
// last mantissa bit is worth 1) gives the double 1.5 * 2^52 + v; one exact
// subtraction removes the offset.  An integer add and one DADD, where the
// general 64-bit conversion is slower on this part.
__device__ __forceinline__ double i2d_exact(int64_t v) {
  return __dsub_rn(__longlong_as_double(0x4338000000000000ll + v), 6755399441055744.0);
}

// (W maxv)^2 < 2^51 bounds |W s2 - s1a s1b| for samples <= maxv
inline bool small_ints(int W, uint32_t maxv) {
  const double m = (double)W * (double)maxv;
  return m * m < 2251799813685248.0;
}

// line statistic of element (a, b) (b < 0: the mean of band a) at line t of the block
__device__ __forceinline__ double ema_stat(const EmaSrc& s, int64_t t, int a, int b) {
  const double Wd = (double)s.W;
  if (b < 0) {
    return s.int_stats ? (double)__ldg(s.S1i + t * s.d + a) / Wd : __ldg(s.mu_hat + t * s.d + a);
  }
  const int64_t dd = (int64_t)s.d * s.d;
  const int64_t ab = (int64_t)a * s.d + b;
  if (s.int_stats) {
    const int64_t s1a = (int64_t)__ldg(s.S1i + t * s.d + a);
    const int64_t s1b = (int64_t)__ldg(s.S1i + t * s.d + b);
    const int64_t s2 = (int64_t)__ldg(s.S2i + t * dd + ab);
    const int64_t v = (int64_t)s.W * s2 - s1a * s1b;
    return (s.small_ints ? i2d_exact(v) : (double)v) * s.rw12;
  }
  const double ea = __dsub_rn(__ldg(s.mu_hat + t * s.d + a), __ldg(s.shift + t * s.d + a));
  const double eb = __dsub_rn(__ldg(s.mu_hat + t * s.d + b), __ldg(s.shift + t * s.d + b));
  return ema_khat(__ldg(s.S2f + t * dd + ab), ea, eb, Wd, s.rw1);
}

__device__ __forceinline__ void ema_element(const EmaSrc& s, int64_t q, int& a, int& b) {
  if (q >= s.P) {
    a = (int)(q - s.P);
    b = -1;
    return;
  }
  // a float square root (FP64 is scarce here) and exact integer correction
  int r = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
  while ((int64_t)r * (r + 1) / 2 > q) --r;
  while ((int64_t)(r + 1) * (r + 2) / 2 <= q) ++r;
  a = r;
  b = (int)(q - (int64_t)r * (r + 1) / 2);
}

// pass A: chunk g's aggregate from zero, E[g][q] = sum_t w_t Khat_t with
// w_t = alpha (1 - alpha)^(te - 1 - t), the line that starts the EMA (t0 + t = 0)
// taking (1 - alpha)^(te - 1 - t): the value the recursion of Sec. III-C reaches
// over the chunk from a zero state.  It only feeds the carry into the next
// chunks (pass B); pass C then runs the recursion itself line by line.  The
// weights are a per-chunk table, so an element of the integer sums takes one
// exact conversion and one multiply-add per line (Khat = v / (W (W - 1)) with
// the integer v, the division applied once per chunk), instead of the five FP64
// operations of the recursion.
__global__ void __launch_bounds__(128) ema_pass_a(EmaSrc s, int T, double alpha, int64_t t0,
                                                  double* __restrict__ E) {
  __shared__ double wt[kEmaChunk];
  const int g = blockIdx.y;
  const int tb = g * kEmaChunk, te = min(T, tb + kEmaChunk);
  const double beta = 1.0 - alpha;
  if (threadIdx.x == 0) {
    double w = 1.0;
    for (int t = te - 1; t >= tb; --t) {
      wt[t - tb] = (t0 + t == 0) ? w : w * alpha;
      w *= beta;
    }
  }
  __syncthreads();
  const int64_t n = s.P + s.d;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int a, b;
  ema_element(s, q, a, b);
  double u = 0.0;
  if (s.int_stats && b >= 0) {
    const int64_t dd = (int64_t)s.d * s.d, ab = (int64_t)a * s.d + b;
    for (int t8 = tb; t8 < te; t8 += kEmaPre) {
      double v[kEmaPre];
#pragma unroll
      for (int j = 0; j < kEmaPre; ++j) {
        const int t = t8 + j < te ? t8 + j : te - 1;
        const int64_t s1a = (int64_t)__ldg(s.S1i + t * s.d + a);
        const int64_t s1b = (int64_t)__ldg(s.S1i + t * s.d + b);
        const int64_t s2 = (int64_t)__ldg(s.S2i + t * dd + ab);
        const int64_t iv = (int64_t)s.W * s2 - s1a * s1b;
        v[j] = s.small_ints ? i2d_exact(iv) : (double)iv;
      }
#pragma unroll
      for (int j = 0; j < kEmaPre; ++j)
        if (t8 + j < te) u = fma(wt[t8 + j - tb], v[j], u);
    }
    u *= s.rw12;
  } else {
    for (int t8 = tb; t8 < te; t8 += kEmaPre) {
      double kh[kEmaPre];
#pragma unroll
      for (int j = 0; j < kEmaPre; ++j) kh[j] = t8 + j < te ? ema_stat(s, t8 + j, a, b) : 0.0;
#pragma unroll
      for (int j = 0; j < kEmaPre; ++j)
        if (t8 + j < te) u = fma(wt[t8 + j - tb], kh[j], u);
    }
  }
  E[(int64_t)g * n + q] = u;
}

// pass B: chain chunk results; Cin[g][q] = state entering chunk g
__global__ void __launch_bounds__(128) ema_pass_b(int64_t n, int T, int G, double alpha,
                                                  int64_t t0, const double* __restrict__ E,
                                                  double* __restrict__ Cin,
                                                  double* __restrict__ Kst,
                                                  double* __restrict__ must, int64_t P) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double beta = 1.0 - alpha;
  double* st = q < P ? Kst + q : must + (q - P);
  double s = *st;
  double bp = 1.0;                       // (1-a)^kEmaChunk
  for (int i = 0; i < kEmaChunk; ++i) bp *= beta;
  // the chunk aggregates are loaded kEmaPre at a time ahead of the chain, which
  // then waits on no load
  for (int g8 = 0; g8 < G; g8 += kEmaPre) {
    double ev[kEmaPre];
#pragma unroll
    for (int j = 0; j < kEmaPre; ++j) ev[j] = g8 + j < G ? E[(int64_t)(g8 + j) * n + q] : 0.0;
#pragma unroll
    for (int j = 0; j < kEmaPre; ++j) {
      const int g = g8 + j;
      if (g >= G) break;
      Cin[(int64_t)g * n + q] = s;
      const int tb = g * kEmaChunk, te = min(T, tb + kEmaChunk);
      const bool has_init = (t0 + tb <= 0) && (t0 + te > 0);
      double w = bp;
      if (te - tb != kEmaChunk) {
        w = 1.0;
        for (int i = tb; i < te; ++i) w *= beta;
      }
      s = has_init ? ev[j] : __dadd_rn(__dmul_rn(w, s), ev[j]);
    }
  }
  *st = s;
}

// pass C: rerun each chunk from its carried-in state, write the per-line values
__global__ void __launch_bounds__(128) ema_pass_c(EmaSrc s, int T, double alpha, int64_t t0,
                                                  int order, const double* __restrict__ Cin,
                                                  double* __restrict__ Kst,
                                                  double* __restrict__ must,
                                                  double* __restrict__ mu_t,
                                                  double* __restrict__ K_t) {
  const int64_t n = s.P + s.d;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int g = blockIdx.y;
  int a, b;
  ema_element(s, q, a, b);
  const double beta = 1.0 - alpha;
  double* st = q < s.P ? Kst + q : must + (q - s.P);
  double v = Cin ? Cin[(int64_t)g * n + q] : *st;
  const int tb = g * kEmaChunk, te = Cin ? min(T, tb + kEmaChunk) : T;
  for (int t8 = tb; t8 < te; t8 += kEmaPre) {
    double kh[kEmaPre];
#pragma unroll
    for (int j = 0; j < kEmaPre; ++j) kh[j] = t8 + j < te ? ema_stat(s, t8 + j, a, b) : 0.0;
#pragma unroll
    for (int j = 0; j < kEmaPre; ++j) {
      const int t = t8 + j;
      if (t >= te) break;
      const bool first = (t0 + t == 0);
      const double post = first ? kh[j] : ema_mix(v, kh[j], alpha, beta);
      const double out = (order == 0 || first) ? post : v;
      if (b < 0) mu_t[(int64_t)t * s.d + a] = out;
      else K_t[(int64_t)t * s.P + q] = out;
      v = post;
    }
  }
  if (!Cin) *st = v;
}

// ---- IMC: the equal-weight ablation of Sec. IV-C (batch Welford) ----------
// After global line g (p pixels each) the state is the mean and the 1/(n-1)
// covariance of all n = (g+1)p pixels seen.  With delta_g = mu_hat_g - mu_{g-1}:
//   mu_g = mu_{g-1} + delta_g / (g+1)   (the mean of the line means: S_g / (g+1),
//                                        S_g = sum_{s <= g} mu_hat_s),
//   M_g  = M_{g-1} + (p-1) K_hat_g + (g p^2 / ((g+1) p)) delta_g delta_g^T,
//   K_g  = M_g / ((g+1)p - 1),
// (M = (n-1) K, the scatter).  Both are prefix sums over the block's lines,
// computed in 32-line chunks: chunk sums, a carry over chunks, per-line values.
// Per-line constants come from a table (one thread per line), so no element
// divides per line.

// per-line table, 4 x T: weight of delta delta^T, 1/((g+1)p - 1), 1/(gp - 1), 1/(g+1)
__global__ void __launch_bounds__(128) imc_table_kernel(int T, int W, int64_t t0,
                                                        double* __restrict__ tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int64_t g = t0 + t;
  const double na = (double)g * W, n = na + W;
  tab[t] = na * W / n;
  tab[T + t] = 1.0 / (n - 1.0);
  tab[2 * T + t] = g > 0 ? 1.0 / (na - 1.0) : 0.0;
  tab[3 * T + t] = 1.0 / (double)(g + 1);
}

// means, pass A: E1[c][a] = sum of the line means of chunk c
__global__ void __launch_bounds__(128) imc_mean_a(EmaSrc s, int T, double* __restrict__ E1) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s.d) return;
  const int c = blockIdx.y;
  const int tb = c * kEmaChunk, te = min(T, tb + kEmaChunk);
  double u = 0.0;
  for (int t = tb; t < te; ++t) u += ema_stat(s, t, a, -1);
  E1[(int64_t)c * s.d + a] = u;
}

// means, pass C: per line mu_t (the order's) and delta_g; the state is left to imc_mean_state
__global__ void __launch_bounds__(128) imc_mean_c(EmaSrc s, int T, int64_t t0, int order,
                                                  const double* __restrict__ mu_state,
                                                  const double* __restrict__ E1,
                                                  const double* __restrict__ tab,
                                                  double* __restrict__ mu_t,
                                                  double* __restrict__ dlt) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s.d) return;
  const int c = blockIdx.y;
  const int tb = c * kEmaChunk, te = min(T, tb + kEmaChunk);
  double S = t0 > 0 ? mu_state[a] * (double)t0 : 0.0;
  for (int cc = 0; cc < c; ++cc) S += E1[(int64_t)cc * s.d + a];
  const int64_t g0 = t0 + tb;
  double prev = g0 == 0 ? 0.0 : (tb == 0 ? mu_state[a] : S * (1.0 / (double)g0));
  for (int t = tb; t < te; ++t) {
    const int64_t g = t0 + t;
    const double mh = ema_stat(s, t, a, -1);
    S += mh;
    const double post = g == 0 ? mh : S * tab[3 * T + t];
    dlt[(int64_t)t * s.d + a] = g == 0 ? 0.0 : mh - prev;
    mu_t[(int64_t)t * s.d + a] = (order == 0 || g == 0) ? post : prev;
    prev = post;
  }
}

__global__ void __launch_bounds__(128) imc_mean_state(int d, int G, int T, int64_t t0,
                                                      const double* __restrict__ E1,
                                                      double* __restrict__ mu_state) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d) return;
  double S = t0 > 0 ? mu_state[a] * (double)t0 : 0.0;
  for (int c = 0; c < G; ++c) S += E1[(int64_t)c * d + a];
  mu_state[a] = S / (double)(t0 + T);
}

// scatter increment of element (a, b) at line t of the block
__device__ __forceinline__ double imc_inc(const EmaSrc& s, int64_t t, int a, int b,
                                          const double* __restrict__ dlt,
                                          const double* __restrict__ tab) {
  const double kh = ema_stat(s, t, a, b);
  return kh * ((double)s.W - 1.0) +
         __ldg(dlt + t * s.d + a) * __ldg(dlt + t * s.d + b) * __ldg(tab + t);
}

// pass A: the chunk's sum of increments, E[c][q]
__global__ void __launch_bounds__(128) imc_pass_a(EmaSrc s, int T,
                                                  const double* __restrict__ dlt,
                                                  const double* __restrict__ tab,
                                                  double* __restrict__ E) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= s.P) return;
  const int c = blockIdx.y;
  int a, b;
  ema_element(s, q, a, b);
  const int tb = c * kEmaChunk, te = min(T, tb + kEmaChunk);
  double u = 0.0;
  for (int t = tb; t < te; ++t) u += imc_inc(s, t, a, b, dlt, tab);
  E[(int64_t)c * s.P + q] = u;
}

// pass B: scatter entering each chunk, Cin[c][q]; the state's K becomes the
// covariance after the block
__global__ void __launch_bounds__(128) imc_pass_b(int64_t P, int T, int G, int W, int64_t t0,
                                                  const double* __restrict__ E,
                                                  double* __restrict__ Cin,
                                                  double* __restrict__ Kst) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  double m = t0 > 0 ? Kst[q] * ((double)t0 * W - 1.0) : 0.0;
  for (int c = 0; c < G; ++c) {
    Cin[(int64_t)c * P + q] = m;
    m += E[(int64_t)c * P + q];
  }
  Kst[q] = m / ((double)(t0 + T) * W - 1.0);
}

// pass C: per-line covariances from each chunk's carried-in scatter (or, with
// no carry, from the state: the whole block as one chunk, state updated here)
__global__ void __launch_bounds__(128) imc_pass_c(EmaSrc s, int T, int64_t t0, int order,
                                                  const double* __restrict__ dlt,
                                                  const double* __restrict__ tab,
                                                  const double* __restrict__ Cin,
                                                  double* __restrict__ Kst,
                                                  double* __restrict__ K_t) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= s.P) return;
  const int c = blockIdx.y;
  int a, b;
  ema_element(s, q, a, b);
  const double Wd = (double)s.W;
  double m = Cin ? Cin[(int64_t)c * s.P + q] : (t0 > 0 ? Kst[q] * ((double)t0 * Wd - 1.0) : 0.0);
  const int tb = c * kEmaChunk, te = Cin ? min(T, tb + kEmaChunk) : T;
  for (int t = tb; t < te; ++t) {
    const int64_t g = t0 + t;
    const double post = m + imc_inc(s, t, a, b, dlt, tab);
    const double out = (order == 0 || g == 0) ? post * __ldg(tab + T + t)
                                              : m * __ldg(tab + 2 * T + t);
    K_t[(int64_t)t * s.P + q] = out;
    m = post;
  }
  if (!Cin) Kst[q] = m / ((double)(t0 + T) * Wd - 1.0);
}

// ---- S6: line-by-line normalisation (Sec. III-E) -------------------------
// Sum of v over the block: a shuffle tree per warp, then the warps' sums added
// in warp order by thread 0 alone (the result is valid in thread 0 only).  An
// FP64 warp instruction costs this part's SM about 19 cycles of its FP64 pipe
// however few lanes it uses, so the tail of the reduction, the division, the
// square root and the reciprocal run once per line, not once per warp.
__device__ double block_sum0(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) tot += sh[i];
  }
  return tot;
}

// One line: delta_N, mask and the warm-up flag of global line `line`.
template <typename ST>
__device__ __forceinline__ void normalise_body(const ST* __restrict__ dl, int W, double threshold,
                                               int64_t line, int64_t warmup,
                                               ST* __restrict__ dn, uint8_t* __restrict__ mask,
                                               uint8_t* __restrict__ detecting) {
  __shared__ double sh[32];
  __shared__ double bc[2];   // the line's mean and 1 / sigma, from thread 0
  double s = 0.0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) s += to_d(dl[i]);
  const double ts = block_sum0(s, sh);
  if (threadIdx.x == 0) bc[0] = ts / (double)W;
  __syncthreads();
  const double mean = bc[0];
  double v = 0.0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double e = __dsub_rn(to_d(dl[i]), mean);
    v = __fma_rn(e, e, v);
  }
  const double tv = block_sum0(v, sh);
  if (threadIdx.x == 0) {
    const double sd = sqrt(tv / (double)W);
    bc[1] = sd > 0.0 ? 1.0 / sd : 0.0;   // one division per line, not per pixel
  }
  __syncthreads();
  const double rsd = bc[1];
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double z = (to_d(dl[i]) - mean) * rsd;
    if (dn) dn[i] = (ST)z;
    if (mask) mask[i] = (uint8_t)(z >= threshold);
  }
  if (detecting && threadIdx.x == 0) *detecting = (uint8_t)(line >= warmup);
}

template <typename ST>
__global__ void __launch_bounds__(256) normalise_kernel(const ST* __restrict__ delta, int W,
                                                        double threshold, int64_t t0,
                                                        int64_t warmup, ST* __restrict__ dn,
                                                        uint8_t* __restrict__ mask,
                                                        uint8_t* __restrict__ detecting) {
  const int t = blockIdx.x;
  const int64_t o = (int64_t)t * W;
  normalise_body<ST>(delta + o, W, threshold, t0 + t, warmup, dn ? dn + o : nullptr,
                     mask ? mask + o : nullptr, detecting ? detecting + t : nullptr);
}

// ---- batched form -------------------------------------------------------
// EMA of one line per stream: each CTA updates 128 state elements of one
// stream (item tile = element block); line 0 of a stream initialises.
__global__ void __launch_bounds__(128) b_ema_kernel(BStream* __restrict__ S,
                                                    const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  BStream& s = S[it.s];
  const int d = s.d;
  const int64_t P = packed_size(d);
  const int64_t q = (int64_t)it.tile * 128 + threadIdx.x;
  if (q >= P + d) return;
  const bool first = (s.t == 0);
  const double alpha = s.alpha, beta = 1.0 - alpha;
  const double Wd = (double)s.W;
  if (q < P) {
    int a = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);   // corrected below
    while ((int64_t)a * (a + 1) / 2 > q) --a;
    while ((int64_t)(a + 1) * (a + 2) / 2 <= q) ++a;
    const int b = (int)(q - (int64_t)a * (a + 1) / 2);
    const double ea = __dsub_rn(s.mu_hat[a], s.shift[a]);
    const double eb = __dsub_rn(s.mu_hat[b], s.shift[b]);
    // the scatter's chunk sums, added in chunk order (as the single-stream scatter does)
    const double* sp = s.S2f + (int64_t)a * d + b;
    double S2 = sp[0];
    for (int c = 1; c < s.nch; ++c) S2 = __dadd_rn(S2, sp[(int64_t)c * d * d]);
    const double kh = ema_khat(S2, ea, eb, Wd, __drcp_rn(Wd - 1.0));
    const double prev = s.K_state[q];
    const double post = first ? kh : ema_mix(prev, kh, alpha, beta);
    s.K_t[q] = (s.order == 0 || first) ? post : prev;
    s.K_state[q] = post;
  } else {
    const int a = (int)(q - P);
    const double mh = s.mu_hat[a];
    const double prev = s.mu_state[a];
    const double post = first ? mh : ema_mix(prev, mh, alpha, beta);
    s.mu_t[a] = (s.order == 0 || first) ? post : prev;
    s.mu_state[a] = post;
  }
}

// Normalisation per stream; thread 0 then advances the stream's line count.
template <typename ST>
__global__ void __launch_bounds__(256) b_normalise_kernel(BStream* __restrict__ S,
                                                          const BItem* __restrict__ items) {
  BStream& s = S[items[blockIdx.x].s];
  const bool st64 = (s.route == 0);
  if ((sizeof(ST) == 8) == st64)
    normalise_body<ST>((const ST*)s.delta, s.W, s.threshold, s.t, s.warmup, (ST*)s.dn, s.mask,
                       s.det);
  __syncthreads();
  if (threadIdx.x == 0) s.t += 1;
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
                     double* K_state, double* mu_t, double* K_t, double* scratch,
                     cudaStream_t st, uint32_t maxv) {
  // both reciprocals correctly rounded on the host (IEEE division), as
  // __drcp_rn and the device's double division would give
  const double Wd = (double)W;
  EmaSrc s{int_stats, small_ints(W, maxv), S1i, S2i, mu_hat, shift, S2f, d, W, packed_size(d),
           1.0 / (Wd - 1.0), 1.0 / (Wd * (Wd - 1.0))};
  const int64_t n = s.P + d;
  const unsigned bx = (unsigned)((n + 127) / 128);
  const int G = (T + kEmaChunk - 1) / kEmaChunk;
  if (G <= 1 || !scratch) {
    ema_pass_c<<<dim3(bx, 1), 128, 0, st>>>(s, T, alpha, t0, order, nullptr, K_state, mu_state,
                                           mu_t, K_t);
    return;
  }
  double* E = scratch;
  double* Cin = scratch + (int64_t)G * n;
  ema_pass_a<<<dim3(bx, G), 128, 0, st>>>(s, T, alpha, t0, E);
  ema_pass_b<<<bx, 128, 0, st>>>(n, T, G, alpha, t0, E, Cin, K_state, mu_state, s.P);
  ema_pass_c<<<dim3(bx, G), 128, 0, st>>>(s, T, alpha, t0, order, Cin, K_state, mu_state, mu_t,
                                         K_t);
}

void launch_imc_scan(bool int_stats, const uint64_t* S1i, const uint64_t* S2i,
                     const double* mu_hat, const double* shift, const double* S2f, int T, int d,
                     int W, int64_t t0, int order, double* mu_state, double* K_state,
                     double* mu_t, double* K_t, double* work, double* scratch,
                     cudaStream_t st, uint32_t maxv) {
  const double Wd = (double)W;
  EmaSrc s{int_stats, small_ints(W, maxv), S1i, S2i, mu_hat, shift, S2f, d, W, packed_size(d),
           1.0 / (Wd - 1.0), 1.0 / (Wd * (Wd - 1.0))};
  const int G = (T + kEmaChunk - 1) / kEmaChunk;
  double* dlt = work;                         // T x d
  double* tab = work + (int64_t)T * d;        // 4 x T
  double* E1 = tab + 4 * (int64_t)T;          // G x d
  const unsigned bd = (unsigned)((d + 127) / 128);
  imc_table_kernel<<<(T + 127) / 128, 128, 0, st>>>(T, W, t0, tab);
  imc_mean_a<<<dim3(bd, G), 128, 0, st>>>(s, T, E1);
  imc_mean_c<<<dim3(bd, G), 128, 0, st>>>(s, T, t0, order, mu_state, E1, tab, mu_t, dlt);
  imc_mean_state<<<bd, 128, 0, st>>>(d, G, T, t0, E1, mu_state);
  const unsigned bx = (unsigned)((s.P + 127) / 128);
  if (G <= 1 || !scratch) {
    imc_pass_c<<<dim3(bx, 1), 128, 0, st>>>(s, T, t0, order, dlt, tab, nullptr, K_state, K_t);
    return;
  }
  double* E = scratch;
  double* Cin = scratch + (int64_t)G * s.P;
  imc_pass_a<<<dim3(bx, G), 128, 0, st>>>(s, T, dlt, tab, E);
  imc_pass_b<<<bx, 128, 0, st>>>(s.P, T, G, W, t0, E, Cin, K_state);
  imc_pass_c<<<dim3(bx, G), 128, 0, st>>>(s, T, t0, order, dlt, tab, Cin, K_state, K_t);
}

size_t imc_work_doubles(int d, int T) {
  const int G = (T + kEmaChunk - 1) / kEmaChunk;
  return (size_t)T * d + 4 * (size_t)T + (size_t)G * d;
}

size_t ema_scratch_doubles(int d, int T) {
  const int G = (T + kEmaChunk - 1) / kEmaChunk;
  return G <= 1 ? 0 : (size_t)2 * G * (size_t)(packed_size(d) + d);
}

void launch_batch_ema(const BStream* S, const BItem* items, int n_items, cudaStream_t st) {
  if (n_items > 0) b_ema_kernel<<<n_items, 128, 0, st>>>(const_cast<BStream*>(S), items);
}

void launch_batch_normalise(const BStream* S, const BItem* items, int n, bool fp64,
                            cudaStream_t st) {
  if (n <= 0) return;
  if (fp64) b_normalise_kernel<double><<<n, 256, 0, st>>>(const_cast<BStream*>(S), items);
  else b_normalise_kernel<float><<<n, 256, 0, st>>>(const_cast<BStream*>(S), items);
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

const DeviceShape& device_shape() {
  static const DeviceShape shape = [] {
    DeviceShape r{1, 0};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      cudaDeviceGetAttribute(&r.n_sm, cudaDevAttrMultiProcessorCount, dev);
      cudaDeviceGetAttribute(&r.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    cudaGetLastError();
    if (r.n_sm <= 0) r.n_sm = 1;
    return r;
  }();
  return shape;
}

}  // namespace erx

// S2 line statistics (Sec. III-C): line mean and centred scatter matrix.
//
// Two routes:
//  * exact integer sums for u16 samples without projection: sum_i x_i and
//    sum_i x_i x_i^T accumulated with 32-bit integer multiply-adds (products of
//    b-bit samples are < 2^(2b); partial sums are widened to 64 bits before
//    they can wrap), so K_hat = (p S2 - S1 S1^T) / (p (p-1)) is formed later
//    from exact integers with a single rounding.  On GB300 the integer pipe
//    issues 64 IMAD/clk/SM against 2 DFMA/clk/SM.
//  * floating point: a mean pass, then the scatter of (z_i - c) about a shift c
//    accumulated in double or float; the EMA step corrects for c != mean.
//
// Both tile the lower triangle of the d x d output into 64 x 64 blocks, one
// CTA per (block pair, line); 256 threads each own a 4 x 4 sub-block.
#include "erx_batch.cuh"
#include "erx_internal.cuh"

namespace erx {
namespace {

constexpr int SB = 64;    // output block edge
constexpr int KCI = 64;   // pixels per shared-memory chunk, integer route
constexpr int KCF = 32;   // pixels per chunk, floating route
constexpr int kMeanThreads = 1024;   // line mean: threads per line

__device__ __forceinline__ void block_pair(int q, int& I, int& J) {
  int i = 0;
  while ((i + 1) * (i + 2) / 2 <= q) ++i;
  I = i;
  J = q - i * (i + 1) / 2;
}

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }

// FP32 scatter accumulation: products are summed with FMAs in runs of kRun
// pixels, and each run's sum is added into an unevaluated float pair (hi, lo)
// by Knuth's TwoSum (the exact rounding error of hi + run goes into lo).  A
// plain running FP32 sum over all p pixels loses digits at every addition to a
// sum that has grown to p products; here a run's sum holds at most kRun of them
// and the pair keeps the rest exactly, so K_hat is formed from a sum about as
// accurate as its kRun-pixel runs (the error of the scores that use it shrank
// about 15x at kappa 1e4 - 1e5 against the plain sum).  FP64 sums need none of this.
constexpr int kRun = 8;

__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bv = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__global__ void __launch_bounds__(256) stats_int_kernel(
    const uint16_t* __restrict__ X, int64_t line_stride, int W, int d, uint32_t maxv,
    int flush_mask, uint64_t* __restrict__ S1, uint64_t* __restrict__ S2,
    unsigned long long* __restrict__ err, int64_t t0) {
  __shared__ __align__(16) uint32_t xa[KCI][SB];
  __shared__ __align__(16) uint32_t xb[KCI][SB];
  int I, J;
  block_pair(blockIdx.x, I, J);
  const int t = blockIdx.y;
  const bool diag = (I == J);
  const uint16_t* x = X + (int64_t)t * line_stride;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int a0 = I * SB, b0 = J * SB;
  uint32_t acc[4][4];
  uint64_t tot[4][4];
  uint64_t s1[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0u, tot[i][j] = 0ull;
  bool bad = false;
  const uint32_t(*xbp)[SB] = diag ? xa : xb;

  for (int i0 = 0; i0 < W; i0 += KCI) {
    for (int e = threadIdx.x; e < KCI * SB; e += 256) {
      const int p = e / SB, c = e % SB, i = i0 + p;
      uint32_t va = 0, vb = 0;
      if (i < W) {
        if (a0 + c < d) va = x[(int64_t)i * d + a0 + c];
        if (!diag && b0 + c < d) vb = x[(int64_t)i * d + b0 + c];
      }
      bad |= (va > maxv) | (vb > maxv);
      xa[p][c] = va;
      if (!diag) xb[p][c] = vb;
    }
    __syncthreads();
    const int kn = min(KCI, W - i0);
    for (int k = 0; k < kn; ++k) {
      const uint4 av = *reinterpret_cast<const uint4*>(&xa[k][ty * 4]);
      const uint4 bv = *reinterpret_cast<const uint4*>(&xbp[k][tx * 4]);
      const uint32_t a[4] = {av.x, av.y, av.z, av.w};
      const uint32_t b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
      if (((k + 1) & flush_mask) == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) tot[i][j] += acc[i][j], acc[i][j] = 0u;
      }
      if (diag && ty == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) s1[j] += b[j];
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) tot[i][j] += acc[i][j], acc[i][j] = 0u;
    __syncthreads();
  }
  if (bad) atomicMin(&err[kErrRange], (unsigned long long)(t0 + t));
  uint64_t* s2 = S2 + (int64_t)t * d * d;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= d) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + tx * 4 + j;
      if (b < d) s2[(int64_t)a * d + b] = tot[i][j];
    }
  }
  if (diag && ty == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + tx * 4 + j;
      if (b < d) S1[(int64_t)t * d + b] = s1[j];
    }
  }
}

// Line mean of one line (x: its first sample, pixel stride ps): kMeanThreads
// threads, G = kMeanThreads / d of them per band, each summing every G-th pixel.
// FP64 form (float_shift false): every sample added in FP64.  Other forms:
// runs of 8 samples summed in FP32 first (relative error <= 7 * 2^-24 of the
// run, far below those forms' tolerances), an eighth of the FP64 adds.
template <typename InT>
__device__ __forceinline__ void mean_body(const InT* __restrict__ x, int ps, int W, int d,
                                          bool float_shift, double* __restrict__ mu_hat,
                                          double* __restrict__ shift) {
  __shared__ double part[kMeanThreads];
  const int G = max(1, (int)blockDim.x / d);
  const int g = threadIdx.x / d, b = threadIdx.x % d;
  double s = 0.0;
  if (g < G && float_shift) {
    for (int i = g; i < W; i += 8 * G) {
      float f = 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int ii = i + u * G;
        if (ii < W) f += (float)x[(int64_t)ii * ps + b];
      }
      s += (double)f;
    }
  } else if (g < G) {
    for (int i = g; i < W; i += G) s += to_d(x[(int64_t)i * ps + b]);
  }
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < d) {
    double tot = 0.0;
    for (int q = 0; q < G; ++q) tot += part[q * d + threadIdx.x];
    const double m = tot / (double)W;
    mu_hat[threadIdx.x] = m;
    shift[threadIdx.x] = float_shift ? (double)(float)m : m;
  }
}

template <typename InT>
__global__ void __launch_bounds__(kMeanThreads) mean_kernel(const InT* __restrict__ X, int64_t line_stride,
                                                   int ps, int W, int d, bool float_shift,
                                                   double* __restrict__ mu_hat,
                                                   double* __restrict__ shift) {
  const int t = blockIdx.x;
  mean_body<InT>(X + (int64_t)t * line_stride, ps, W, d, float_shift, mu_hat + (int64_t)t * d,
                 shift + (int64_t)t * d);
}

// One SBT x SBT block pair `pair` of the scatter of one line about `shift`
// (the line's d values), over the pixel chunks c_first .. c_last - 1
// (kScatterChunk pixels each): chunk c's sum goes to s2 (the line's d x d) when
// c == c_first, and is added to what s2 holds after that (each entry is only
// ever touched by its own thread).  256 threads, each an (SBT/16) x (SBT/16)
// sub-block; SBT = 32 wastes less of the triangle (used in FP64, where every
// multiply-add counts), SBT = 64 reuses registers more.  FP32 sums are
// compensated per kRun-pixel run (two_sum_into).
template <typename InT, typename AccT, int SBT = SB>
__device__ __forceinline__ void stats_fp_body(const InT* __restrict__ x, int ps, int W, int d,
                                              const double* __restrict__ shift,
                                              double* __restrict__ s2, int pair, int c_first,
                                              int c_last) {
  constexpr int TP = SBT / 16;
  __shared__ __align__(16) AccT xa[KCF][SBT];
  __shared__ __align__(16) AccT xb[KCF][SBT];
  __shared__ AccT cs[2 * SBT];
  int I, J;
  block_pair(pair, I, J);
  const bool diag = (I == J);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int a0 = I * SBT, b0 = J * SBT;
  if (threadIdx.x < 2 * SBT) {
    const int c = threadIdx.x < SBT ? a0 + threadIdx.x : b0 + threadIdx.x - SBT;
    cs[threadIdx.x] = c < d ? (AccT)shift[c] : (AccT)0;
  }
  constexpr bool kComp = sizeof(AccT) == 4;
  const AccT(*xbp)[SBT] = diag ? xa : xb;
  // staging: thread (sp, sc) holds column sc of the pixels sp, sp + kPStep, ...
  // of a KCF-pixel stage in registers; the next stage's loads are issued before
  // the current stage's multiply-adds, so their latency is hidden behind them
  constexpr int kPStep = 256 / SBT, kPer = KCF / kPStep;
  static_assert(kPer * kPStep == KCF, "whole stages per thread");
  const int sc = threadIdx.x % SBT, sp = threadIdx.x / SBT;
  // the raw samples are held (the centring happens at the store, so that no
  // instruction waits on these loads before the multiply-adds)
  InT pa[kPer], pb[kPer];
  uint32_t oka = 0u, okb = 0u;   // bit u: sample u is inside the line and the bands
  auto fetch = [&](int i0, int p1) {
    oka = okb = 0u;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int i = i0 + sp + u * kPStep;
      const bool va = i < p1 && a0 + sc < d, vb = !diag && i < p1 && b0 + sc < d;
      pa[u] = va ? x[(int64_t)i * ps + a0 + sc] : InT(0);
      pb[u] = vb ? x[(int64_t)i * ps + b0 + sc] : InT(0);
      oka |= (uint32_t)va << u;
      okb |= (uint32_t)vb << u;
    }
  };
  // FP64 accumulation (DFMA-bound) keeps the plain staging: each stage loaded
  // and centred just before its multiply-adds, element by element (measured
  // 11 % faster there than the batched and prefetched staging)
  constexpr bool kPrefetch = sizeof(AccT) == 4;
  const int pend = min(W, c_last * kScatterChunk);
  __syncthreads();
  if (kPrefetch && c_first * kScatterChunk < pend)
    fetch(c_first * kScatterChunk, min(W, (c_first + 1) * kScatterChunk));
  for (int ch = c_first; ch < c_last; ++ch) {
  AccT acc[TP][TP];
  float lo[TP][TP], hi[TP][TP];
#pragma unroll
  for (int i = 0; i < TP; ++i)
#pragma unroll
    for (int j = 0; j < TP; ++j) acc[i][j] = (AccT)0, lo[i][j] = 0.f, hi[i][j] = 0.f;
  const int p1 = min(W, (ch + 1) * kScatterChunk);
  for (int i0 = ch * kScatterChunk; i0 < p1; i0 += KCF) {
    if constexpr (kPrefetch) {
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        xa[sp + u * kPStep][sc] = ((oka >> u) & 1u) ? (AccT)pa[u] - cs[sc] : (AccT)0;
        if (!diag)
          xb[sp + u * kPStep][sc] = ((okb >> u) & 1u) ? (AccT)pb[u] - cs[SBT + sc] : (AccT)0;
      }
    } else {
      for (int e = threadIdx.x; e < KCF * SBT; e += 256) {
        const int p = e / SBT, c = e % SBT, i = i0 + p;
        AccT va = 0, vb = 0;
        if (i < p1) {
          if (a0 + c < d) va = (AccT)x[(int64_t)i * ps + a0 + c] - cs[c];
          if (!diag && b0 + c < d) vb = (AccT)x[(int64_t)i * ps + b0 + c] - cs[SBT + c];
        }
        xa[p][c] = va;
        if (!diag) xb[p][c] = vb;
      }
    }
    __syncthreads();
    {
      // the next stage: the rest of this chunk, else the next chunk's first
      const int nx = i0 + KCF < p1 ? i0 + KCF : (ch + 1) * kScatterChunk;
      if (kPrefetch && nx < pend) fetch(nx, min(W, (nx / kScatterChunk + 1) * kScatterChunk));
    }
    const int kn = min(KCF, p1 - i0);
    for (int k0 = 0; k0 < kn; k0 += kRun) {
      const int k1 = min(kn, k0 + kRun);
      auto step = [&](int k) {
        AccT a[TP], b[TP];
#pragma unroll
        for (int i = 0; i < TP; ++i) a[i] = xa[k][ty * TP + i], b[i] = xbp[k][tx * TP + i];
#pragma unroll
        for (int i = 0; i < TP; ++i)
#pragma unroll
          for (int j = 0; j < TP; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      };
      if (k1 - k0 == kRun) {   // a whole run (all but a chunk's ragged tail): unrolled
#pragma unroll
        for (int k = 0; k < kRun; ++k) step(k0 + k);
      } else {
        for (int k = k0; k < k1; ++k) step(k);
      }
      if constexpr (kComp) {
#pragma unroll
        for (int i = 0; i < TP; ++i)
#pragma unroll
          for (int j = 0; j < TP; ++j) {
            two_sum_into(hi[i][j], lo[i][j], (float)acc[i][j]);
            acc[i][j] = (AccT)0;
          }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TP; ++i) {
    const int a = a0 + ty * TP + i;
    if (a >= d) continue;
#pragma unroll
    for (int j = 0; j < TP; ++j) {
      const int b = b0 + tx * TP + j;
      if (b < d) {
        const double part = kComp ? (double)hi[i][j] + (double)lo[i][j] : (double)acc[i][j];
        double* o = s2 + (int64_t)a * d + b;
        *o = ch == c_first ? part : __dadd_rn(*o, part);
      }
    }
  }
  }   // chunk
}

// three CTAs per SM (two for the 64 x 64 blocks: room for the compensated FP32
// sums and the next stage's prefetched samples without spills)
template <typename InT, typename AccT, int SBT>
__global__ void __launch_bounds__(256, SBT == 64 ? 2 : 3) stats_fp_kernel(const InT* __restrict__ X,
                                                       int64_t line_stride, int ps, int W, int d,
                                                       const double* __restrict__ shift,
                                                       double* __restrict__ S2f) {
  const int t = blockIdx.y;
  stats_fp_body<InT, AccT, SBT>(X + (int64_t)t * line_stride, ps, W, d, shift + (int64_t)t * d,
                                S2f + (int64_t)t * d * d, blockIdx.x, 0, scatter_chunks(W));
}

// Small d (projected lines, d <= 16): one CTA per line, one thread per entry
// (a, b) of the lower triangle, walking all pixels; four independent partial
// sums per thread (FP32: over kRun pixels, then compensated as above).  The
// 64 x 64 tiles above would be nearly all padding here.
constexpr int kSmallD = 16;

template <typename InT, typename AccT>
__device__ __forceinline__ void stats_small_body(const InT* __restrict__ x, int ps, int W, int d,
                                                 const double* __restrict__ shift,
                                                 double* __restrict__ s2, int c_first,
                                                 int c_last) {
  const int P = d * (d + 1) / 2;
  const int q = threadIdx.x;
  if (q >= P) return;
  int a = 0;
  while ((a + 1) * (a + 2) / 2 <= q) ++a;
  const int b = q - a * (a + 1) / 2;
  const AccT ca = (AccT)shift[a], cb = (AccT)shift[b];
  constexpr bool kComp = sizeof(AccT) == 4;
  double* o = s2 + (int64_t)a * d + b;
  for (int ch = c_first; ch < c_last; ++ch) {   // chunk sums added in order, as stats_fp_body
    const int p0 = ch * kScatterChunk, p1 = min(W, p0 + kScatterChunk);
    float hi = 0.f, lo = 0.f;
    AccT s0 = 0, s1 = 0, s2a = 0, s3 = 0;
    int i = p0;
    for (; i + 4 <= p1; i += 4) {
      s0 = fma((AccT)x[(int64_t)i * ps + a] - ca, (AccT)x[(int64_t)i * ps + b] - cb, s0);
      s1 = fma((AccT)x[(int64_t)(i + 1) * ps + a] - ca, (AccT)x[(int64_t)(i + 1) * ps + b] - cb,
               s1);
      s2a = fma((AccT)x[(int64_t)(i + 2) * ps + a] - ca, (AccT)x[(int64_t)(i + 2) * ps + b] - cb,
                s2a);
      s3 = fma((AccT)x[(int64_t)(i + 3) * ps + a] - ca, (AccT)x[(int64_t)(i + 3) * ps + b] - cb,
               s3);
      if constexpr (kComp) {
        if (((i + 4 - p0) & (kRun - 1)) == 0) {   // every kRun pixels of the chunk
          two_sum_into(hi, lo, (float)((s0 + s1) + (s2a + s3)));
          s0 = s1 = s2a = s3 = 0;
        }
      }
    }
    for (; i < p1; ++i)
      s0 = fma((AccT)x[(int64_t)i * ps + a] - ca, (AccT)x[(int64_t)i * ps + b] - cb, s0);
    double part;
    if constexpr (kComp) {
      two_sum_into(hi, lo, (float)((s0 + s1) + (s2a + s3)));
      part = (double)hi + (double)lo;
    } else {
      part = (double)((s0 + s1) + (s2a + s3));
    }
    *o = ch == c_first ? part : __dadd_rn(*o, part);
  }
}

template <typename InT, typename AccT>
__global__ void __launch_bounds__(256) stats_small_kernel(const InT* __restrict__ X,
                                                          int64_t line_stride, int ps, int W,
                                                          int d, const double* __restrict__ shift,
                                                          double* __restrict__ S2f) {
  const int t = blockIdx.x;
  stats_small_body<InT, AccT>(X + (int64_t)t * line_stride, ps, W, d, shift + (int64_t)t * d,
                              S2f + (int64_t)t * d * d, 0, scatter_chunks(W));
}

__host__ __device__ inline int n_pairs(int d, int sb = SB) {
  const int nb = (d + sb - 1) / sb;
  return nb * (nb + 1) / 2;
}

// Batched form: one CTA per stream (mean) / per (stream, block pair) item.
__global__ void __launch_bounds__(kMeanThreads) b_mean_kernel(const BStream* __restrict__ S,
                                                              const BItem* __restrict__ items,
                                                              bool float_shift) {
  const BStream& s = S[items[blockIdx.x].s];
  mean_body<float>(s.x, s.d, s.W, s.d, float_shift, s.mu_hat, s.shift);
}

template <typename AccT>
__global__ void __launch_bounds__(256, sizeof(AccT) == 4 ? 2 : 3) b_stats_kernel(const BStream* __restrict__ S,
                                                      const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  const BStream& s = S[it.s];
  const int64_t dd = (int64_t)s.d * s.d;
  if (s.d <= kSmallD) {
    const int ch = it.tile;
    stats_small_body<float, AccT>(s.x, s.d, s.W, s.d, s.shift, s.S2f + ch * dd, ch, ch + 1);
  } else if (sizeof(AccT) == 8 || s.d <= 32) {   // 32 x 32 blocks, as the single-stream path
    const int np = n_pairs(s.d, 32), pr = it.tile % np, ch = it.tile / np;
    stats_fp_body<float, AccT, 32>(s.x, s.d, s.W, s.d, s.shift, s.S2f + ch * dd, pr, ch, ch + 1);
  } else {
    const int np = n_pairs(s.d, SB), pr = it.tile % np, ch = it.tile / np;
    stats_fp_body<float, AccT, SB>(s.x, s.d, s.W, s.d, s.shift, s.S2f + ch * dd, pr, ch, ch + 1);
  }
}

}  // namespace

// output block edge of the floating scatter: 32 in FP64 (every multiply-add
// counts) and for d <= 32 (a 64 x 64 block would leave three quarters of the
// threads idle), 64 otherwise
int fp_block(int d, bool fp64) { return fp64 || d <= 32 ? 32 : SB; }

// work items of one stream's scatter: (block pair, pixel chunk); d <= 16: (chunk)
int batch_stats_tiles(int d, int W, bool fp64) {
  return (d <= kSmallD ? 1 : n_pairs(d, fp_block(d, fp64))) * scatter_chunks(W);
}
int batch_scatter_chunks(int, int W) { return scatter_chunks(W); }

void launch_batch_mean(const BStream* S, const BItem* items, int n, bool float_shift,
                       cudaStream_t st) {
  if (n > 0) b_mean_kernel<<<n, kMeanThreads, 0, st>>>(S, items, float_shift);
}

void launch_batch_stats(const BStream* S, const BItem* items, int n_items, bool fp64,
                        cudaStream_t st) {
  if (n_items <= 0) return;
  if (fp64) b_stats_kernel<double><<<n_items, 256, 0, st>>>(S, items);
  else b_stats_kernel<float><<<n_items, 256, 0, st>>>(S, items);
}

void launch_stats_int(const uint16_t* x, int64_t line_stride, int W, int d, uint32_t maxv,
                      int T, uint64_t* S1, uint64_t* S2, unsigned long long* err, int64_t t0,
                      cudaStream_t st) {
  // flush 32-bit partial sums every F pixels with F * maxv^2 < 2^32, F a power of 2 <= 64
  const uint64_t m2 = (uint64_t)maxv * maxv;
  int f = 64;
  while (f > 1 && (uint64_t)f * m2 > 0xFFFFFFFFull) f >>= 1;
  dim3 grid(n_pairs(d), T);
  stats_int_kernel<<<grid, 256, 0, st>>>(x, line_stride, W, d, maxv, f - 1, S1, S2, err, t0);
}

void launch_mean(int in_type, const void* x, int64_t line_stride, int ps, int W, int d, int T,
                 bool float_shift, double* mu_hat, double* shift, cudaStream_t st) {
  if (in_type == 0)
    mean_kernel<uint16_t><<<T, kMeanThreads, 0, st>>>((const uint16_t*)x, line_stride, ps, W, d,
                                             float_shift, mu_hat, shift);
  else if (in_type == 1)
    mean_kernel<float><<<T, kMeanThreads, 0, st>>>((const float*)x, line_stride, ps, W, d, float_shift,
                                          mu_hat, shift);
  else
    mean_kernel<double><<<T, kMeanThreads, 0, st>>>((const double*)x, line_stride, ps, W, d, float_shift,
                                           mu_hat, shift);
}

void launch_stats_fp(int in_type, bool fp64, const void* x, int64_t line_stride, int ps, int W,
                     int d, int T, const double* shift, double* S2f, cudaStream_t st) {
  if (d <= kSmallD) {
#define ERX_SMALL(IT, AT) \
  stats_small_kernel<IT, AT><<<T, 256, 0, st>>>((const IT*)x, line_stride, ps, W, d, shift, S2f)
    if (fp64) {
      if (in_type == 0) ERX_SMALL(uint16_t, double);
      else if (in_type == 1) ERX_SMALL(float, double);
      else ERX_SMALL(double, double);
    } else {
      if (in_type == 0) ERX_SMALL(uint16_t, float);
      else if (in_type == 1) ERX_SMALL(float, float);
      else ERX_SMALL(double, float);
    }
#undef ERX_SMALL
    return;
  }
  // FP64 and d <= 32: 32 x 32 blocks; FP32 otherwise: 64 x 64
  const int sbt = fp_block(d, fp64);
  const dim3 grid(n_pairs(d, sbt), T);
#define ERX_SFP(IT, AT, SBT)                                                                \
  stats_fp_kernel<IT, AT, SBT><<<grid, 256, 0, st>>>((const IT*)x, line_stride, ps, W, d, \
                                                     shift, S2f)
  if (fp64) {
    if (in_type == 0) ERX_SFP(uint16_t, double, 32);
    else if (in_type == 1) ERX_SFP(float, double, 32);
    else ERX_SFP(double, double, 32);
  } else if (sbt == 32) {
    if (in_type == 0) ERX_SFP(uint16_t, float, 32);
    else if (in_type == 1) ERX_SFP(float, float, 32);
    else ERX_SFP(double, float, 32);
  } else {
    if (in_type == 0) ERX_SFP(uint16_t, float, SB);
    else if (in_type == 1) ERX_SFP(float, float, SB);
    else ERX_SFP(double, float, SB);
  }
#undef ERX_SFP
}

}  // namespace erx

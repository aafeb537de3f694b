// S5 (Sec. III-D): delta_i = sqrt(m_i . m_i) with L_t m_i = z_i - mu_t.
//
// FP64 form: solves block by block with the blocked factor of k_factor.cu
// (packed L_t whose 32 x 32 diagonal blocks hold D_J = L_JJ^{-1}):
//   y_J = r_J - sum_{k < j0} L_Jk m_k,   m_J = D_J y_J,
// exactly d(d+1)/2 multiply-adds per pixel, as forward substitution.
// one thread per pixel.  The pixel's centred vector r_i is staged
// in shared memory (odd row pitch, so the 8-byte loads of a warp hit distinct
// bank pairs) and overwritten by m_i block by block; rows of the factor are
// read with warp-uniform loads; the 32 values y_J of a block sit in
// registers.  The kernel is bound by the FP64 pipe (2 DFMA/clk/SM on GB300).
//
// FP32 form: with the full inverse X = L^{-1} (FP32, from the blocked factor),
// m = X r is one lower-triangular product, register-tiled over pixels x
// outputs.  A CTA owns 64 pixels; four warps cover 64 pixels x 32 outputs of
// a block, each thread a 4 x 4 tile; R^T is kept k-major in shared memory and
// each 32-row band of X is staged k-major, so both operand loads are 16-byte
// and conflict-free.  The centred samples are (x - mu_hi) - mu_lo with mu split
// into two floats, which keeps r accurate to float rounding without FP64 work
// per pixel.
#include <algorithm>
#include <cmath>

#include "erx_batch.cuh"
#include "erx_internal.cuh"

namespace erx {
namespace {

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }
template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

constexpr int kPixF64 = 64;
constexpr int kNB = kFactorBlock;

// Pixels tile*64 .. tile*64+63 of one line (x, pixel stride ps) scored with
// mu (d) and the blocked factor L (packed); delta: the line's W scores.
template <typename InT>
__device__ __forceinline__ void solve_fp64_body(const InT* __restrict__ x, int ps, int W, int d,
                                                const double* __restrict__ mu,
                                                const double* __restrict__ L,
                                                double* __restrict__ delta, int tile) {
  extern __shared__ __align__(16) double r[];
  const int dp = d | 1;
  const int i0 = tile * kPixF64;
  for (int e = threadIdx.x; e < kPixF64 * d; e += kPixF64) {
    const int p = e / d, k = e - p * d, i = i0 + p;
    r[p * dp + k] = i < W ? to_d(x[(int64_t)i * ps + k]) - mu[k] : 0.0;
  }
  __syncthreads();
  const int i = i0 + threadIdx.x;
  if (i >= W) return;
  double* rr = r + threadIdx.x * dp;
  double d2 = 0.0;
  for (int j0 = 0; j0 < d; j0 += kNB) {
    const int nb = min(kNB, d - j0);
    double y[kNB];
#pragma unroll
    for (int jj = 0; jj < kNB; ++jj) {
      y[jj] = 0.0;
      if (jj < nb) {
        const int j = j0 + jj;
        const double* Lj = L + j * (j + 1) / 2;
        // one chain: a warp's DFMA holds its SMSP's share of the FP64 pipe
        // (0.5 lane/clk) for longer than the result latency, so a dependent
        // chain does not stall, and no combining additions are needed
        double a0 = rr[j];
        for (int k = 0; k < j0; ++k) a0 = fma(-__ldg(Lj + k), rr[k], a0);
        y[jj] = a0;
      }
    }
#pragma unroll
    for (int jj = 0; jj < kNB; ++jj) {
      if (jj < nb) {
        const int j = j0 + jj;
        const double* Dj = L + j * (j + 1) / 2 + j0;
        double s = 0.0;
#pragma unroll
        for (int kk = 0; kk <= jj; ++kk) s = fma(__ldg(Dj + kk), y[kk], s);
        rr[j] = s;
        d2 = fma(s, s, d2);
      }
    }
  }
  delta[i] = sqrt(d2);
}

// H threads per pixel, NPX pixels per tile (H * NPX threads).  Per 32-row
// block the H threads of a pixel take the rows jj = H u + h of y_J (written in
// place of r_J), then the same rows of m_J = D_J y_J, held in registers until
// all have read y_J; the squares are summed in row order by one thread.  Every
// sum is taken in the same order as in the one-thread body, so all variants
// give the same bits.  Uses:
//  * large d (> 128), H = 2, NPX = 64: a 64-pixel tile holds 113 KiB of
//    residuals, two CTAs fit on an SM, and one thread per pixel would be four
//    warps per SM, too few to cover the DFMA chains and the L2 reads of L;
//  * launches with fewer 64-pixel tiles than SMs (a line or a few pushed
//    alone), H = 16, NPX = 8: the line's pixels spread over up to 8x as many
//    SMs, four warps each, so a single line's score takes a few tens of
//    microseconds instead of the 10 SMs' worth of FP64 time.
template <typename InT, int H, int NPX>
__device__ __forceinline__ void solve_fp64_multi_body(const InT* __restrict__ x, int ps, int W,
                                                      int d, const double* __restrict__ mu,
                                                      const double* __restrict__ L,
                                                      double* __restrict__ delta, int tile) {
  extern __shared__ __align__(16) double r[];
  const int dp = d | 1;
  const int i0 = tile * NPX;
  for (int e = threadIdx.x; e < NPX * d; e += H * NPX) {
    const int p = e / d, k = e - p * d, i = i0 + p;
    r[p * dp + k] = i < W ? to_d(x[(int64_t)i * ps + k]) - mu[k] : 0.0;
  }
  __syncthreads();
  const int p = threadIdx.x % NPX, h = threadIdx.x / NPX;   // pixel, row phase
  const int i = i0 + p;
  double* rr = r + p * dp;
  for (int j0 = 0; j0 < d; j0 += kNB) {
    const int nb = min(kNB, d - j0);
#pragma unroll
    for (int u = 0; u < kNB / H; ++u) {
      const int jj = H * u + h;
      if (jj < nb) {
        const int j = j0 + jj;
        const double* Lj = L + j * (j + 1) / 2;
        double a0 = rr[j];
        for (int k = 0; k < j0; ++k) a0 = fma(-__ldg(Lj + k), rr[k], a0);
        rr[j] = a0;
      }
    }
    __syncthreads();
    double m[kNB / H];
#pragma unroll
    for (int u = 0; u < kNB / H; ++u) {
      const int jj = H * u + h;
      double s = 0.0;
      if (jj < nb) {
        const double* Dj = L + (j0 + jj) * (j0 + jj + 1) / 2 + j0;
        const double* yj = rr + j0;
#pragma unroll
        for (int kk = 0; kk < H * u + H; ++kk)
          if (kk <= jj) s = fma(__ldg(Dj + kk), yj[kk], s);
      }
      m[u] = s;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kNB / H; ++u)
      if (H * u + h < nb) rr[j0 + H * u + h] = m[u];
    __syncthreads();
  }
  if (h == 0 && i < W) {
    double d2 = 0.0;
    for (int j = 0; j < d; ++j) d2 = fma(rr[j], rr[j], d2);
    delta[i] = sqrt(d2);
  }
}

// Persistent grid (a whole number of waves): CTA c takes tiles c, c + grid, ...
// of the T x ntiles (line, tile) pairs.  H = 1: one thread per pixel.
template <typename InT, int H, int NPX>
__global__ void __launch_bounds__(H * NPX) solve_fp64_kernel(
    const InT* __restrict__ X, int64_t line_stride, int ps, int W, int d,
    const double* __restrict__ mu_t, const double* __restrict__ Lf, double* __restrict__ delta,
    int T) {
  const int ntiles = (W + NPX - 1) / NPX;
  const int64_t total = (int64_t)T * ntiles;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int t = (int)(w / ntiles), tile = (int)(w % ntiles);
    __syncthreads();          // the previous tile's threads are done with shared memory
    if constexpr (H == 1)
      solve_fp64_body<InT>(X + (int64_t)t * line_stride, ps, W, d, mu_t + (int64_t)t * d,
                           Lf + (int64_t)t * packed_size(d), delta + (int64_t)t * W, tile);
    else
      solve_fp64_multi_body<InT, H, NPX>(X + (int64_t)t * line_stride, ps, W, d,
                                         mu_t + (int64_t)t * d, Lf + (int64_t)t * packed_size(d),
                                         delta + (int64_t)t * W, tile);
  }
}

// Lines scored alone (fewer 64-pixel tiles than SMs): NPX pixels per CTA, H
// threads per pixel, over a persistent grid.  The CTA stages the line's
// blocked factor in shared memory once (coalesced; the other layouts read it
// from L2 row by row, a dependent load per multiply-add), and the solve is
// reorganised right-looking: once m_J of block J is final, every row of the
// later blocks takes block J's 32 terms, two rows per thread at a time, so a
// thread runs independent chains instead of one long one.  Every y_j
// still receives its multiply-adds in ascending k, m_J = D_J y_J its terms in
// ascending order, and the squares are summed in row order: the bits of the
// other layouts.
template <typename InT, int H, int NPX>
__global__ void __launch_bounds__(H * NPX, 1) solve_fp64_line_kernel(
    const InT* __restrict__ X, int64_t line_stride, int ps, int W, int d,
    const double* __restrict__ mu_t, const double* __restrict__ Lf, double* __restrict__ delta,
    int T) {
  constexpr int NT = H * NPX;
  extern __shared__ __align__(16) double sm[];
  const int P = d * (d + 1) / 2;
  const int dp = d | 1;
  double* Ls = sm;                          // the packed blocked factor
  double* r = sm + ((P + 1) & ~1);          // [NPX][dp] residuals, overwritten by m
  const int tid = threadIdx.x;
  const int p = tid % NPX, h = tid / NPX;
  double* rr = r + p * dp;
  const int ntiles = (W + NPX - 1) / NPX;
  const int64_t total = (int64_t)T * ntiles;
  int staged = -1;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int t = (int)(w / ntiles), tile = (int)(w % ntiles);
    __syncthreads();                        // the previous tile is done with shared memory
    // staging: eight loads in flight per thread before their stores
    if (t != staged) {
      const double* L = Lf + (int64_t)t * P;
      for (int q0 = tid; q0 < P; q0 += 8 * NT) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (q0 + u * NT < P) v[u] = __ldg(L + q0 + u * NT);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (q0 + u * NT < P) Ls[q0 + u * NT] = v[u];
      }
      staged = t;
    }
    const InT* x = X + (int64_t)t * line_stride;
    const double* mu = mu_t + (int64_t)t * d;
    const int i0 = tile * NPX;
#pragma unroll
    for (int pp = 0; pp < NPX; ++pp) {
      const int i = i0 + pp;
      for (int k = tid; k < d; k += NT)
        r[pp * dp + k] = i < W ? to_d(__ldg(x + (int64_t)i * ps + k)) - __ldg(mu + k) : 0.0;
    }
    __syncthreads();
    static_assert(H >= kNB + 1, "rows of a block on threads h < 32, the squares on h = H - 1");
    double d2 = 0.0;                       // the squares, in row order (thread h = H - 1)
    for (int j0 = 0; j0 < d; j0 += kNB) {
      const int nb = min(kNB, d - j0);
      // m_J = D_J y_J: thread h < nb takes row h (h + 1 multiply-adds, ascending)
      double s1 = 0.0;
      if (h < nb) {
        const double* D1 = Ls + (j0 + h) * (j0 + h + 1) / 2 + j0;
        const double* y = rr + j0;
#pragma unroll 4
        for (int kk = 0; kk <= h; ++kk) s1 = fma(D1[kk], y[kk], s1);
      } else if (h == H - 1 && j0 > 0) {
        // meanwhile the previous block's squares (its m are final)
#pragma unroll 8
        for (int jj = 0; jj < kNB; ++jj) d2 = fma(rr[j0 - kNB + jj], rr[j0 - kNB + jj], d2);
      }
      __syncthreads();
      if (h < nb) rr[j0 + h] = s1;
      __syncthreads();
      if (j0 + kNB >= d && h == H - 1)   // the last block's squares
        for (int jj = 0; jj < nb; ++jj) d2 = fma(rr[j0 + jj], rr[j0 + jj], d2);
      // rows of the later blocks take this block's terms, k ascending (a block
      // with rows after it is a whole one): rows dealt out one per thread per
      // pass, two passes at a time so that each thread runs two chains
      const double* mJ = rr + j0;
      for (int j = j0 + kNB + h; j < d; j += 2 * H) {
        const int j2 = j + H < d ? j + H : j;
        const double* L1 = Ls + j * (j + 1) / 2 + j0;
        const double* L2 = Ls + j2 * (j2 + 1) / 2 + j0;
        double a1 = rr[j], a2 = rr[j2];
#pragma unroll
        for (int kk = 0; kk < kNB; ++kk) {
          const double mk = mJ[kk];
          a1 = fma(-L1[kk], mk, a1);
          a2 = fma(-L2[kk], mk, a2);
        }
        rr[j] = a1;
        if (j2 != j) rr[j2] = a2;
      }
      __syncthreads();
    }
    if (h == H - 1 && i0 + p < W) delta[(int64_t)t * W + i0 + p] = sqrt(d2);
  }
}

// Batched form: one CTA per (stream, pixel tile) item, H threads per pixel
// over NPX-pixel tiles (the layouts of the single-stream path, same bits):
// layout 0 = (1, 64), 1 = (2, 64), 2 = (16, 8); chosen per band count by the
// autotuner (default: 1 above 128 dimensions, else 0).
template <int H, int NPX>
__global__ void __launch_bounds__(H * NPX) b_solve_fp64_kernel(
    const BStream* __restrict__ S, const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  const BStream& s = S[it.s];
  if constexpr (H == 1)
    solve_fp64_body<float>(s.x, s.d, s.W, s.d, s.mu_t, s.Lf, (double*)s.delta, it.tile);
  else
    solve_fp64_multi_body<float, H, NPX>(s.x, s.d, s.W, s.d, s.mu_t, s.Lf, (double*)s.delta,
                                         it.tile);
}

constexpr int kPixF32 = 64;   // pixels per CTA
constexpr int kOutB = kNB;    // outputs per block of the factor
constexpr int kLS = kOutB + 4;   // row pitch of the staged factor band (16-byte multiple)

template <typename InT>
__device__ __forceinline__ void solve_fp32_body(const InT* __restrict__ x, int ps, int W, int d,
                                                const double* __restrict__ mu,
                                                const float* __restrict__ Lg,
                                                float* __restrict__ delta, int tile) {
  extern __shared__ __align__(16) float smf[];
  float* rT = smf;                          // [d][kPixF32]: r, k-major
  float* LT = smf + d * kPixF32;            // [d][kLS]: rows of L^{-1}, k-major
  __shared__ float mu_hi[kMaxDim], mu_lo[kMaxDim];
  __shared__ float d2w[2][kPixF32];
  const int i0 = tile * kPixF32;
  for (int k = threadIdx.x; k < d; k += 128) {
    const double m = mu[k];
    const float h = (float)m;
    mu_hi[k] = h;
    mu_lo[k] = (float)(m - (double)h);
  }
  __syncthreads();
  // pixel-fastest, so the transposed stores hit distinct banks.  Where pixel
  // rows allow it, four consecutive bands per load (16 bytes of float, 8 of u16)
  constexpr bool kVecIn = sizeof(InT) <= 4;
  const bool vec = kVecIn && (d % 4) == 0 && (ps % 4) == 0 &&
                   ((uintptr_t)x % (4 * sizeof(InT))) == 0;
  if (vec) {
    const int p = threadIdx.x & (kPixF32 - 1), i = i0 + p;
    const InT* xp = x + (int64_t)(i < W ? i : 0) * ps;
#pragma unroll 4
    for (int k4 = (threadIdx.x / kPixF32) * 4; k4 < d; k4 += 8) {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (i < W) {
        if constexpr (sizeof(InT) == 4) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(xp + k4));
          v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
        } else if constexpr (sizeof(InT) == 2) {
          const uint2 w = __ldg(reinterpret_cast<const uint2*>(xp + k4));
          v[0] = (float)(w.x & 0xffffu), v[1] = (float)(w.x >> 16);
          v[2] = (float)(w.y & 0xffffu), v[3] = (float)(w.y >> 16);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (v[u] - mu_hi[k4 + u]) - mu_lo[k4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) rT[(k4 + u) * kPixF32 + p] = v[u];
    }
  } else {
    for (int e = threadIdx.x; e < kPixF32 * d; e += 128) {
      const int k = e / kPixF32, p = e - k * kPixF32, i = i0 + p;
      float v = 0.f;
      if (i < W) v = (to_f(x[(int64_t)i * ps + k]) - mu_hi[k]) - mu_lo[k];
      rT[k * kPixF32 + p] = v;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ph = warp & 1, oh = warp >> 1;
  const int lp = lane & 7, lo = lane >> 3;
  const int pcol = ph * 32 + lp * 4;        // first of this thread's 4 pixels
  const int ocol = oh * 16 + lo * 4;        // first of its 4 outputs within a block
  float d2[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < d; j0 += kOutB) {
    const int j1 = min(d, j0 + kOutB);
    __syncthreads();
    // one warp per row of the band, lanes along k: each row is read contiguously
    for (int jj = warp; jj < kOutB; jj += 4) {
      const int j = j0 + jj;
      const float* Lj = Lg + j * (j + 1) / 2;
      for (int k = lane; k < j1; k += 32) LT[k * kLS + jj] = (j < d && k <= j) ? Lj[k] : 0.f;
    }
    __syncthreads();
    // m_J = X_{J, k < j1} r (X = L^{-1}: lower triangular, zeros above the diagonal)
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
    for (int k = 0; k < j1; ++k) {
      const float4 rv = *reinterpret_cast<const float4*>(rT + k * kPixF32 + pcol);
      const float4 lv = *reinterpret_cast<const float4*>(LT + k * kLS + ocol);
      const float ra[4] = {rv.x, rv.y, rv.z, rv.w};
      const float la[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ra[a], la[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) d2[a] = fmaf(acc[a][b], acc[a][b], d2[a]);
  }
  // reduce over the 4 output groups of a warp (lane bits 3, 4), then the 2 output halves
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    d2[a] += __shfl_xor_sync(0xffffffffu, d2[a], 8);
    d2[a] += __shfl_xor_sync(0xffffffffu, d2[a], 16);
  }
  __syncthreads();
  if (lo == 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a) d2w[oh][pcol + a] = d2[a];
  }
  __syncthreads();
  if (threadIdx.x < kPixF32) {
    const int i = i0 + threadIdx.x;
    if (i < W) delta[i] = sqrtf(d2w[0][threadIdx.x] + d2w[1][threadIdx.x]);
  }
}

template <typename InT>
__global__ void __launch_bounds__(128) solve_fp32_kernel(
    const InT* __restrict__ X, int64_t line_stride, int ps, int W, int d,
    const double* __restrict__ mu_t, const float* __restrict__ Lf32, float* __restrict__ delta) {
  const int t = blockIdx.y;
  solve_fp32_body<InT>(X + (int64_t)t * line_stride, ps, W, d, mu_t + (int64_t)t * d,
                       Lf32 + (int64_t)t * packed_size(d), delta + (int64_t)t * W, blockIdx.x);
}



__global__ void __launch_bounds__(128) b_solve_fp32_kernel(const BStream* __restrict__ S,
                                                           const BItem* __restrict__ items) {
  const BItem it = items[blockIdx.x];
  const BStream& s = S[it.s];
  solve_fp32_body<float>(s.x, s.d, s.W, s.d, s.mu_t, s.Lf32, (float*)s.delta, it.tile);
}

size_t smem_fp64(int d, int npx = kPixF64) { return (size_t)npx * (d | 1) * sizeof(double); }
size_t smem_fp32(int d) {
  return (size_t)d * (kPixF32 + kLS) * sizeof(float);
}

}  // namespace

// single lines: 48 threads per pixel over 5-pixel tiles (8 warps; 128 CTAs, one
// per SM, for a 640-pixel line)
constexpr int kLineH = 48, kLinePix = 5;
size_t line_smem(int d) {
  return (size_t)(((packed_size(d) + 1) & ~1) + kLinePix * (d | 1)) * sizeof(double);
}

cudaError_t configure_solve_kernels() {
  cudaError_t e = cudaSuccess;
  const int m64 = (int)smem_fp64(kMaxDim), m32 = (int)smem_fp32(kMaxDim);
#define ERX_CFG(K, M) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, M)
#define ERX_CFG3(IT)                                 \
  ERX_CFG((solve_fp64_kernel<IT, 1, kPixF64>), m64); \
  ERX_CFG((solve_fp64_kernel<IT, 2, kPixF64>), m64); \
  ERX_CFG((solve_fp64_kernel<IT, 16, 8>), m64);     \
  ERX_CFG((solve_fp64_line_kernel<IT, kLineH, kLinePix>), (int)line_smem(kMaxDim));
  ERX_CFG3(uint16_t)
  ERX_CFG3(float)
  ERX_CFG3(double)
#undef ERX_CFG3
  // residual tiles take nearly all of the SM's shared memory (two 113 KiB
  // tiles at d = 224); L streams through L2
#define ERX_CARVE(K)     \
  if (e == cudaSuccess) \
  e = cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout, 100)
  ERX_CARVE((solve_fp64_kernel<uint16_t, 1, kPixF64>));
  ERX_CARVE((solve_fp64_kernel<float, 1, kPixF64>));
  ERX_CARVE((solve_fp64_kernel<double, 1, kPixF64>));
  ERX_CARVE((solve_fp64_kernel<uint16_t, 2, kPixF64>));
  ERX_CARVE((solve_fp64_kernel<float, 2, kPixF64>));
  ERX_CARVE((solve_fp64_kernel<double, 2, kPixF64>));
#undef ERX_CARVE
  ERX_CFG(solve_fp32_kernel<uint16_t>, m32);
  ERX_CFG(solve_fp32_kernel<float>, m32);
  ERX_CFG(solve_fp32_kernel<double>, m32);
  ERX_CFG((b_solve_fp64_kernel<1, kPixF64>), m64);
  ERX_CFG((b_solve_fp64_kernel<2, kPixF64>), m64);
  ERX_CFG((b_solve_fp64_kernel<16, 8>), m64);
  ERX_CFG(b_solve_fp32_kernel, m32);
#undef ERX_CFG
  return e;
}

// pixel tiles of one stream's score: route 0 (FP64) by its thread layout
int batch_solve_tiles(int route, int W, int layout) {
  return route == 0 ? (W + (layout == 2 ? 8 : kPixF64) - 1) / (layout == 2 ? 8 : kPixF64)
                    : route == 1 ? (W + kPixF32 - 1) / kPixF32 : (W + 127) / 128;
}

void launch_batch_solve_simt(const BStream* S, const BItem* items, int n_items, int dmax,
                             cudaStream_t st) {
  if (n_items > 0) b_solve_fp32_kernel<<<n_items, 128, smem_fp32(dmax), st>>>(S, items);
}

// FP64 route, the items of one thread layout (dmax: their streams' largest d)
void launch_batch_solve_fp64(int layout, const BStream* S, const BItem* items, int n_items,
                             int dmax, cudaStream_t st) {
  if (n_items <= 0) return;
  if (layout == 0)
    b_solve_fp64_kernel<1, kPixF64><<<n_items, kPixF64, smem_fp64(dmax), st>>>(S, items);
  else if (layout == 1)
    b_solve_fp64_kernel<2, kPixF64><<<n_items, 2 * kPixF64, smem_fp64(dmax), st>>>(S, items);
  else
    b_solve_fp64_kernel<16, 8><<<n_items, 128, smem_fp64(dmax, 8), st>>>(S, items);
}

constexpr int kPairMinD = 129;   // two threads per pixel from here on

template <typename InT, int H, int NPX>
void launch_fp64_t(const InT* x, int64_t line_stride, int ps, int W, int d, int T,
                   const double* mu_t, const double* Linv, double* delta, int n_sm,
                   cudaStream_t st) {
  const int threads = H * NPX;
  const size_t sm = (size_t)NPX * (d | 1) * sizeof(double);
  // a whole number of waves: resident CTAs per SM times the SM count
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_fp64_kernel<InT, H, NPX>, threads,
                                                sm);
  per_sm = std::max(1, per_sm);
  const int64_t total = (int64_t)T * ((W + NPX - 1) / NPX);
  const int grid = (int)std::min<int64_t>(total, (int64_t)n_sm * per_sm);
  solve_fp64_kernel<InT, H, NPX><<<grid, threads, sm, st>>>(x, line_stride, ps, W, d, mu_t,
                                                             Linv, delta, T);
}

template <typename InT>
void launch_fp64_line(const InT* x, int64_t line_stride, int ps, int W, int d, int T,
                      const double* mu_t, const double* Linv, double* delta, int n_sm,
                      cudaStream_t st) {
  const size_t sm = line_smem(d);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, solve_fp64_line_kernel<InT, kLineH, kLinePix>, kLineH * kLinePix, sm);
  per_sm = std::max(1, per_sm);
  const int64_t total = (int64_t)T * ((W + kLinePix - 1) / kLinePix);
  const int grid = (int)std::min<int64_t>(total, (int64_t)n_sm * per_sm);
  solve_fp64_line_kernel<InT, kLineH, kLinePix><<<grid, kLineH * kLinePix, sm, st>>>(
      x, line_stride, ps, W, d, mu_t, Linv, delta, T);
}

template <typename InT>
void launch_fp64_in(const InT* x, int64_t line_stride, int ps, int W, int d, int T,
                    const double* mu_t, const double* Linv, double* delta, cudaStream_t st) {
  const int n_sm = device_shape().n_sm;
  const int64_t tiles64 = (int64_t)T * ((W + kPixF64 - 1) / kPixF64);
  if (tiles64 < n_sm)
    launch_fp64_line<InT>(x, line_stride, ps, W, d, T, mu_t, Linv, delta, n_sm, st);
  else if (d >= kPairMinD)
    launch_fp64_t<InT, 2, kPixF64>(x, line_stride, ps, W, d, T, mu_t, Linv, delta, n_sm, st);
  else
    launch_fp64_t<InT, 1, kPixF64>(x, line_stride, ps, W, d, T, mu_t, Linv, delta, n_sm, st);
}

void launch_solve_fp64(int in_type, const void* x, int64_t line_stride, int ps, int W, int d,
                       int T, const double* mu_t, const double* Linv, double* delta,
                       cudaStream_t st) {
  if (in_type == 0)
    launch_fp64_in((const uint16_t*)x, line_stride, ps, W, d, T, mu_t, Linv, delta, st);
  else if (in_type == 1)
    launch_fp64_in((const float*)x, line_stride, ps, W, d, T, mu_t, Linv, delta, st);
  else
    launch_fp64_in((const double*)x, line_stride, ps, W, d, T, mu_t, Linv, delta, st);
}

void launch_solve_fp32(int in_type, const void* x, int64_t line_stride, int ps, int W, int d,
                       int T, const double* mu_t, const float* Linv32, float* delta,
                       cudaStream_t st) {
  dim3 grid((W + kPixF32 - 1) / kPixF32, T);
  const size_t sm = smem_fp32(d);
  if (in_type == 0)
    solve_fp32_kernel<uint16_t><<<grid, 128, sm, st>>>((const uint16_t*)x, line_stride, ps, W,
                                                       d, mu_t, Linv32, delta);
  else if (in_type == 1)
    solve_fp32_kernel<float><<<grid, 128, sm, st>>>((const float*)x, line_stride, ps, W, d,
                                                    mu_t, Linv32, delta);
  else
    solve_fp32_kernel<double><<<grid, 128, sm, st>>>((const double*)x, line_stride, ps, W, d,
                                                     mu_t, Linv32, delta);
}

}  // namespace erx

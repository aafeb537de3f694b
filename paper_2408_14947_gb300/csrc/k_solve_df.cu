// S5 (Sec. III-D) with FP64-level accuracy on the FP32 pipe: double-float
// arithmetic (ERX_FORM_FP64E).
//
// GB300 issues 61x more FP32 than FP64 work per clock.  Here every value of the
// score (the residual r = z - mu_t, the blocked factor, y, m and |m|^2) is a
// double-float: an unevaluated sum hi + lo of two floats, about 48 significant
// bits.  The building blocks are the error-free transformations:
//   TwoSum(a, b):  s = a + b, e = (a - (s - (s - a))) + (b - (s - a)), s + e = a + b exactly;
//   TwoProd(a, b): p = a b, e = fma(a, b, -p), p + e = a b exactly;
// Every sum of products (the rows of y and m, and |m|^2) is a compensated dot
// product in the manner of Ogita, Rump and Oishi's Dot2 ("Accurate sum and
// dot product", 2005) with double-float operands: the running sum takes each
// rounded product exactly by TwoSum, a second float gathers the products'
// and the sums' rounding errors (the term bl cl is dropped, below 2^-48 of the
// product), and the pair is renormalised once at the end.  12 FP32 operations
// per term.  The operations use the _rn intrinsics so the compiler cannot fuse
// a product into a following sum (which would break TwoSum).
//
// The solve is the blocked one of the FP64 form (k_solve.cu): per 32-row
// block, y_J = r_J - sum_{k < j0} L_Jk m_k, then m_J = D_J y_J, with the
// pixel's residuals in shared memory (float2 hi/lo, odd row pitch).  Four
// threads share a pixel (rows 4u + h of each block: eight independent chains
// per thread) over 32-pixel tiles, so up to 16 warps per SM keep the FP32 pipe
// issuing; each 32-row block of the factor is staged in shared memory once per
// tile.  delta = sqrt(hi + lo) in FP64.  The factor and mu_t are split into
// hi/lo floats per line by a first kernel.
#include <algorithm>
#include <cmath>

#include "erx_internal.cuh"

namespace erx {
namespace {

constexpr int kNB = kFactorBlock;

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

// One term of a compensated dot product (Ogita, Rump and Oishi's Dot2, with
// double-float operands): the running sum s takes the rounded product exactly
// (TwoSum), c gathers the rounding errors of the products and of the sums;
// s + c is renormalised once at the end (df_norm).  s -= b c.
__device__ __forceinline__ void dot2_fnma(float& s, float& c, float bh, float bl, float ch,
                                          float cl) {
  const float p = __fmul_rn(bh, ch);
  float q = __fmaf_rn(bh, ch, -p);
  q = __fmaf_rn(bh, cl, q);
  q = __fmaf_rn(bl, ch, q);
  const float t = __fsub_rn(s, p);
  const float v = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(-p, v));
  c = __fadd_rn(c, __fsub_rn(e, q));
  s = t;
}

// (s, c) -> a normalised double-float (Fast2Sum: |c| is far below |s| or s is 0)
__device__ __forceinline__ float2 df_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

// x - mu for an exact float x and a double-float mu
__device__ __forceinline__ float2 df_sub(float x, float2 mu) {
  const float sh = __fsub_rn(x, mu.x);
  const float v = __fsub_rn(sh, x);
  const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(sh, v)), __fsub_rn(-mu.x, v));
  const float el = __fsub_rn(e, mu.y);
  const float nh = __fadd_rn(sh, el);
  return make_float2(nh, __fsub_rn(el, __fsub_rn(nh, sh)));
}

__device__ __forceinline__ float2 split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// per line: the blocked factor (P values) and mu_t (d values) as hi/lo floats
__global__ void __launch_bounds__(256) split_df_kernel(const double* __restrict__ Lf,
                                                       const double* __restrict__ mu, int64_t P,
                                                       int d, int T, float2* __restrict__ L2,
                                                       float2* __restrict__ mu2) {
  const int64_t n = (int64_t)T * P, m = (int64_t)T * d;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + m;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) L2[i] = split(Lf[i]);
    else mu2[i - n] = split(mu[i - n]);
  }
}

// rows j0 .. j0+31 of the packed factor: one contiguous range of this many values
__host__ __device__ inline int df_stage_len(int j0, int nb) { return nb * j0 + nb * (nb + 1) / 2; }
__host__ __device__ inline int df_stage_max(int d) {
  const int j0 = (d - 1) / kNB * kNB;
  return std::max(df_stage_len(j0, d - j0), d > kNB ? df_stage_len(j0 - kNB, kNB) : 0);
}

// H threads per pixel (rows jj = H u + h of each block), NPX pixels per tile.
// Shared memory: the tile's residuals [NPX][d | 1], then the rows of the
// current block of the factor (staged once per block for the whole tile).
template <typename InT, int H, int NPX>
__device__ __forceinline__ void solve_df_body(const InT* __restrict__ x, int ps, int W, int d,
                                              const float2* __restrict__ mu2,
                                              const float2* __restrict__ L,
                                              double* __restrict__ delta, int tile) {
  extern __shared__ __align__(16) float2 r2[];
  const int dp = d | 1;
  float2* Ls = r2 + NPX * dp;
  const int i0 = tile * NPX;
  for (int e = threadIdx.x; e < NPX * d; e += H * NPX) {
    const int p = e / d, k = e - p * d, i = i0 + p;
    r2[p * dp + k] = i < W ? df_sub(to_f(x[(int64_t)i * ps + k]), __ldg(mu2 + k))
                           : make_float2(0.f, 0.f);
  }
  const int p = threadIdx.x % NPX, h = threadIdx.x / NPX;
  const int i = i0 + p;
  float2* rr = r2 + p * dp;
  constexpr int R = kNB / H;   // rows of a block per thread
  for (int j0 = 0; j0 < d; j0 += kNB) {
    const int nb = min(kNB, d - j0);
    const int base = j0 * (j0 + 1) / 2;
    __syncthreads();          // the previous block is done with Ls (and r2 is staged)
    for (int e = threadIdx.x; e < df_stage_len(j0, nb); e += H * NPX) Ls[e] = __ldg(L + base + e);
    __syncthreads();
    // y_J in place of r_J: the thread's R rows at once (R independent chains),
    // each a compensated dot product
    {
      float sh[R], sc[R];
      const float2* Lj[R];
      bool act[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int jj = H * q + h, j = j0 + jj;
        act[q] = jj < nb;
        Lj[q] = Ls + (act[q] ? j * (j + 1) / 2 - base : 0);
        const float2 a = act[q] ? rr[j] : make_float2(0.f, 0.f);
        sh[q] = a.x, sc[q] = a.y;
      }
      // j0 is a multiple of 32
#pragma unroll 4
      for (int k = 0; k < j0; ++k) {
        const float2 m = rr[k];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const float2 l = Lj[q][k];
          dot2_fnma(sh[q], sc[q], l.x, l.y, m.x, m.y);
        }
      }
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (act[q]) rr[j0 + H * q + h] = df_norm(sh[q], sc[q]);
    }
    __syncthreads();
    // m_J = D_J y_J, rows H u + h, held until every thread has read y_J (a
    // rolled inner loop: the unrolled double-float steps overflow the
    // instruction cache)
    float2 mm[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int jj = H * u + h;
      float sh = 0.f, sc = 0.f;
      if (jj < nb) {
        const float2* Dj = Ls + (j0 + jj) * (j0 + jj + 1) / 2 - base + j0;
        const float2* yj = rr + j0;
#pragma unroll 1
        for (int kk = 0; kk <= jj; ++kk) {
          const float2 dv = Dj[kk], yv = yj[kk];
          dot2_fnma(sh, sc, -dv.x, -dv.y, yv.x, yv.y);
        }
      }
      mm[u] = df_norm(sh, sc);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < R; ++u)
      if (H * u + h < nb) rr[j0 + H * u + h] = mm[u];
  }
  __syncthreads();
  if (h == 0 && i < W) {
    float sh = 0.f, sc = 0.f;
    for (int j = 0; j < d; ++j) {
      const float2 m = rr[j];
      dot2_fnma(sh, sc, -m.x, -m.y, m.x, m.y);
    }
    delta[i] = sqrt((double)sh + (double)sc);
  }
}

// persistent grid: CTA c takes tiles c, c + grid, ... of the T x ntiles pairs
template <typename InT, int H, int NPX>
__global__ void __launch_bounds__(H * NPX) solve_df_kernel(
    const InT* __restrict__ X, int64_t line_stride, int ps, int W, int d,
    const float2* __restrict__ mu2, const float2* __restrict__ L2, double* __restrict__ delta,
    int T) {
  const int ntiles = (W + NPX - 1) / NPX;
  const int64_t total = (int64_t)T * ntiles;
  const int64_t P = packed_size(d);
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int t = (int)(w / ntiles), tile = (int)(w % ntiles);
    __syncthreads();
    solve_df_body<InT, H, NPX>(X + (int64_t)t * line_stride, ps, W, d, mu2 + (int64_t)t * d,
                               L2 + (int64_t)t * P, delta + (int64_t)t * W, tile);
  }
}

// four threads per pixel over 32-pixel tiles (128 threads): up to four CTAs and
// 16 warps per SM at d <= 128, enough independent double-float chains to keep
// the FP32 pipe issuing
constexpr int kHdf = 4, kNpx = 32;

size_t smem_df(int d, int npx) {
  return ((size_t)npx * (d | 1) + (size_t)df_stage_max(d)) * sizeof(float2);
}

template <typename InT, int H, int NPX>
void launch_df_t(const InT* x, int64_t line_stride, int ps, int W, int d, int T,
                 const float2* mu2, const float2* L2, double* delta, cudaStream_t st) {
  const int n_sm = device_shape().n_sm;
  const int threads = H * NPX;
  const size_t sm = smem_df(d, NPX);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_df_kernel<InT, H, NPX>, threads,
                                                sm);
  per_sm = std::max(1, per_sm);
  const int64_t total = (int64_t)T * ((W + NPX - 1) / NPX);
  const int grid = (int)std::min<int64_t>(total, (int64_t)n_sm * per_sm);
  solve_df_kernel<InT, H, NPX><<<grid, threads, sm, st>>>(x, line_stride, ps, W, d, mu2, L2,
                                                          delta, T);
}

}  // namespace

cudaError_t configure_solve_df_kernels() {
  cudaError_t e = cudaSuccess;
  const int m = (int)smem_df(kMaxDim, kNpx);
  e = cudaFuncSetAttribute(solve_df_kernel<uint16_t, kHdf, kNpx>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_df_kernel<float, kHdf, kNpx>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  return e;
}

void launch_solve_df(int in_type, const void* x, int64_t line_stride, int ps, int W, int d, int T,
                     const double* mu_t, const double* Lf, float2* mu2, float2* L2,
                     double* delta, cudaStream_t st) {
  const int64_t P = packed_size(d);
  const int64_t n = (int64_t)T * (P + d);
  const int gs = (int)std::min<int64_t>((n + 255) / 256, 4096);
  split_df_kernel<<<gs, 256, 0, st>>>(Lf, mu_t, P, d, T, L2, mu2);
  if (in_type == 0)
    launch_df_t<uint16_t, kHdf, kNpx>((const uint16_t*)x, line_stride, ps, W, d, T, mu2, L2,
                                      delta, st);
  else
    launch_df_t<float, kHdf, kNpx>((const float*)x, line_stride, ps, W, d, T, mu2, L2, delta, st);
}

}  // namespace erx

// S4 (Sec. III-D): L_t = chol(K_t + ridge I), FP64, one CTA per line.
//
// Output format ("blocked factor", packed lower, row j at j(j+1)/2): the
// entries of L_t, except that each 32 x 32 diagonal block L_JJ is replaced by
// its inverse D_J = L_JJ^{-1}.  The score kernels then solve L m = r block by
// block, m_J = D_J (r_J - sum_{K<J} L_JK m_K), which costs the same d(d+1)/2
// multiply-adds per pixel as a product with a full L^{-1} but needs only the
// d/32 small inverses (d * 32^2 / 6 DFMA) instead of the full d^3/6.
//
// The packed factor (d(d+1)/2 doubles, 197 KiB at d = 224) lives in shared
// memory; each pivot takes one reciprocal square root (l_jj = a_jj rsqrt(a_jj)).  Right-looking Cholesky: per column j the pivot is checked and
// square-rooted, the column scaled, and the trailing triangle updated
// A_ik -= l_ij l_kj with its elements spread evenly over all threads (the FP64
// pipe is 2 lanes/clk/SM on GB300, so idle lanes of a partial warp cost as
// much as busy ones).  Each diagonal block is then inverted by one warp, one
// column per lane, with the block in registers.  A pivot that is not positive
// and finite records the line in the error slot and poisons its scores (NaN).
#include <cmath>

#include "erx_batch.cuh"
#include "erx_internal.cuh"

namespace erx {
namespace {

constexpr int kThreads = 256;
constexpr int kNB = kFactorBlock;

__device__ __forceinline__ int pidx(int i, int k) { return i * (i + 1) / 2 + k; }

// Factor one line's K (packed, src) into the blocked factor (dst, dst32);
// `line` is the global line index reported on a bad pivot.
__device__ __forceinline__ void chol_body(const double* __restrict__ src, int d, double ridge,
                                          double* __restrict__ dst, float* __restrict__ d32,
                                          unsigned long long* __restrict__ err, int64_t line) {
  extern __shared__ __align__(16) double sm[];
  const int P = d * (d + 1) / 2;
  double* A = sm;
  double* col = sm + P;          // scaled column of the current step
  double* rdiag = col + d;       // 1 / l_jj
  __shared__ double s_inv;
  for (int q = threadIdx.x; q < P; q += kThreads) A[q] = src[q];
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += kThreads) A[pidx(j, j)] += ridge;
  __syncthreads();

  for (int j = 0; j < d; ++j) {
    if (threadIdx.x == 0) {
      double ajj = A[pidx(j, j)];
      if (!(ajj > 0.0) || !isfinite(ajj)) {
        atomicMin(&err[kErrNotPD], (unsigned long long)line);
        ajj = __longlong_as_double(0x7ff8000000000000ll);
      }
      const double ri = rsqrt(ajj);                   // 1 / l_jj
      A[pidx(j, j)] = ajj * ri;                       // l_jj
      s_inv = ri;
      rdiag[j] = ri;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = j + 1 + threadIdx.x; i < d; i += kThreads) {
      const double v = A[pidx(i, j)] * inv;
      A[pidx(i, j)] = v;
      col[i] = v;
    }
    __syncthreads();
    // trailing triangle rows/cols j+1 .. d-1: m(m+1)/2 elements, enumerated evenly
    const int m = d - 1 - j;
    const int n = m * (m + 1) / 2;
    for (int q = threadIdx.x; q < n; q += kThreads) {
      int r = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
      while (r * (r + 1) / 2 > q) --r;
      while ((r + 1) * (r + 2) / 2 <= q) ++r;
      const int c = q - r * (r + 1) / 2;
      const int i = j + 1 + r, k = j + 1 + c;
      const int p = pidx(i, k);
      A[p] = fma(-col[i], col[k], A[p]);
    }
    __syncthreads();
  }

  __syncthreads();
  // invert each 32 x 32 diagonal block in place, warp w taking blocks w, w + 8, ...:
  // columns right to left; with T = the already inverted trailing part of the
  // block, column j becomes -(1/l_jj) T l_col (lane i computes row i), so no
  // per-lane arrays are needed and the kernel keeps few registers.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (d + kNB - 1) / kNB;
  for (int bk = warp; bk < nblk; bk += kThreads / 32) {
    const int j0 = bk * kNB;
    const int nb = min(kNB, d - j0);
    for (int j = nb - 1; j >= 0; --j) {
      const double djj = rdiag[j0 + j];               // 1 / l_jj
      const int i = lane;
      double s = 0.0;
      if (i > j && i < nb) {
        const double* Ti = A + pidx(j0 + i, j0);
        for (int k = j + 1; k <= i; ++k) s = fma(Ti[k], A[pidx(j0 + k, j0 + j)], s);
      }
      __syncwarp();
      if (i > j && i < nb) A[pidx(j0 + i, j0 + j)] = -djj * s;
      if (i == j) A[pidx(j0 + j, j0 + j)] = djj;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < P; q += kThreads) dst[q] = A[q];
  if (d32) {
    for (int q = threadIdx.x; q < P; q += kThreads) d32[q] = (float)A[q];
  }
}

__global__ void __launch_bounds__(kThreads, 4) chol_kernel(const double* __restrict__ K_t, int d,
                                                       double ridge, double* __restrict__ Lf,
                                                       float* __restrict__ Lf32,
                                                       unsigned long long* __restrict__ err,
                                                       int64_t t0) {
  const int t = blockIdx.x;
  const int64_t P = packed_size(d);
  chol_body(K_t + t * P, d, ridge, Lf + t * P, Lf32 ? Lf32 + t * P : nullptr, err, t0 + t);
}

// Batched form: one CTA per stream.
__global__ void __launch_bounds__(kThreads, 4) b_chol_kernel(const BStream* __restrict__ S,
                                                         bool want32,
                                                         unsigned long long* __restrict__ err) {
  const BStream& s = S[blockIdx.x];
  chol_body(s.K_t, s.d, s.ridge, s.Lf, want32 ? s.Lf32 : nullptr, err, blockIdx.x);
}

// Full inverse X = L^{-1} in FP32 from the float blocked factor, for the FP32,
// TF32 and BF16 forms (their score kernels then apply X with one triangular
// product instead of a block-by-block solve).  One CTA per line, in place in
// shared memory and in the caller's buffer.  Column blocks left to right, row
// blocks top to bottom:  X_KK = D_K (already stored),
//   X_JK = -D_J (sum_{M=K}^{J-1} L_JM X_MK),   J > K,
// which reads only L entries of rows >= J and X entries of column block K
// above row block J, so X_JK can overwrite L_JK.  d^3/6 FP32 multiply-adds.
__device__ __forceinline__ void trinv32_body(float* __restrict__ Lf32, int d) {
  extern __shared__ __align__(16) float S[];
  __shared__ float Tm[kNB * kNB];
  const int P = d * (d + 1) / 2;
  for (int q = threadIdx.x; q < P; q += kThreads) S[q] = Lf32[q];
  __syncthreads();
  const int nblk = (d + kNB - 1) / kNB;
  for (int K = 0; K < nblk; ++K) {
    const int k0 = K * kNB, k1 = min(d, k0 + kNB);
    for (int J = K + 1; J < nblk; ++J) {
      const int j0 = J * kNB, j1 = min(d, j0 + kNB);
      // T = sum_M L_JM X_MK over columns m in [k0, j0)
      for (int e = threadIdx.x; e < kNB * kNB; e += kThreads) {
        const int jj = e / kNB, kk = e % kNB;
        const int j = j0 + jj, k = k0 + kk;
        float acc = 0.f;
        if (j < j1 && k < k1) {
          const float* Lj = S + pidx(j, 0);
          for (int m = k; m < j0; ++m) acc = fmaf(Lj[m], S[pidx(m, k)], acc);
        }
        Tm[e] = acc;
      }
      __syncthreads();
      // X_JK = -D_J T (D_J lower triangular, rows j, cols i <= j of block J)
      for (int e = threadIdx.x; e < kNB * kNB; e += kThreads) {
        const int jj = e / kNB, kk = e % kNB;
        const int j = j0 + jj, k = k0 + kk;
        if (j < j1 && k < k1) {
          const float* Dj = S + pidx(j, j0);
          float acc = 0.f;
          for (int ii = 0; ii <= jj; ++ii) acc = fmaf(Dj[ii], Tm[ii * kNB + kk], acc);
          S[pidx(j, k)] = -acc;
        }
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < P; q += kThreads) Lf32[q] = S[q];
}

__global__ void __launch_bounds__(kThreads) trinv32_kernel(float* __restrict__ Lf32, int d) {
  trinv32_body(Lf32 + (int64_t)blockIdx.x * packed_size(d), d);
}

__global__ void __launch_bounds__(kThreads) b_trinv32_kernel(const BStream* __restrict__ S) {
  const BStream& s = S[blockIdx.x];
  trinv32_body(s.Lf32, s.d);
}

}  // namespace

void launch_trinv32(float* Lf32, int d, int T, cudaStream_t st) {
  trinv32_kernel<<<T, kThreads, (size_t)packed_size(d) * sizeof(float), st>>>(Lf32, d);
}

void launch_batch_trinv32(const BStream* S, int n, int dmax, cudaStream_t st) {
  b_trinv32_kernel<<<n, kThreads, (size_t)packed_size(dmax) * sizeof(float), st>>>(S);
}

cudaError_t configure_factor_kernels() {
  const int m = (int)((packed_size(kMaxDim) + 2 * kMaxDim) * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(b_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  const int m32 = (int)(packed_size(kMaxDim) * sizeof(float));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(trinv32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, m32);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(b_trinv32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, m32);
  return e;
}

void launch_batch_chol(const BStream* S, int n, int dmax, bool want32, unsigned long long* err,
                       cudaStream_t st) {
  const size_t smem = (size_t)(packed_size(dmax) + 2 * dmax) * sizeof(double);
  b_chol_kernel<<<n, kThreads, smem, st>>>(S, want32, err);
}

void launch_chol_inv(const double* K_t, int d, int T, double ridge, double* Lf, float* Lf32,
                     unsigned long long* err, int64_t t0, cudaStream_t st) {
  const size_t smem = (size_t)(packed_size(d) + 2 * d) * sizeof(double);
  chol_kernel<<<T, kThreads, smem, st>>>(K_t, d, ridge, Lf, Lf32, err, t0);
}

}  // namespace erx

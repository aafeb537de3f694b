// S4 (Sec. III-D): L_t = chol(K_t + ridge I) and L_t^{-1}, FP64, one CTA per line.
//
// The packed lower triangle (d(d+1)/2 doubles, 197 KiB at d = 224) lives in
// shared memory for the whole factorisation:
//   Cholesky, right-looking: for each column j the pivot is checked and
//   square-rooted, the column below it scaled, and the trailing triangle
//   updated, A_ik -= l_ij l_kj (one warp per row, lanes along the row).
//   Inverse, in place, columns right to left: with T = inverse of the
//   trailing factor already stored, column j of L^{-1} is
//   -(1/l_jj) T l_col (a lower-triangular mat-vec, one warp per row).
// A pivot that is not positive and finite records the line in the error slot
// and poisons the line's scores with NaN.
#include <cmath>

#include "erx_internal.cuh"

namespace erx {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int pidx(int i, int k) { return i * (i + 1) / 2 + k; }

__global__ void __launch_bounds__(kThreads) chol_inv_kernel(const double* __restrict__ K_t, int d,
                                                           double ridge,
                                                           double* __restrict__ Linv,
                                                           float* __restrict__ Linv32,
                                                           unsigned long long* __restrict__ err,
                                                           int64_t t0) {
  extern __shared__ __align__(16) double sm[];
  const int P = d * (d + 1) / 2;
  double* A = sm;
  double* col = sm + P;
  __shared__ double s_inv;
  const int t = blockIdx.x;
  const double* src = K_t + (int64_t)t * P;
  for (int q = threadIdx.x; q < P; q += kThreads) A[q] = src[q];
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += kThreads) A[pidx(j, j)] += ridge;
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kThreads >> 5;
  // ---- Cholesky
  for (int j = 0; j < d; ++j) {
    if (threadIdx.x == 0) {
      double ajj = A[pidx(j, j)];
      if (!(ajj > 0.0) || !isfinite(ajj)) {
        atomicMin(&err[kErrNotPD], (unsigned long long)(t0 + t));
        ajj = __longlong_as_double(0x7ff8000000000000ll);
      }
      const double l = sqrt(ajj);
      A[pidx(j, j)] = l;
      s_inv = 1.0 / l;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = j + 1 + threadIdx.x; i < d; i += kThreads) {
      const double v = A[pidx(i, j)] * inv;
      A[pidx(i, j)] = v;
      col[i] = v;
    }
    __syncthreads();
    for (int i = j + 1 + warp; i < d; i += nw) {
      const double li = col[i];
      double* row = A + pidx(i, 0);
      for (int k = j + 1 + lane; k <= i; k += 32) row[k] = fma(-li, col[k], row[k]);
    }
    __syncthreads();
  }
  // ---- inverse of the lower factor, in place
  for (int j = d - 1; j >= 0; --j) {
    if (threadIdx.x == 0) A[pidx(j, j)] = 1.0 / A[pidx(j, j)];
    for (int i = j + 1 + threadIdx.x; i < d; i += kThreads) col[i] = A[pidx(i, j)];
    __syncthreads();
    const double djj = A[pidx(j, j)];
    for (int i = j + 1 + warp; i < d; i += nw) {
      const double* row = A + pidx(i, 0);
      double s = 0.0;
      for (int k = j + 1 + lane; k <= i; k += 32) s = fma(row[k], col[k], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) A[pidx(i, j)] = -djj * s;
    }
    __syncthreads();
  }
  double* dst = Linv + (int64_t)t * P;
  for (int q = threadIdx.x; q < P; q += kThreads) dst[q] = A[q];
  if (Linv32) {
    float* d32 = Linv32 + (int64_t)t * P;
    for (int q = threadIdx.x; q < P; q += kThreads) d32[q] = (float)A[q];
  }
}

}  // namespace

cudaError_t configure_factor_kernels() {
  return cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)((packed_size(kMaxDim) + kMaxDim) * sizeof(double)));
}

void launch_chol_inv(const double* K_t, int d, int T, double ridge, double* Linv, float* Linv32,
                     unsigned long long* err, int64_t t0, cudaStream_t st) {
  const size_t smem = (size_t)(packed_size(d) + d) * sizeof(double);
  chol_inv_kernel<<<T, kThreads, smem, st>>>(K_t, d, ridge, Linv, Linv32, err, t0);
}

}  // namespace erx

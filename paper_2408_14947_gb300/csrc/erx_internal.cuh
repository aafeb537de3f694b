// Internal declarations shared by the ERX CUDA translation units.
//
// Device data layout of one block of T lines (all row-major):
//   lines      caller's [T][p][b] samples (u16 / f32 / f64), line stride given
//   Z          [T][p][d] projected pixels when SRP is on (double or float)
//   S1i, S2i   exact integer sums  sum_i x_i  [T][d]  and  sum_i x_i x_i^T  [T][d][d]
//   mu_hat     [T][d] line means (double);  shift [T][d] centring shift c
//   S2f        [T][d][d] sums  sum_i (z_i - c)(z_i - c)^T  (double)
//   mu_t, K_t  [T][d], [T][P] statistics each line is scored with (P = d(d+1)/2,
//              packed lower triangle, row j starts at j(j+1)/2)
//   Linv       [T][P] blocked factor: packed lower L_t with each 32 x 32 diagonal
//              block replaced by its inverse (double); Linv32 its float copy
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace erx {

constexpr int kMaxDim = 224;   // packed FP64 factor must fit one SM's shared memory
constexpr int kFactorBlock = 32;  // diagonal blocks of the factor are stored inverted
// The floating centred scatter of a line is summed per
// chunk of kScatterChunk pixels; the chunk sums are then added in FP64 in
// chunk order.  A single-stream launch adds them as it goes; the batched form
// gives each chunk its own CTA and adds the chunk sums in the EMA kernel, in the
// same order, so both give the same bits.
constexpr int kScatterChunk = 256;
__host__ __device__ inline int scatter_chunks(int W) {
  return (W + kScatterChunk - 1) / kScatterChunk;
}

// error slots (unsigned long long, min-reduced line index; ~0ull = none)
enum { kErrNotPD = 0, kErrRange = 1, kErrTimeout = 2, kErrSlots = 3 };

__host__ __device__ inline int64_t packed_size(int d) { return (int64_t)d * (d + 1) / 2; }

// S3 arithmetic shared by every EMA kernel, with the rounding of each
// operation fixed (no contraction into FMAs), so that all kernels that update
// the state produce the same bits.
#ifdef __CUDACC__
// K_hat_ab from the scatter S_ab about shift c: (S_ab - p e_a e_b) / (p - 1), e = mu_hat - c
// rw1 = 1 / (W - 1), correctly rounded (W - 1 is exact)
__device__ __forceinline__ double ema_khat(double S, double ea, double eb, double Wd, double rw1) {
  return __dmul_rn(__dsub_rn(S, __dmul_rn(__dmul_rn(Wd, ea), eb)), rw1);
}
// (1 - a) s + a x, both products rounded before the sum (as written in Sec. III-C)
__device__ __forceinline__ double ema_mix(double s, double x, double alpha, double beta) {
  return __dadd_rn(__dmul_rn(beta, s), __dmul_rn(alpha, x));
}

// S4's diagonal blocks D_J = L_JJ^{-1}, shared by every factor kernel so that
// all of them give the same bits.  The nb x nb block at (j0, j0) of the packed
// lower matrix A (row i at i(i+1)/2) is inverted in place, lane i of each warp
// taking row i; ri[k] = 1 / l_kk.  From X L = I: X_kk = ri_k and, for i > j,
//   X_ij = -ri_j * sum_{k = j+1 .. i} X_ik l_kj,
// the sum taken from k = i down to k = j + 1.  Columns are finished right to
// left.  When column k is final, every row i > k adds its term X_ik l_kj to
// its partial sums S_ij (j < k), kept in place of l_ij (row i of L is read only
// while column i is finished, which is earlier), and row k then starts its own
// sums with the first term ri_k l_kj, one lane per j.  From one column to the
// next the chain is a multiplication and one multiply-add (not a whole sum as
// in a column-by-column evaluation), with the same d^3/6 multiply-adds.
//
// NW warps share a block (warp w of the group: w = 0 .. NW-1): warp w adds the
// terms of the columns j = k-1-w, k-1-w-NW, ... (each warp's multiply-adds run
// on its own SM sub-partition's FP64 unit); with NW > 1 warp 0 finishes X_ik
// into shared memory for all (one multiplication instead of one per warp) and
// warp 1 starts row k's sums.  Every S_ij still receives one multiply-add per
// step, in the same order, whatever NW.  NW > 1 synchronises the group with
// named barrier `bar` (NW * 32 threads).
template <int NW>
__device__ __forceinline__ void invert_diag_block(double* __restrict__ A, int j0, int nb,
                                                  const double* __restrict__ ri, int w, int lane,
                                                  int bar = 1) {
  auto row = [&](int i) { return A + (j0 + i) * (j0 + i + 1) / 2 + j0; };
  auto sync = [&]() {
    if constexpr (NW == 1)
      __syncwarp();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NW * 32) : "memory");
  };
  double* Si = row(lane);            // dereferenced for lane < nb only
  for (int k = nb - 1; k >= 0; --k) {
    const double rk = ri[k];
    const double* Lk = row(k);
    double x = 0.0;
    if constexpr (NW == 1) {
      if (lane > k && lane < nb) {
        x = -rk * Si[k];             // X_ik: S_ik has all its terms
        Si[k] = x;
      }
    } else {
      if (w == 0 && lane > k && lane < nb) Si[k] = -rk * Si[k];
      sync();
      if (lane > k && lane < nb) x = Si[k];
    }
    if (lane > k && lane < nb) {
      // this warp's columns, four at a time (loads, multiply-adds, stores) so
      // that the multiply-adds do not wait on each other's stores
      int j = k - 1 - w;
      for (; j >= 3 * NW; j -= 4 * NW) {
        double l[4], s[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) l[u] = Lk[j - u * NW], s[u] = Si[j - u * NW];
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = fma(x, l[u], s[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) Si[j - u * NW] = s[u];
      }
      for (; j >= 0; j -= NW) Si[j] = fma(x, Lk[j], Si[j]);
    }
    sync();
    // row k starts its sums (row k of L is no longer read)
    if (w == (NW > 1 ? 1 : 0) && lane < k) row(k)[lane] = fma(rk, row(k)[lane], 0.0);
    sync();
  }
  if (w == 0 && lane < nb) Si[lane] = ri[lane];
  sync();
}
#endif

// Opt the kernels that need it into large dynamic shared memory on the
// current device (called once per device at context creation).
cudaError_t configure_factor_kernels();
cudaError_t configure_solve_kernels();

// ---- launchers (all asynchronous on `st`) -------------------------------

// Exact integer sums for u16 input without projection.  maxv = 2^bits - 1.
void launch_stats_int(const uint16_t* x, int64_t line_stride, int W, int d, uint32_t maxv,
                      int T, uint64_t* S1, uint64_t* S2, unsigned long long* err, int64_t t0,
                      cudaStream_t st);

// Exact integer sums on the tensor cores (bf16 6-bit split, FP32 accumulation
// exact below 2^24): u16 samples < 2^12, no projection, d + 1 <= 128, p <= 2048.
bool stats_tc_supported(int d, int W, int bits);
cudaError_t configure_stats_tc_kernel();
void launch_stats_tc(const uint16_t* x, int64_t line_stride, int W, int d, uint32_t maxv, int T,
                     int n_sm, uint64_t* S1, uint64_t* S2, unsigned long long* err, int64_t t0,
                     cudaStream_t st);

// Line means (double) and centring shifts c (= mean, or the mean rounded to
// float when `float_shift`).  in_type: 0 u16, 1 f32, 2 f64.  ps = pixel stride.
void launch_mean(int in_type, const void* x, int64_t line_stride, int ps, int W, int d, int T,
                 bool float_shift, double* mu_hat, double* shift, cudaStream_t st);

// Centred scatter sums about `shift`, accumulated in double (fp64=true) or float.
void launch_stats_fp(int in_type, bool fp64, const void* x, int64_t line_stride, int ps, int W,
                     int d, int T, const double* shift, double* S2f, cudaStream_t st);

// EMA scan over the T lines of a block: turns line statistics into the
// statistics each line is scored with and advances the state.  `scratch`
// holds ema_scratch_doubles(d, T) doubles (NULL: sequential scan).
size_t ema_scratch_doubles(int d, int T);
// SM count and shared memory per SM of the current device, queried once
// (thread-safe initialisation; one device per process)
struct DeviceShape {
  int n_sm;
  int smem_per_sm;
};
const DeviceShape& device_shape();

// maxv: the largest sample of integer statistics (it bounds their sums)
void launch_ema_scan(bool int_stats, const uint64_t* S1i, const uint64_t* S2i,
                     const double* mu_hat, const double* shift, const double* S2f, int T, int d,
                     int W, double alpha, int64_t t0, int order, double* mu_state,
                     double* K_state, double* mu_t, double* K_t, double* scratch,
                     cudaStream_t st, uint32_t maxv = 0xffffu);

// IMC (equal-weight ablation, batch Welford) in place of the EMA scan: same
// outputs; `work` holds imc_work_doubles(d, T) doubles.
size_t imc_work_doubles(int d, int T);
void launch_imc_scan(bool int_stats, const uint64_t* S1i, const uint64_t* S2i,
                     const double* mu_hat, const double* shift, const double* S2f, int T, int d,
                     int W, int64_t t0, int order, double* mu_state, double* K_state,
                     double* mu_t, double* K_t, double* work, double* scratch,
                     cudaStream_t st, uint32_t maxv = 0xffffu);

// Cholesky of K_t + ridge I, diagonal blocks inverted, one CTA per line.
// invert: replace the 32 x 32 diagonal blocks by their inverses in FP64 (the
// FP64 score kernels and the encoder's loss need them; the FP32 routes invert
// them in trinv32 instead)
void launch_chol_inv(const double* K_t, int d, int T, double ridge, double* Linv, float* Linv32,
                     unsigned long long* err, int64_t t0, cudaStream_t st, bool invert = true,
                     bool leave_room = false);
// The same factor for a few lines, each over a cluster of chol_cluster_ctas()
// CTAs on as many SMs (k_factor_cluster.cu); bit-equal to launch_chol_inv's
// one-CTA kernels.  configure_cluster_factor returns the clusters that fit on
// the device at once (0: the cluster form is not used).
int chol_cluster_ctas();
int configure_cluster_factor(int smem_per_sm);
void launch_chol_cluster(const double* K_t, int d, int T, double ridge, double* Lf, float* Lf32,
                         unsigned long long* err, int64_t t0, bool invert, int smem_per_sm,
                         cudaStream_t st);

// In place: the float blocked factor of T lines becomes the full L^{-1} (FP32).
void launch_trinv32(float* Lf32, int d, int T, cudaStream_t st);

// delta_i = || m_i ||, L m_i = z_i - mu_t solved block by block, FP64 arithmetic.
void launch_solve_fp64(int in_type, const void* x, int64_t line_stride, int ps, int W, int d,
                       int T, const double* mu_t, const double* Linv, double* delta,
                       cudaStream_t st);

// delta_i with FP32 arithmetic (register-tiled SIMT).
void launch_solve_fp32(int in_type, const void* x, int64_t line_stride, int ps, int W, int d,
                       int T, const double* mu_t, const float* Linv32, float* delta,
                       cudaStream_t st);

// delta_i on the tensor cores: fmt 2 = TF32, 1 = BF16 operands, FP32 accumulation.
cudaError_t configure_solve_tc_kernels();
// S5 in double-float (FP64E form): splits the blocked factor and mu_t into
// hi/lo floats (L2: T x P, mu2: T x d), then scores; in_type 0 (u16) or 1 (f32)
cudaError_t configure_solve_df_kernels();
void launch_solve_df(int in_type, const void* x, int64_t line_stride, int ps, int W, int d, int T,
                     const double* mu_t, const double* Lf, float2* mu2, float2* L2,
                     double* delta, cudaStream_t st);
// S2 centred scatter of float lines on the tensor cores (fmt 1 BF16, 2 TF32)
bool syrk_tc_supported(const void* x, int64_t line_stride, int ps, int W, int d);
cudaError_t configure_syrk_tc_kernels();
void launch_syrk_tc(int fmt, const float* x, int64_t line_stride, int W, int d, int T, int n_sm,
                    const double* shift, double* S2f, unsigned long long* err, int64_t t0,
                    cudaStream_t st);
void launch_solve_tc(int fmt, int in_type, const void* x, int64_t line_stride, int ps, int W,
                     int d, int T, const double* mu_t, const float* Lf32, float* delta,
                     unsigned long long* err, int64_t t0, cudaStream_t st);

// Per-line normalisation (Sec. III-E), mask and warm-up flags.
void launch_normalise(bool fp64, const void* delta, int W, int T, double threshold,
                      int64_t t0, int64_t warmup, void* delta_n, uint8_t* mask,
                      uint8_t* detecting, cudaStream_t st);

// Sparse projection Z = X W (column lists), output double or float.
void launch_project(int in_type, const void* x, int64_t line_stride, int B, int W, int d, int T,
                    const int* colptr, const int* rows, const double* vals, bool out_fp64,
                    void* z, cudaStream_t st);

}  // namespace erx
struct erx_encoder;
namespace erx {
int encoder_k(const ::erx_encoder* e);
int encoder_bands(const ::erx_encoder* e);
void encoder_forward_on(::erx_encoder* e, const float* x, int64_t n, float* codes,
                        cudaStream_t st);
}  // namespace erx

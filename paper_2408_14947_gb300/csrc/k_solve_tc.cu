// S5 (Sec. III-D) on the tensor cores: BF16, TF32 or 3xTF32 operands, FP32
// accumulation.
//
// With the full inverse X = L_t^{-1} (FP32, made from the blocked factor by
// trinv32), the scores of a 128-pixel tile are one lower-triangular product
//   M = R X^T  (R: 128 x d centred pixels),  delta_i = |M_i|.
// The contraction runs K-outer in 32-column chunks: chunk k0 .. k0+31 of R
// meets rows j >= k0 of X (X is zero above its diagonal), so one MMA of
// N = dK - k0 per K step accumulates into TMEM columns k0 .. dK-1 (pixel p is
// TMEM lane p).  Two stage buffers: while the MMAs of chunk c run, the threads
// stage chunk c+1 (R from registers loaded one chunk ahead, X from L2 with all
// of a thread's loads issued before the stage's wait), and one thread issues
// the MMAs and commits them to the stage's mbarrier.  Operand
// tiles are K-major, no swizzle.  r is formed as (x - mu_hi) - mu_lo with mu
// split into two floats; TF32 operands are rounded to nearest (cvt.rna).
// 3xTF32 (FMT 3) splits each operand v as hi = tf32(v), lo = tf32(v - hi) and
// accumulates Hi Hi' + Hi Lo' + Lo Hi'.
#include <cuda_bf16.h>

#include "erx_batch.cuh"
#include "erx_internal.cuh"
#include "tc_util.cuh"

namespace erx {
namespace {

constexpr int kPix = 128;
constexpr int kB = kFactorBlock;     // 32 columns per K chunk
constexpr uint32_t kLBO = 128;
constexpr uint32_t kWaitLimit = 1u << 26;

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

__device__ __forceinline__ uint32_t tf32_bits(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// 16 bytes of operand data (4 tf32 or 8 bf16 values) from consecutive floats;
// for FMT 3 also the 16 bytes of the low parts
template <int FMT>
__device__ __forceinline__ void pack16(const float* v, uint4& hi, uint4& lo) {
  if constexpr (FMT == 1) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&b);
    }
    hi = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
    uint32_t h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = tf32_bits(v[i]);
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    if constexpr (FMT == 3) {
      uint32_t l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) l[i] = tf32_bits(v[i] - __uint_as_float(h[i]));
      lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
}

__host__ __device__ inline int tc_dk(int d) { return (d + kB - 1) / kB * kB; }
constexpr int kTcDKMax = (kMaxDim + kB - 1) / kB * kB;   // 224
// TMEM columns: the smallest power of two >= dK (at least 32)
__host__ __device__ inline uint32_t tc_cols(int d) {
  const int dk = tc_dk(d);
  return dk <= 32 ? 32u : dk <= 64 ? 64u : dk <= 128 ? 128u : 256u;
}

// bytes of one stage: R chunk (128 x 32) and X chunk (dK x 32), hi (and lo)
__host__ __device__ inline int tc_stage_bytes(int d, int fmt) {
  const int E = fmt == 1 ? 2 : 4, NT = fmt == 3 ? 2 : 1;
  return NT * (kPix + tc_dk(d)) * kB * E;
}

// the 32 values x[k0 .. k0+31] of one pixel (0 beyond d or for an invalid pixel)
template <typename InT, bool VEC>
__device__ __forceinline__ void load_chunk(const InT* __restrict__ xp, bool valid, int k0, int d,
                                           float (&v)[kB]) {
  if constexpr (VEC && sizeof(InT) == 4) {
    // float lines, 16-byte aligned pixel rows, d a multiple of 4
#pragma unroll
    for (int u = 0; u < kB / 4; ++u) {
      const int k = k0 + 4 * u;
      float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid && k < d) f = __ldg(reinterpret_cast<const float4*>(xp + k));
      v[4 * u] = f.x, v[4 * u + 1] = f.y, v[4 * u + 2] = f.z, v[4 * u + 3] = f.w;
    }
  } else if constexpr (VEC) {
    // u16 lines, 8-byte aligned pixel rows, d a multiple of 4: four samples per load
#pragma unroll
    for (int u = 0; u < kB / 4; ++u) {
      const int k = k0 + 4 * u;
      uint2 w = make_uint2(0u, 0u);
      if (valid && k < d) w = __ldg(reinterpret_cast<const uint2*>(xp + k));
      v[4 * u] = (float)(w.x & 0xffffu), v[4 * u + 1] = (float)(w.x >> 16);
      v[4 * u + 2] = (float)(w.y & 0xffffu), v[4 * u + 3] = (float)(w.y >> 16);
    }
  } else {
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int k = k0 + u;
      v[u] = (valid && k < d) ? to_f(xp[k]) : 0.f;
    }
  }
}

// Pixels tile*128 .. +127 of one line (x, pixel stride ps) with mu (d) and the
// FP32 inverse factor Xg (packed lower); delta: the line's W scores; `line` is
// reported on a timeout.  FMT 1: BF16, 2: TF32, 3: 3xTF32.  DKM: the largest
// dK the instance takes (128 or 224); it sizes the registers that hold a
// thread's share of an X chunk, so that d <= 128 keeps four CTAs per SM.
template <typename InT, int FMT, bool VEC, int DKM>
__device__ __forceinline__ void solve_tc_body(const InT* __restrict__ x, int ps, int W, int d,
                                              const double* __restrict__ mu,
                                              const float* __restrict__ Xg,
                                              float* __restrict__ delta,
                                              unsigned long long* __restrict__ err, int64_t line,
                                              int tile) {
  constexpr int E = FMT == 1 ? 2 : 4;     // bytes per element
  constexpr int CK = 16 / E;              // elements per 16-byte core row
  constexpr int KS = 32 / E;              // K per MMA
  constexpr int NT = FMT == 3 ? 2 : 1;
  constexpr uint32_t SBO = (kB / CK) * 128u;
  constexpr int FK = FMT == 1 ? 1 : 2;
  // 16-byte groups of an X chunk per thread at the largest dK
  constexpr int kXIt = (DKM * (kB / CK) + kPix - 1) / kPix;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ float mu_hi[kMaxDim], mu_lo[kMaxDim];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int i0 = tile * kPix;
  const int dK = tc_dk(d);
  const int nK = dK / kB;
  const uint32_t ncols = tc_cols(d);
  const int r_bytes = kPix * kB * E, x_bytes = dK * kB * E;
  const int stage = tc_stage_bytes(d, FMT);
  auto off = [](int row, int k) -> uint32_t {
    return (uint32_t)(row >> 3) * SBO + (uint32_t)(k / CK) * kLBO + (uint32_t)(row & 7) * 16u;
  };
  for (int k = tid; k < d; k += kPix) {
    const double m = mu[k];
    const float h = (float)m;
    mu_hi[k] = h;
    mu_lo[k] = (float)(m - (double)h);
  }
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  const int p = tid, i = i0 + p;
  const bool valid = i < W;
  const InT* xp = x + (int64_t)(valid ? i : 0) * ps;
  float cur[kB];
  load_chunk<InT, VEC>(xp, valid, 0, d, cur);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  bool ok = true;
  for (int kc = 0; kc < nK; ++kc) {
    const int b = kc & 1, k0 = kc * kB;
    unsigned char* Rh = sm + b * stage;
    unsigned char* Rl = Rh + r_bytes;                   // FMT 3 only
    unsigned char* Xh = Rh + NT * r_bytes;
    unsigned char* Xl = Xh + x_bytes;                   // FMT 3 only
    float nxt[kB];
    if (kc + 1 < nK) load_chunk<InT, VEC>(xp, valid, k0 + kB, d, nxt);
    // rows j = k0 .. dK-1 of X, columns k0 .. k0+31 (zero above the diagonal and
    // beyond d): all of this thread's loads from L2 are issued here, before the
    // stage's wait, and packed after it
    const int nrows = dK - k0;
    const int ne = nrows * (kB / CK);
    float xv[kXIt][CK];
#pragma unroll
    for (int it = 0; it < kXIt; ++it) {
      const int e = tid + it * kPix;
      const int j = k0 + e / (kB / CK), kb = k0 + (e % (kB / CK)) * CK;
      const float* Xj = Xg + (int64_t)j * (j + 1) / 2;
#pragma unroll
      for (int u = 0; u < CK; ++u)
        xv[it][u] = (e < ne && j < d && kb + u <= j) ? __ldg(Xj + kb + u) : 0.f;
    }
    if (kc >= 2) {
      const bool w_ok = tc::mbar_wait(&mbar[b], (uint32_t)((kc - 2) >> 1) & 1u, kWaitLimit);
      if (__syncthreads_or(!w_ok)) {
        ok = false;
        break;
      }
    }
    // this pixel's row of the R chunk
#pragma unroll
    for (int g = 0; g < kB / CK; ++g) {
      float v[CK];
#pragma unroll
      for (int u = 0; u < CK; ++u) {
        const int k = k0 + g * CK + u;
        v[u] = (valid && k < d) ? (cur[g * CK + u] - mu_hi[k]) - mu_lo[k] : 0.f;
      }
      uint4 hi, lo;
      pack16<FMT>(v, hi, lo);
      *reinterpret_cast<uint4*>(Rh + off(p, g * CK)) = hi;
      if constexpr (FMT == 3) *reinterpret_cast<uint4*>(Rl + off(p, g * CK)) = lo;
    }
    // the X chunk
#pragma unroll
    for (int it = 0; it < kXIt; ++it) {
      const int e = tid + it * kPix;
      if (e < ne) {
        const int jj = e / (kB / CK), kg = e % (kB / CK);
        uint4 hi, lo;
        pack16<FMT>(xv[it], hi, lo);
        *reinterpret_cast<uint4*>(Xh + off(jj, kg * CK)) = hi;
        if constexpr (FMT == 3) *reinterpret_cast<uint4*>(Xl + off(jj, kg * CK)) = lo;
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t id = tc::idesc(FK, kPix, nrows);
      const uint32_t aRh = tc::smem_u32(Rh), aXh = tc::smem_u32(Xh);
#pragma unroll
      for (int s = 0; s < kB / KS; ++s) {
        const uint32_t ko = (uint32_t)s * 2u * kLBO;
        const uint64_t da = tc::desc(aRh + ko, kLBO, SBO);
        const uint64_t db = tc::desc(aXh + ko, kLBO, SBO);
        const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
        if constexpr (FMT == 1) {
          tc::mma_bf16(tmem + (uint32_t)k0, da, db, id, acc);
        } else {
          tc::mma_tf32(tmem + (uint32_t)k0, da, db, id, acc);
          if constexpr (FMT == 3) {
            const uint64_t dal = tc::desc(tc::smem_u32(Rl) + ko, kLBO, SBO);
            const uint64_t dbl = tc::desc(tc::smem_u32(Xl) + ko, kLBO, SBO);
            tc::mma_tf32(tmem + (uint32_t)k0, da, dbl, id, 1u);
            tc::mma_tf32(tmem + (uint32_t)k0, dal, db, id, 1u);
          }
        }
      }
      tc::commit(&mbar[b]);
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) cur[u] = nxt[u];
  }
  // wait for the last commit of each buffer
  uint32_t pending_parity[2] = {0u, 0u};
  bool pending[2] = {false, false};
  for (int J = nK - 1; J >= 0 && J >= nK - 2; --J) {
    pending[J & 1] = true;
    pending_parity[J & 1] = (uint32_t)(J >> 1) & 1u;
  }
  if (ok) {
    bool w_ok = true;
    for (int b = 0; b < 2; ++b)
      if (pending[b]) w_ok &= tc::mbar_wait(&mbar[b], pending_parity[b], kWaitLimit);
    ok = !__syncthreads_or(!w_ok);
  }
  float d2 = 0.f;
  if (ok) {
    tc::fence_after_sync();
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    for (int c0 = 0; c0 < dK; c0 += 16) {
      uint32_t v[16];
      tc::tmem_ld16(lane_base + (uint32_t)c0, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < d) {
          const float m = __uint_as_float(v[j]);
          d2 = fmaf(m, m, d2);
        }
    }
  } else {
    // one more bounded wait for the MMAs still in flight before TMEM is released
    for (int b = 0; b < 2; ++b)
      if (pending[b]) tc::mbar_wait(&mbar[b], pending_parity[b], kWaitLimit);
    if (tid == 0) atomicMin(&err[kErrTimeout], (unsigned long long)line);
  }
  if (valid) delta[i] = ok ? sqrtf(d2) : __int_as_float(0x7fc00000);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, ncols);
}

template <typename InT, int FMT, bool VEC, int DKM>
__global__ void __launch_bounds__(kPix, DKM <= 128 ? 4 : 1) solve_tc_kernel(
    const InT* __restrict__ X, int64_t line_stride, int ps, int W, int d,
    const double* __restrict__ mu_t, const float* __restrict__ Lf32, float* __restrict__ delta,
    unsigned long long* __restrict__ err, int64_t t0) {
  const int t = blockIdx.y;
  solve_tc_body<InT, FMT, VEC, DKM>(X + (int64_t)t * line_stride, ps, W, d, mu_t + (int64_t)t * d,
                               Lf32 + (int64_t)t * packed_size(d), delta + (int64_t)t * W, err,
                               t0 + t, blockIdx.x);
}

// Batched form: one CTA per (stream, 128-pixel tile) item.
template <int FMT, int DKM>
__global__ void __launch_bounds__(kPix, DKM <= 128 ? 4 : 1) b_solve_tc_kernel(
    const BStream* __restrict__ S, const BItem* __restrict__ items,
    unsigned long long* __restrict__ err) {
  const BItem it = items[blockIdx.x];
  const BStream& s = S[it.s];
  if (((uintptr_t)s.x % 16) == 0 && (s.d % 4) == 0)
    solve_tc_body<float, FMT, true, DKM>(s.x, s.d, s.W, s.d, s.mu_t, s.Lf32, (float*)s.delta,
                                         err, it.s, it.tile);
  else
    solve_tc_body<float, FMT, false, DKM>(s.x, s.d, s.W, s.d, s.mu_t, s.Lf32, (float*)s.delta,
                                          err, it.s, it.tile);
}

// Dynamic shared memory of one CTA: two stages, raised where needed so that no
// more CTAs share an SM than its 512 TMEM columns hold (no CTA then waits in
// tcgen05.alloc for another's columns).
size_t launch_smem(int d, int fmt) {
  const size_t need = 2 * (size_t)tc_stage_bytes(d, fmt);
  const int maxc = 512 / (int)tc_cols(d);
  const size_t pad = (size_t)device_shape().smem_per_sm / (size_t)(maxc + 1) + 1;
  return need > pad ? need : pad;
}

}  // namespace

cudaError_t configure_solve_tc_kernels() {
  cudaError_t e = cudaSuccess;
  // the TMEM padding of launch_smem needs the SM's shared memory size
  if (device_shape().smem_per_sm <= 0) return cudaErrorInvalidDevice;
  // the largest request of any d <= kMaxDim
  auto most = [](int fmt) {
    size_t m = 0;
    for (int d = 1; d <= kMaxDim; d += 31) m = m > launch_smem(d, fmt) ? m : launch_smem(d, fmt);
    const size_t top = launch_smem(kMaxDim, fmt);
    return (int)(m > top ? m : top);
  };
  const int m1 = most(1), m2 = most(2), m3 = most(3);
#define ERX_CFG(K, M) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, M)
#define ERX_CFG_T(IT, V, K)                            \
  ERX_CFG((solve_tc_kernel<IT, 1, V, K>), m1);         \
  ERX_CFG((solve_tc_kernel<IT, 2, V, K>), m2);         \
  ERX_CFG((solve_tc_kernel<IT, 3, V, K>), m3);
#define ERX_CFG_K(K)                                   \
  ERX_CFG_T(uint16_t, false, K)                        \
  ERX_CFG_T(float, false, K)                           \
  ERX_CFG_T(double, false, K)                          \
  ERX_CFG_T(uint16_t, true, K)                         \
  ERX_CFG_T(float, true, K)                            \
  ERX_CFG((b_solve_tc_kernel<1, K>), m1);              \
  ERX_CFG((b_solve_tc_kernel<2, K>), m2);              \
  ERX_CFG((b_solve_tc_kernel<3, K>), m3);
  ERX_CFG_K(128)
  ERX_CFG_K(kTcDKMax)
#undef ERX_CFG_K
#undef ERX_CFG_T
#undef ERX_CFG
  return e;
}

void launch_batch_solve_tc(int fmt, const BStream* S, const BItem* items, int n_items, int dmax,
                           unsigned long long* err, cudaStream_t st) {
  const size_t sm = launch_smem(dmax, fmt);
#define ERX_B(F, K) b_solve_tc_kernel<F, K><<<n_items, kPix, sm, st>>>(S, items, err)
#define ERX_BK(K)                 \
  if (fmt == 1) ERX_B(1, K);      \
  else if (fmt == 2) ERX_B(2, K); \
  else ERX_B(3, K);
  if (tc_dk(dmax) <= 128) {
    ERX_BK(128)
  } else {
    ERX_BK(kTcDKMax)
  }
#undef ERX_BK
#undef ERX_B
}

void launch_solve_tc(int fmt, int in_type, const void* x, int64_t line_stride, int ps, int W,
                     int d, int T, const double* mu_t, const float* Lf32, float* delta,
                     unsigned long long* err, int64_t t0, cudaStream_t st) {
  dim3 grid((W + kPix - 1) / kPix, T);
  const size_t sm = launch_smem(d, fmt);
  // vector loads: float lines whose pixel rows start on 16 bytes, u16 lines
  // whose pixel rows start on 8 bytes (four samples per load either way)
  const bool vec = in_type == 1 && ((uintptr_t)x % 16) == 0 && (ps % 4) == 0 &&
                   (line_stride % 4) == 0 && (d % 4) == 0;
  const bool vec16 = in_type == 0 && ((uintptr_t)x % 8) == 0 && (ps % 4) == 0 &&
                     (line_stride % 4) == 0 && (d % 4) == 0;
#define ERX_L(IT, F, V, K)                                                             \
  solve_tc_kernel<IT, F, V, K><<<grid, kPix, sm, st>>>((const IT*)x, line_stride, ps, W, d, \
                                                       mu_t, Lf32, delta, err, t0)
#define ERX_LF(F, K)                                   \
  if (vec16) ERX_L(uint16_t, F, true, K);              \
  else if (in_type == 0) ERX_L(uint16_t, F, false, K); \
  else if (vec) ERX_L(float, F, true, K);              \
  else if (in_type == 1) ERX_L(float, F, false, K);    \
  else ERX_L(double, F, false, K);
#define ERX_LK(K)           \
  if (fmt == 1) {           \
    ERX_LF(1, K)            \
  } else if (fmt == 2) {    \
    ERX_LF(2, K)            \
  } else {                  \
    ERX_LF(3, K)            \
  }
  if (tc_dk(d) <= 128) {
    ERX_LK(128)
  } else {
    ERX_LK(kTcDKMax)
  }
#undef ERX_LK
#undef ERX_LF
#undef ERX_L
}

}  // namespace erx

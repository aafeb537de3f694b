// S5 (Sec. III-D) on the tensor cores: TF32 or BF16 operands, FP32 accumulation.
//
// With the full inverse X = L_t^{-1} (FP32, made from the blocked factor by
// trinv32), the scores of a 128-pixel tile are one lower-triangular product
//   M = R X^T  (R: 128 x d centred pixels),  delta_i = |M_i|,
// computed as independent 128 x 32 output blocks: block J needs K = j0 + 32
// (X is zero above its diagonal).  The pixels' rows of R stay in shared memory
// for the whole tile; the 32 rows of X of block J are staged into one of two
// buffers while the MMAs of block J-1 run (one thread issues them and commits
// them to the buffer's mbarrier), and all blocks accumulate into their own TMEM
// columns, drained once at the end (pixel p is TMEM lane p).  Operand tiles are
// K-major, no swizzle.  r is formed as (x - mu_hi) - mu_lo with mu split into
// two floats; TF32 operands are rounded to nearest (cvt.rna).
#include <cuda_bf16.h>

#include "erx_batch.cuh"
#include "erx_internal.cuh"
#include "tc_util.cuh"

namespace erx {
namespace {

constexpr int kPix = 128;
constexpr int kB = kFactorBlock;     // 32 outputs per block
constexpr uint32_t kLBO = 128;
constexpr uint32_t kWaitLimit = 1u << 26;

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

__device__ __forceinline__ uint32_t tf32_bits(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// 16 bytes of operand data (4 tf32 or 8 bf16 values) from consecutive floats
template <int FMT>
__device__ __forceinline__ uint4 pack16(const float* v) {
  if (FMT == 2) {
    return make_uint4(tf32_bits(v[0]), tf32_bits(v[1]), tf32_bits(v[2]), tf32_bits(v[3]));
  } else {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&b);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__host__ __device__ inline int tc_dk(int d) { return (d + kB - 1) / kB * kB; }
// TMEM columns: the smallest power of two >= dK (at least 32)
__host__ __device__ inline uint32_t tc_cols(int d) {
  const int dk = tc_dk(d);
  return dk <= 32 ? 32u : dk <= 64 ? 64u : dk <= 128 ? 128u : 256u;
}

// FMT 2: TF32 (4-byte elements, 4 per core row, K = 8 per MMA);
// FMT 1: BF16 (2-byte elements, 8 per core row, K = 16 per MMA).
// Pixels tile*128 .. +127 of one line (x, pixel stride ps) with mu (d) and the
// FP32 inverse factor Xg (packed lower); delta: the line's W scores; `line` is
// reported on a timeout.
template <typename InT, int FMT>
__device__ __forceinline__ void solve_tc_body(const InT* __restrict__ x, int ps, int W, int d,
                                              const double* __restrict__ mu,
                                              const float* __restrict__ Xg,
                                              float* __restrict__ delta,
                                              unsigned long long* __restrict__ err, int64_t line,
                                              int tile) {
  constexpr int E = FMT == 2 ? 4 : 2;     // bytes per element
  constexpr int CK = 16 / E;              // elements per 16-byte core row
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ float mu_hi[kMaxDim], mu_lo[kMaxDim];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int i0 = tile * kPix;
  const int dK = tc_dk(d);
  const uint32_t ncols = tc_cols(d);
  const uint32_t sbo = (uint32_t)(dK / CK) * 128u;
  unsigned char* Rt = sm;                                  // [128][dK]
  unsigned char* Xt0 = Rt + (size_t)kPix * dK * E;         // [2][32][dK]
  const size_t xt_bytes = (size_t)kB * dK * E;
  auto off = [sbo](int row, int k) -> uint32_t {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k / CK) * kLBO + (uint32_t)(row & 7) * 16u;
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
  __syncthreads();
  // r of this thread's pixel into its row of Rt (zero beyond d or beyond the line)
  const int p = tid, i = i0 + p;
  const bool valid = i < W;
  const InT* xp = x + (int64_t)(valid ? i : 0) * ps;
  for (int k0 = 0; k0 < dK; k0 += CK) {
    float v[CK];
#pragma unroll
    for (int u = 0; u < CK; ++u) {
      const int k = k0 + u;
      v[u] = (valid && k < d) ? (to_f(xp[k]) - mu_hi[k]) - mu_lo[k] : 0.f;
    }
    *reinterpret_cast<uint4*>(Rt + off(p, k0)) = pack16<FMT>(v);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t id = tc::idesc(FMT, kPix, kB);
  const int nblk = dK / kB;
  bool ok = true;
  for (int J = 0; J < nblk && ok; ++J) {
    const int b = J & 1;
    unsigned char* Xt = Xt0 + b * xt_bytes;
    if (J >= 2) {
      const bool w_ok = tc::mbar_wait(&mbar[b], (uint32_t)((J - 2) >> 1) & 1u, kWaitLimit);
      if (__syncthreads_or(!w_ok)) {
        ok = false;
        break;
      }
    }
    // rows j0 .. j0+31 of X, columns k < j0 + 32 (zero above the diagonal and beyond d)
    const int j0 = J * kB, kcols = j0 + kB;
    for (int e = tid; e < kB * (kcols / CK); e += kPix) {
      const int jj = e % kB, kg = e / kB, j = j0 + jj;
      float v[CK];
#pragma unroll
      for (int u = 0; u < CK; ++u) {
        const int k = kg * CK + u;
        v[u] = (j < d && k <= j) ? Xg[j * (j + 1) / 2 + k] : 0.f;
      }
      *reinterpret_cast<uint4*>(Xt + off(jj, kg * CK)) = pack16<FMT>(v);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t aR = tc::smem_u32(Rt), aX = tc::smem_u32(Xt);
      for (int kk = 0; kk < kcols / (2 * CK); ++kk) {
        const uint32_t ko = (uint32_t)kk * 2u * kLBO;
        const uint64_t da = tc::desc(aR + ko, kLBO, sbo);
        const uint64_t db = tc::desc(aX + ko, kLBO, sbo);
        if (FMT == 2) tc::mma_tf32(tmem + (uint32_t)j0, da, db, id, kk > 0);
        else tc::mma_bf16(tmem + (uint32_t)j0, da, db, id, kk > 0);
      }
      tc::commit(&mbar[b]);
    }
  }
  // wait for the last commit of each buffer
  uint32_t pending_parity[2] = {0u, 0u};
  bool pending[2] = {false, false};
  for (int J = nblk - 1; J >= 0 && J >= nblk - 2; --J) {
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

template <typename InT, int FMT>
__global__ void __launch_bounds__(kPix) solve_tc_kernel(
    const InT* __restrict__ X, int64_t line_stride, int ps, int W, int d,
    const double* __restrict__ mu_t, const float* __restrict__ Lf32, float* __restrict__ delta,
    unsigned long long* __restrict__ err, int64_t t0) {
  const int t = blockIdx.y;
  solve_tc_body<InT, FMT>(X + (int64_t)t * line_stride, ps, W, d, mu_t + (int64_t)t * d,
                          Lf32 + (int64_t)t * packed_size(d), delta + (int64_t)t * W, err,
                          t0 + t, blockIdx.x);
}

// Batched form: one CTA per (stream, 128-pixel tile) item.
template <int FMT>
__global__ void __launch_bounds__(kPix) b_solve_tc_kernel(const BStream* __restrict__ S,
                                                          const BItem* __restrict__ items,
                                                          unsigned long long* __restrict__ err) {
  const BItem it = items[blockIdx.x];
  const BStream& s = S[it.s];
  solve_tc_body<float, FMT>(s.x, s.d, s.W, s.d, s.mu_t, s.Lf32, (float*)s.delta, err, it.s,
                            it.tile);
}

size_t smem_bytes(int d, int fmt) {
  const int E = fmt == 2 ? 4 : 2;
  return (size_t)(kPix + 2 * kB) * tc_dk(d) * E;
}

}  // namespace

cudaError_t configure_solve_tc_kernels() {
  cudaError_t e = cudaSuccess;
  const int m2 = (int)smem_bytes(kMaxDim, 2), m1 = (int)smem_bytes(kMaxDim, 1);
#define ERX_CFG(K, M) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, M)
  ERX_CFG((solve_tc_kernel<uint16_t, 2>), m2);
  ERX_CFG((solve_tc_kernel<float, 2>), m2);
  ERX_CFG((solve_tc_kernel<double, 2>), m2);
  ERX_CFG((solve_tc_kernel<uint16_t, 1>), m1);
  ERX_CFG((solve_tc_kernel<float, 1>), m1);
  ERX_CFG((solve_tc_kernel<double, 1>), m1);
  ERX_CFG((b_solve_tc_kernel<2>), m2);
  ERX_CFG((b_solve_tc_kernel<1>), m1);
#undef ERX_CFG
  return e;
}

void launch_batch_solve_tc(int fmt, const BStream* S, const BItem* items, int n_items, int dmax,
                           unsigned long long* err, cudaStream_t st) {
  if (fmt == 2)
    b_solve_tc_kernel<2><<<n_items, kPix, smem_bytes(dmax, 2), st>>>(S, items, err);
  else
    b_solve_tc_kernel<1><<<n_items, kPix, smem_bytes(dmax, 1), st>>>(S, items, err);
}

void launch_solve_tc(int fmt, int in_type, const void* x, int64_t line_stride, int ps, int W,
                     int d, int T, const double* mu_t, const float* Lf32, float* delta,
                     unsigned long long* err, int64_t t0, cudaStream_t st) {
  dim3 grid((W + kPix - 1) / kPix, T);
  const size_t sm = smem_bytes(d, fmt);
#define ERX_L(IT, F)                                                                           \
  solve_tc_kernel<IT, F><<<grid, kPix, sm, st>>>((const IT*)x, line_stride, ps, W, d, mu_t, \
                                                 Lf32, delta, err, t0)
  if (fmt == 2) {
    if (in_type == 0) ERX_L(uint16_t, 2);
    else if (in_type == 1) ERX_L(float, 2);
    else ERX_L(double, 2);
  } else {
    if (in_type == 0) ERX_L(uint16_t, 1);
    else if (in_type == 1) ERX_L(float, 1);
    else ERX_L(double, 1);
  }
#undef ERX_L
}

}  // namespace erx

// S2 (Sec. III-C) on the tensor cores for floating-point lines: the centred
// scatter  S2_ab = sum_i (z_ia - c_a)(z_ib - c_b)  about the shift c (the
// line mean rounded to float, from the mean kernel), with BF16 (FMT 1, round
// to nearest) or TF32 (FMT 2, cvt.rna) operands and FP32 accumulation in
// tensor memory.
//
// Operand: the chunk's centred values as a bands x pixels tile (K = pixels),
// K-major, no swizzle.  Bands 0..127 are one M = 128 tile (N = d, or 128 when
// d > 128: only the lower triangle is kept); for d > 128 bands 128..255 are a
// second M tile with N = d.  TMEM: tile 0 at column 0, tile 1 at column 128.
//
// One persistent CTA per SM walks lines.  The line's 32-pixel chunks (32 x d
// floats, contiguous) arrive in a 3-stage ring of bulk asynchronous copies
// issued ahead; warps 0-7 convert a chunk into the operand tile of one of two
// buffers while the MMAs of the previous chunk run, and warp 8's lane 0
// issues the MMAs and the copies (so the converters do not wait for the
// issue; each converter's items are worked out once).  At the end of a line
// the accumulators are drained to the FP64 scatter array.
#include <cuda_bf16.h>

#include "erx_internal.cuh"
#include "tc_util.cuh"

namespace erx {
namespace {

constexpr int kConv = 256;              // converter threads (warps 0-7)
constexpr int kThreads = kConv + 32;    // + the issuing warp
constexpr int kKC = 32;                 // pixels per chunk
constexpr int kMaxItems = (kMaxDim * (kKC / 4) + kConv - 1) / kConv;   // items per converter
constexpr int kStages = 3;              // raw ring depth
constexpr uint32_t kLBO = 128;          // next core matrix along K
constexpr uint32_t kWaitLimit = 1u << 26;

__host__ __device__ inline int syrk_rows(int d) { return d <= 128 ? 128 : 256; }
__host__ __device__ inline int syrk_raw_bytes(int d) { return ((kKC * d * 4) + 127) & ~127; }

__device__ __forceinline__ uint32_t tf32_bits(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

template <int FMT>
__global__ void __launch_bounds__(kThreads, 1) syrk_tc_kernel(
    const float* __restrict__ X, int64_t line_stride, int W, int d, int T,
    const double* __restrict__ shift, double* __restrict__ S2f,
    unsigned long long* __restrict__ err, int64_t t0) {
  constexpr int E = FMT == 1 ? 2 : 4;           // operand bytes
  constexpr int CK = 16 / E;                    // pixels per 16-byte core row
  constexpr int KS = 32 / E;                    // pixels per MMA (K)
  constexpr uint32_t SBO = (kKC / CK) * 128u;   // next 8 bands
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t rbar[kStages];
  __shared__ uint32_t tslot;
  __shared__ float sh[kMaxDim];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = syrk_rows(d);
  const int tile_bytes = R * kKC * E;
  const int raw_bytes = syrk_raw_bytes(d);
  unsigned char* raw = sm + 2 * tile_bytes;
  const int N0 = d <= 128 ? ((d + 15) & ~15) : 128;
  const int N1 = d <= 128 ? 0 : ((d + 15) & ~15);
  const uint32_t ncols = d <= 128 ? 128u : 512u;
  // rows >= d of every tile stay zero
  for (int i = tid; i < 2 * tile_bytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    for (int r = 0; r < kStages; ++r) tc::mbar_init(&rbar[r], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t id0 = tc::idesc(FMT, 128, N0);
  const uint32_t id1 = tc::idesc(FMT, 128, N1 > 0 ? N1 : 16);
  const int nchunk = (W + kKC - 1) / kKC;
  const int nlines = blockIdx.x < T ? (T - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int Q = nlines * nchunk;
  const int items = d * (kKC / CK);
  auto issue = [&](int q) {
    if (q >= Q) return;
    const int slot = q % kStages;
    const int t = blockIdx.x + (q / nchunk) * gridDim.x, ci = q % nchunk;
    const int npx = min(kKC, W - ci * kKC);
    const uint32_t bytes = (uint32_t)npx * (uint32_t)d * 4u;
    tc::mbar_expect_tx(&rbar[slot], bytes);
    tc::bulk_g2s(raw + slot * raw_bytes, X + (int64_t)t * line_stride + (int64_t)ci * kKC * d,
                 bytes, &rbar[slot]);
  };
  const bool conv = tid < kConv;        // converter; tid == kConv issues
  if (tid == kConv)
    for (int q = 0; q < kStages; ++q) issue(q);
  // this converter's items: band m, pixel group g
  int im[kMaxItems], ig[kMaxItems], nit = 0;
#pragma unroll
  for (int u = 0; u < kMaxItems; ++u) {
    const int it = tid + u * kConv;
    im[u] = conv ? it % d : 0;
    ig[u] = conv ? it / d : 0;
    if (conv && it < items) nit = u + 1;
  }
  int issued_raw = min(Q, kStages);
  uint32_t issued[2] = {0u, 0u}, done[2] = {0u, 0u};
  bool timed_out = false;
  int q = 0;
  for (; q < Q && !timed_out; ++q) {
    const int t = blockIdx.x + (q / nchunk) * gridDim.x, ci = q % nchunk;
    const int b = q & 1;
    if (ci == 0)
      for (int m = tid; m < d; m += kThreads) sh[m] = (float)shift[(int64_t)t * d + m];
    if (issued[b] != done[b]) {
      const bool ok = tc::mbar_wait(&mbar[b], done[b] & 1u, kWaitLimit);
      if (ok) ++done[b];
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
    }
    {
      const bool ok = tc::mbar_wait(&rbar[q % kStages], (uint32_t)(q / kStages) & 1u, kWaitLimit);
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
    }
    const float* rw = reinterpret_cast<const float*>(raw + (q % kStages) * raw_bytes);
    unsigned char* tH = sm + b * tile_bytes;
    const int npx = min(kKC, W - ci * kKC);
#pragma unroll
    for (int u = 0; u < kMaxItems; ++u) {
      if (u >= nit) break;
      const int m = im[u], g = ig[u];
      const float c = sh[m];
      float v[CK];
#pragma unroll
      for (int u = 0; u < CK; ++u) {
        const int px = g * CK + u;
        v[u] = px < npx ? rw[px * d + m] - c : 0.f;
      }
      const uint32_t off = (uint32_t)(m >> 3) * SBO + (uint32_t)g * kLBO + (uint32_t)(m & 7) * 16u;
      if constexpr (FMT == 1) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
          w[i] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(tH + off) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = tf32_bits(v[i]);
        *reinterpret_cast<uint4*>(tH + off) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == kConv) {
      const uint32_t aH = tc::smem_u32(tH);
#pragma unroll
      for (int s = 0; s < kKC / KS; ++s) {
        const uint32_t ko = (uint32_t)s * 2u * kLBO;
        const uint32_t acc = (ci > 0 || s > 0) ? 1u : 0u;
        const uint64_t bH = tc::desc(aH + ko, kLBO, SBO);
        const uint64_t a1H = tc::desc(aH + 16u * SBO + ko, kLBO, SBO);
        if constexpr (FMT == 1) {
          tc::mma_bf16(tmem, bH, bH, id0, acc);
          if (N1) tc::mma_bf16(tmem + 128u, a1H, bH, id1, acc);
        } else {
          tc::mma_tf32(tmem, bH, bH, id0, acc);
          if (N1) tc::mma_tf32(tmem + 128u, a1H, bH, id1, acc);
        }
      }
      tc::commit(&mbar[b]);
      issue(q + kStages);       // this chunk's raw slot is free: every thread converted it
    }
    issued_raw = min(Q, q + 1 + kStages);
    ++issued[b];
    if (ci != nchunk - 1) continue;
    // end of line t: wait for its MMAs, drain the lower triangle
    for (int bb = 0; bb < 2; ++bb) {
      if (issued[bb] != done[bb]) {
        const bool ok = tc::mbar_wait(&mbar[bb], done[bb] & 1u, kWaitLimit);
        if (ok) ++done[bb];
        timed_out |= !ok;
      }
    }
    if (__syncthreads_or(timed_out)) {
      timed_out = true;
      break;
    }
    tc::fence_after_sync();
    const int quarter = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    double* s2 = S2f + (int64_t)t * d * d;
    for (int mt = 0; mt < (N1 ? 2 : 1); ++mt) {
      const int m = mt * 128 + 32 * quarter + lane;
      const int N = mt ? N1 : N0;
      for (int c0 = (warp >> 2) * 16; conv && c0 < N; c0 += 32) {
        uint32_t v[16];
        tc::tmem_ld16(lane_base + (uint32_t)(mt * 128 + c0), v);
        tc::tmem_ld_wait();
        if (m < d) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c0 + j;
            if (n <= m) s2[(int64_t)m * d + n] = (double)__uint_as_float(v[j]);
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (timed_out) {
    if (tid == 0) atomicMin(&err[kErrTimeout], (unsigned long long)(t0 + blockIdx.x));
    // copies and MMAs still in flight get one more bounded wait before the CTA leaves
    for (int r = q; r < issued_raw; ++r)
      tc::mbar_wait(&rbar[r % kStages], (uint32_t)(r / kStages) & 1u, kWaitLimit);
    for (int bb = 0; bb < 2; ++bb)
      if (issued[bb] != done[bb]) tc::mbar_wait(&mbar[bb], done[bb] & 1u, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, ncols);
}

size_t syrk_smem(int fmt, int d) {
  const int E = fmt == 1 ? 2 : 4;
  return (size_t)2 * syrk_rows(d) * kKC * E + (size_t)kStages * syrk_raw_bytes(d);
}

}  // namespace

bool syrk_tc_supported(const void* x, int64_t line_stride, int ps, int W, int d) {
  // bulk copies: 16-byte aligned line starts and chunk sizes; pixels contiguous
  return d > 16 && d <= kMaxDim && ps == d && W >= 2 && ((uintptr_t)x % 16) == 0 &&
         (line_stride % 4) == 0 && (((int64_t)W * d) % 4) == 0;
}

cudaError_t configure_syrk_tc_kernels() {
  cudaError_t e = cudaSuccess;
#define ERX_CFG(F)                                                                 \
  if (e == cudaSuccess)                                                            \
  e = cudaFuncSetAttribute(syrk_tc_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)syrk_smem(F, kMaxDim))
  ERX_CFG(1);
  ERX_CFG(2);
#undef ERX_CFG
  return e;
}

void launch_syrk_tc(int fmt, const float* x, int64_t line_stride, int W, int d, int T, int n_sm,
                    const double* shift, double* S2f, unsigned long long* err, int64_t t0,
                    cudaStream_t st) {
  const int grid = T < n_sm ? T : n_sm;
  const size_t sm = syrk_smem(fmt, d);
  if (fmt == 1)
    syrk_tc_kernel<1><<<grid, kThreads, sm, st>>>(x, line_stride, W, d, T, shift, S2f, err, t0);
  else
    syrk_tc_kernel<2><<<grid, kThreads, sm, st>>>(x, line_stride, W, d, T, shift, S2f, err, t0);
}

}  // namespace erx

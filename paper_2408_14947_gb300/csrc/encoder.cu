// Learned band encoder: codes c = W2 relu(W1 xn + b1) + b2, xn = (x - shift) * scale.
//
// The learned counterpart of the sparse random projection (Sec. III-B; the
// paper names learning-based extensions as future work): ERX then runs on k
// codes instead of b bands.  It is trained on the GPU so that code-space ERX
// ranks pixels like full-band ERX, one line per step in stream order:
//   1. forward on the tensor cores: codes of the line's p pixels (bf16
//      operands, FP32 accumulation in TMEM), keeping relu(a) in bf16;
//   2. code statistics: line mean/covariance (the FP32 forms' compensated
//      scatter), EMA update and Cholesky of K_e + eps I in FP64 (the pipeline's
//      own kernels; the statistics are constants for the gradient);
//   3. loss and dL/dc per pixel: delta = |L^-1 r|, u = L^-T L^-1 r,
//      dL/dc = (2/p) (log1p(delta) - log1p(target)) / ((1 + delta) delta) u;
//   4. backward on the tensor cores, per 128-pixel tile: dh = (dc W2) * [h > 0],
//      partial dW1 = dh^T xn and dW2 = dc^T h (bf16 operands, FP32 accumulation),
//      and the bias sums;
//   5. deterministic reduction of the tile partials fused with AdamW on the
//      FP32 master weights, which also refreshes their bf16 copies.
// Training and inference share the forward, so the network is scored with the
// arithmetic it was trained with.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/erx.h"
#include "erx_internal.cuh"
#include "tc_util.cuh"

using namespace erx;

namespace {

constexpr int kTile = 128;      // pixels per backward tile (the MMA's M)
constexpr int kThreads = 256;
constexpr int kMaxB = 256, kMaxH = 128, kMaxK = 32;

// ---- forward on the tensor cores -------------------------------------------
// Both layers are dense contractions over a 128-pixel tile (M = 128):
//   layer 1: A = xn (pixels x bands, bf16), B = W1 (hidden x bands, bf16), N = h;
//   layer 2: A = relu(a + b1) (pixels x hidden, bf16), B = W2 (codes x hidden), N = k;
// FP32 accumulation in tensor memory (layer 1 at column 0, layer 2 at column
// 256).  Operand tiles are K-major, no swizzle (8-row x 16-byte core matrices);
// band, hidden and code counts are padded to multiples of 16 with zero weights
// (a padded hidden unit has zero weights and bias, so relu gives 0).  One
// persistent CTA per SM keeps W1 and W2 in shared memory and walks the tiles:
// stage xn = (x - shift) * scale as bf16, layer-1 MMAs, epilogue (bias, relu,
// bf16 into the layer-2 operand, and into hout for training's backward when
// given), layer-2 MMAs, epilogue (bias, FP32 codes).
constexpr int kFT = 256;                    // threads
constexpr uint32_t kFLBO = 128;
constexpr uint32_t kFWait = 1u << 26;

__host__ __device__ inline int pad16(int v) { return (v + 15) & ~15; }
__host__ __device__ inline size_t fwd_tc_smem(int b, int h, int k) {
  const int bK = pad16(b), hP = pad16(h), kP = pad16(k);
  return (size_t)2 * ((size_t)128 * bK + (size_t)hP * bK + (size_t)128 * hP + (size_t)kP * hP) +
         (size_t)4 * (2 * bK + hP + kP);
}

__device__ __forceinline__ uint32_t fwd_off(int row, int kk, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(kk >> 3) * kFLBO + (uint32_t)(row & 7) * 16u;
}

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(kFT, 1) enc_fwd_tc_kernel(
    const float* __restrict__ x, int64_t n, int b, int h, int k, const float* __restrict__ shift,
    const float* __restrict__ scale, const __nv_bfloat16* __restrict__ W1,
    const float* __restrict__ b1, const __nv_bfloat16* __restrict__ W2,
    const float* __restrict__ b2, float* __restrict__ codes, __nv_bfloat16* __restrict__ hout,
    unsigned long long* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smtc[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int bK = pad16(b), hP = pad16(h), kP = pad16(k);
  const uint32_t sbo1 = (uint32_t)(bK / 8) * 128u, sbo2 = (uint32_t)(hP / 8) * 128u;
  unsigned char* A1 = smtc;                                // [128][bK]
  unsigned char* B1 = A1 + (size_t)128 * bK * 2;           // [hP][bK]
  unsigned char* A2 = B1 + (size_t)hP * bK * 2;            // [128][hP]
  unsigned char* B2 = A2 + (size_t)128 * hP * 2;           // [kP][hP]
  float* s_shift = reinterpret_cast<float*>(B2 + (size_t)kP * hP * 2);
  float* s_scale = s_shift + bK;
  float* s_b1 = s_scale + bK;
  float* s_b2 = s_b1 + hP;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // weights, biases and the normalisation, once per CTA (zero padding)
  for (int it = tid; it < hP * (bK / 8); it += kFT) {
    const int j = it / (bK / 8), g = it % (bK / 8);
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q0 = 8 * g + 2 * u;
      const float v0 = (j < h && q0 < b) ? __bfloat162float(W1[(size_t)j * b + q0]) : 0.f;
      const float v1 = (j < h && q0 + 1 < b) ? __bfloat162float(W1[(size_t)j * b + q0 + 1]) : 0.f;
      w[u] = pack_bf2(v0, v1);
    }
    *reinterpret_cast<uint4*>(B1 + fwd_off(j, 8 * g, sbo1)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  for (int it = tid; it < kP * (hP / 8); it += kFT) {
    const int c = it / (hP / 8), g = it % (hP / 8);
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j0 = 8 * g + 2 * u;
      const float v0 = (c < k && j0 < h) ? __bfloat162float(W2[(size_t)c * h + j0]) : 0.f;
      const float v1 = (c < k && j0 + 1 < h) ? __bfloat162float(W2[(size_t)c * h + j0 + 1]) : 0.f;
      w[u] = pack_bf2(v0, v1);
    }
    *reinterpret_cast<uint4*>(B2 + fwd_off(c, 8 * g, sbo2)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  for (int q = tid; q < bK; q += kFT) {
    s_shift[q] = q < b ? shift[q] : 0.f;
    s_scale[q] = q < b ? scale[q] : 0.f;
  }
  for (int j = tid; j < hP; j += kFT) s_b1[j] = j < h ? b1[j] : 0.f;
  for (int c = tid; c < kP; c += kFT) s_b2[c] = c < k ? b2[c] : 0.f;
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t id1 = tc::idesc(1, 128, hP), id2 = tc::idesc(1, 128, kP);
  const int64_t ntile = (n + 127) / 128;
  const bool vec8 = (b % 8) == 0 && ((uintptr_t)x % 16) == 0;   // pixel rows start on 32 bytes
  uint32_t phase = 0;
  bool ok = true;
  // vec8: a thread's items (8 bands of a pixel each) of the next tile are loaded
  // into registers right after the current tile's layer-1 MMAs are issued, so
  // the loads run under the MMAs and both epilogues instead of before them
  constexpr int kFItems = 128 * (kMaxB / 8) / kFT;   // items per thread at most
  const int nit = 128 * (bK / 8);
  float4 pf0[kFItems], pf1[kFItems];
  auto load_tile = [&](int64_t i0n) {
#pragma unroll
    for (int u = 0; u < kFItems; ++u) {
      const int it = tid + u * kFT;
      const int p = it / (bK / 8), g = it % (bK / 8);
      const int64_t i = i0n + p;
      if (it < nit && i < n && 8 * g < b) {
        pf0[u] = __ldg(reinterpret_cast<const float4*>(x + i * b + 8 * g));
        pf1[u] = __ldg(reinterpret_cast<const float4*>(x + i * b + 8 * g + 4));
      }
    }
  };
  auto store_tile = [&](int64_t i0c) {
#pragma unroll
    for (int u = 0; u < kFItems; ++u) {
      const int it = tid + u * kFT;
      if (it >= nit) break;
      const int p = it / (bK / 8), g = it % (bK / 8);
      const int64_t i = i0c + p;
      float v[8];
      if (i < n && 8 * g < b) {
        v[0] = pf0[u].x, v[1] = pf0[u].y, v[2] = pf0[u].z, v[3] = pf0[u].w;
        v[4] = pf1[u].x, v[5] = pf1[u].y, v[6] = pf1[u].z, v[7] = pf1[u].w;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (v[q] - s_shift[8 * g + q]) * s_scale[8 * g + q];
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = 0.f;
      }
      *reinterpret_cast<uint4*>(A1 + fwd_off(p, 8 * g, sbo1)) =
          make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                     pack_bf2(v[6], v[7]));
    }
  };
  if (vec8 && (int64_t)blockIdx.x < ntile) load_tile((int64_t)blockIdx.x * 128);
  for (int64_t tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
    const int64_t i0 = tile * 128;
    // xn of the tile's pixels as bf16 (rows beyond n and bands beyond b: 0)
    if (vec8) {
      // eight bands per item from the two 16-byte loads made while the previous
      // tile was multiplied (prefetch below)
      store_tile(i0);
    } else {
      for (int it = tid; it < 128 * (bK / 8); it += kFT) {
        const int p = it / (bK / 8), g = it % (bK / 8);
        const int64_t i = i0 + p;
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q0 = 8 * g + 2 * u;
          const float v0 = (i < n && q0 < b) ? (x[i * b + q0] - s_shift[q0]) * s_scale[q0] : 0.f;
          const float v1 = (i < n && q0 + 1 < b)
                               ? (x[i * b + q0 + 1] - s_shift[q0 + 1]) * s_scale[q0 + 1]
                               : 0.f;
          w[u] = pack_bf2(v0, v1);
        }
        *reinterpret_cast<uint4*>(A1 + fwd_off(p, 8 * g, sbo1)) =
            make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t a = tc::smem_u32(A1), bb = tc::smem_u32(B1);
      for (int s = 0; s < bK / 16; ++s) {
        const uint32_t ko = (uint32_t)s * 2u * kFLBO;
        tc::mma_bf16(tmem, tc::desc(a + ko, kFLBO, sbo1), tc::desc(bb + ko, kFLBO, sbo1), id1,
                     s > 0);
      }
      tc::commit(&mbar);
    }
    // A1 is read by the MMAs only; the registers are free: the next tile's loads
    if (vec8 && tile + gridDim.x < ntile) load_tile((tile + gridDim.x) * 128);
    ok = tc::mbar_wait(&mbar, phase, kFWait);
    if (ok) phase ^= 1u;      // after a timeout, phase stays the parity still awaited
    if (__syncthreads_or(!ok)) break;
    tc::fence_after_sync();
    // epilogue 1: warp w reads TMEM lanes 32 (w % 4) .. (pixels), 16-column chunks
    {
      const int p = 32 * (warp & 3) + lane;
      const uint32_t lb = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
      for (int c0 = (warp >> 2) * 16; c0 < hP; c0 += 32) {
        uint32_t v[16];
        tc::tmem_ld16(lb + (uint32_t)c0, v);
        tc::tmem_ld_wait();
        uint32_t w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          w[u] = pack_bf2(fmaxf(__uint_as_float(v[2 * u]) + s_b1[c0 + 2 * u], 0.f),
                          fmaxf(__uint_as_float(v[2 * u + 1]) + s_b1[c0 + 2 * u + 1], 0.f));
        *reinterpret_cast<uint4*>(A2 + fwd_off(p, c0, sbo2)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(A2 + fwd_off(p, c0 + 8, sbo2)) =
            make_uint4(w[4], w[5], w[6], w[7]);
        if (hout && i0 + p < n) {
          const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(w);
          __nv_bfloat16* dst = hout + (i0 + p) * h;
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (c0 + u < h) dst[c0 + u] = hb[u];
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t a = tc::smem_u32(A2), bb = tc::smem_u32(B2);
      for (int s = 0; s < hP / 16; ++s) {
        const uint32_t ko = (uint32_t)s * 2u * kFLBO;
        tc::mma_bf16(tmem + 256u, tc::desc(a + ko, kFLBO, sbo2), tc::desc(bb + ko, kFLBO, sbo2),
                     id2, s > 0);
      }
      tc::commit(&mbar);
    }
    ok = tc::mbar_wait(&mbar, phase, kFWait);
    if (ok) phase ^= 1u;      // after a timeout, phase stays the parity still awaited
    if (__syncthreads_or(!ok)) break;
    tc::fence_after_sync();
    // epilogue 2: codes of the tile's pixels
    if (warp < 4) {
      const int p = 32 * warp + lane;
      const int64_t i = i0 + p;
      const uint32_t lb = tmem + 256u + ((uint32_t)(32 * warp) << 16);
      for (int c0 = 0; c0 < kP; c0 += 16) {
        uint32_t v[16];
        tc::tmem_ld16(lb + (uint32_t)c0, v);
        tc::tmem_ld_wait();
        if (i < n) {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (c0 + u < k) codes[i * k + c0 + u] = __uint_as_float(v[u]) + s_b2[c0 + u];
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (!ok) {
    if (tid == 0) atomicMin(&err[kErrTimeout], 0ull);
    tc::mbar_wait(&mbar, phase, kFWait);   // one more bounded wait for MMAs in flight
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 512);
}

// ---- loss and dL/dc -------------------------------------------------------
// Lf: the line's code factor (k <= 32: one diagonal block, i.e. L^-1, packed).
__global__ void __launch_bounds__(kThreads) enc_loss_kernel(
    const float* __restrict__ codes, int p, int k, const double* __restrict__ mu_e,
    const float* __restrict__ Lf, const double* __restrict__ target, float* __restrict__ dc,
    float* __restrict__ loss_part) {
  __shared__ float Li[kMaxK * (kMaxK + 1) / 2];
  __shared__ float mu[kMaxK];
  __shared__ float red[kThreads / 32];
  const int P = k * (k + 1) / 2;
  for (int e = threadIdx.x; e < P; e += kThreads) Li[e] = Lf[e];
  for (int e = threadIdx.x; e < k; e += kThreads) mu[e] = (float)mu_e[e];
  __syncthreads();
  const int i = blockIdx.x * kThreads + threadIdx.x;
  float l2 = 0.f;
  if (i < p) {
    float r[kMaxK], m[kMaxK];
    for (int a = 0; a < k; ++a) r[a] = codes[(int64_t)i * k + a] - mu[a];
    float d2 = 0.f;
    for (int a = 0; a < k; ++a) {
      float s = 0.f;
      for (int c = 0; c <= a; ++c) s = fmaf(Li[a * (a + 1) / 2 + c], r[c], s);
      m[a] = s;
      d2 = fmaf(s, s, d2);
    }
    const float delta = sqrtf(d2);
    const float diff = log1pf(delta) - log1pf((float)target[i]);
    l2 = diff * diff;
    const float coef = delta > 0.f ? 2.f * diff / ((1.f + delta) * delta * (float)p) : 0.f;
    for (int c = 0; c < k; ++c) {          // u = L^-T m
      float s = 0.f;
      for (int a = c; a < k; ++a) s = fmaf(Li[a * (a + 1) / 2 + c], m[a], s);
      dc[(int64_t)i * k + c] = coef * s;
    }
  }
  for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    loss_part[blockIdx.x] = s;
  }
}

// ---- backward on the tensor cores, one 128-pixel tile per CTA --------------
// Three bf16 contractions with FP32 accumulation in TMEM (operands K-major,
// no swizzle, as in the forward):
//   G1  dc W2      A = dc   [128 px][kP]   (K = codes)   B = W2^T [hP][kP]   N = hP
//   G2  dh^T xn    A = dh^T [128 j][128 px] (K = pixels) B = xn^T [bK][128]  N = bK
//   G3  h^T dc     A = h^T  [128 j][128 px]              B = dc^T [kP][128]  N = kP
// G1's result is gated by [h > 0] into dh (FP32, row-major in shared memory,
// also summed for the b1 gradient), then rounded to bf16 and transposed into
// G2's operand.  Hidden units beyond h (up to the M = 128 of G2 and G3) are
// zero rows.  Tile partials: [W1 (h x b) | b1 (h) | W2 (k x h) | b2 (k)].
constexpr int kDhStride = 132;              // floats per row of dh (bank-conflict padding)
constexpr uint32_t kSboPx = 16 * 128;       // 8-row group stride of a 128-pixel K extent

__host__ __device__ inline size_t bwd_tc_smem(int b, int h, int k) {
  const size_t bK = pad16(b), hP = pad16(h), kP = pad16(k);
  return 128 * kP * 2 + hP * kP * 2 + (size_t)128 * kDhStride * 4 + 128 * 128 * 2 +
         bK * 128 * 2 + 128 * 128 * 2 + kP * 128 * 2;
}

__global__ void __launch_bounds__(kThreads, 1) enc_bwd_tc_kernel(
    const float* __restrict__ x, int p, int b, int h, int k, const float* __restrict__ shift,
    const float* __restrict__ scale, const __nv_bfloat16* __restrict__ W2,
    const __nv_bfloat16* __restrict__ hbuf, const float* __restrict__ dc,
    float* __restrict__ part, unsigned long long* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smb[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int bK = pad16(b), hP = pad16(h), kP = pad16(k);
  const uint32_t sboK = (uint32_t)(kP / 8) * 128u;
  unsigned char* A1 = smb;                                   // dc     [128][kP]
  unsigned char* B1 = A1 + (size_t)128 * kP * 2;             // W2^T   [hP][kP]
  float* dhs = reinterpret_cast<float*>(B1 + (size_t)hP * kP * 2);   // dh [128][kDhStride]
  unsigned char* A2 = reinterpret_cast<unsigned char*>(dhs + 128 * kDhStride);  // dh^T [128][128]
  unsigned char* B2 = A2 + (size_t)128 * 128 * 2;            // xn^T   [bK][128]
  unsigned char* A3 = B2 + (size_t)bK * 128 * 2;             // h^T    [128][128]
  unsigned char* B3 = A3 + (size_t)128 * 128 * 2;            // dc^T   [kP][128]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int px0 = blockIdx.x * 128;
  const int np = min(128, p - px0);
  const int64_t nparam = (int64_t)h * b + h + (int64_t)k * h + k;
  float* out = part + (int64_t)blockIdx.x * nparam;

  // ---- stage the operands (zero outside the tile, the hidden units and codes)
  for (int it = tid; it < 128 * (kP / 8); it += kThreads) {          // A1: dc rows
    const int q = it / (kP / 8), g = it % (kP / 8);
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      v[u] = (q < np && 8 * g + u < k) ? dc[(int64_t)(px0 + q) * k + 8 * g + u] : 0.f;
    *reinterpret_cast<uint4*>(A1 + fwd_off(q, 8 * g, sboK)) =
        make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                   pack_bf2(v[6], v[7]));
  }
  for (int it = tid; it < hP * (kP / 8); it += kThreads) {           // B1: W2^T
    const int j = it % hP, g = it / hP;
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      v[u] = (j < h && 8 * g + u < k) ? __bfloat162float(W2[(size_t)(8 * g + u) * h + j]) : 0.f;
    *reinterpret_cast<uint4*>(B1 + fwd_off(j, 8 * g, sboK)) =
        make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                   pack_bf2(v[6], v[7]));
  }
  for (int it = tid; it < bK * 16; it += kThreads) {                 // B2: xn^T
    const int q = it % bK, g = it / bK;
    float v[8];
    const float sh = q < b ? shift[q] : 0.f, sc = q < b ? scale[q] : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = 8 * g + u;
      v[u] = (q < b && r < np) ? (x[(int64_t)(px0 + r) * b + q] - sh) * sc : 0.f;
    }
    *reinterpret_cast<uint4*>(B2 + fwd_off(q, 8 * g, kSboPx)) =
        make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                   pack_bf2(v[6], v[7]));
  }
  for (int it = tid; it < 128 * 16; it += kThreads) {                // A3: h^T
    const int j = it % 128, g = it / 128;
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = 8 * g + u;
      v[u] = (j < h && r < np) ? __bfloat162float(hbuf[(int64_t)(px0 + r) * h + j]) : 0.f;
    }
    *reinterpret_cast<uint4*>(A3 + fwd_off(j, 8 * g, kSboPx)) =
        make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                   pack_bf2(v[6], v[7]));
  }
  for (int it = tid; it < kP * 16; it += kThreads) {                 // B3: dc^T
    const int c = it % kP, g = it / kP;
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = 8 * g + u;
      v[u] = (c < k && r < np) ? dc[(int64_t)(px0 + r) * k + c] : 0.f;
    }
    *reinterpret_cast<uint4*>(B3 + fwd_off(c, 8 * g, kSboPx)) =
        make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                   pack_bf2(v[6], v[7]));
  }
  for (int c = tid; c < k; c += kThreads) {                          // b2: sum of dc
    float s = 0.f;
    for (int r = 0; r < np; ++r) s += dc[(int64_t)(px0 + r) * k + c];
    out[(int64_t)h * b + h + (int64_t)k * h + c] = s;
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  uint32_t phase = 0;

  // ---- G1: dc W2 into TMEM columns 0 .. hP - 1
  if (tid == 0) {
    const uint32_t a = tc::smem_u32(A1), bb = tc::smem_u32(B1);
    const uint32_t id = tc::idesc(1, 128, hP);
    for (int s = 0; s < kP / 16; ++s) {
      const uint32_t ko = (uint32_t)s * 2u * kFLBO;
      tc::mma_bf16(tmem, tc::desc(a + ko, kFLBO, sboK), tc::desc(bb + ko, kFLBO, sboK), id, s > 0);
    }
    tc::commit(&mbar);
  }
  bool ok = tc::mbar_wait(&mbar, phase, kFWait);
  if (ok) phase ^= 1u;        // after a timeout, phase stays the parity still awaited
  if (!__syncthreads_or(!ok)) {
    tc::fence_after_sync();
    // epilogue 1: lane = pixel; dh = (dc W2) * [h > 0] into dhs (FP32)
    const int r = 32 * (warp & 3) + lane;
    const uint32_t lb = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int c0 = (warp >> 2) * 16; c0 < hP; c0 += 32) {
      uint32_t v[16];
      tc::tmem_ld16(lb + (uint32_t)c0, v);
      tc::tmem_ld_wait();
      float o[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int j = c0 + u;
        const bool on = r < np && j < h && __bfloat162float(hbuf[(int64_t)(px0 + r) * h + j]) > 0.f;
        o[u] = on ? __uint_as_float(v[u]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; u += 4)
        *reinterpret_cast<float4*>(dhs + r * kDhStride + c0 + u) =
            make_float4(o[u], o[u + 1], o[u + 2], o[u + 3]);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // dh^T as G2's A operand (bf16), hidden units beyond hP zero; b1 = sum of dh
    for (int it = tid; it < 128 * 16; it += kThreads) {
      const int j = it % 128, g = it / 128;
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = j < hP ? dhs[(8 * g + u) * kDhStride + j] : 0.f;
      *reinterpret_cast<uint4*>(A2 + fwd_off(j, 8 * g, kSboPx)) =
          make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                     pack_bf2(v[6], v[7]));
    }
    for (int j = tid; j < h; j += kThreads) {
      float s = 0.f;
      for (int q = 0; q < np; ++q) s += dhs[q * kDhStride + j];
      out[(int64_t)h * b + j] = s;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- G2 into columns 0 .. bK - 1 (G1's result has been read), G3 into 256 ..
    if (tid == 0) {
      const uint32_t id2 = tc::idesc(1, 128, bK), id3 = tc::idesc(1, 128, kP);
      const uint32_t a2 = tc::smem_u32(A2), b2 = tc::smem_u32(B2);
      const uint32_t a3 = tc::smem_u32(A3), b3 = tc::smem_u32(B3);
      for (int s = 0; s < 8; ++s) {
        const uint32_t ko = (uint32_t)s * 2u * kFLBO;
        tc::mma_bf16(tmem, tc::desc(a2 + ko, kFLBO, kSboPx), tc::desc(b2 + ko, kFLBO, kSboPx),
                     id2, s > 0);
        tc::mma_bf16(tmem + 256u, tc::desc(a3 + ko, kFLBO, kSboPx),
                     tc::desc(b3 + ko, kFLBO, kSboPx), id3, s > 0);
      }
      tc::commit(&mbar);
    }
    ok = tc::mbar_wait(&mbar, phase, kFWait);
    if (ok) phase ^= 1u;      // after a timeout, phase stays the parity still awaited
    if (!__syncthreads_or(!ok)) {
      tc::fence_after_sync();
      // epilogue 2: lane = hidden unit j; dW1 row j, dW2 column j
      const int j = 32 * (warp & 3) + lane;
      const uint32_t lb2 = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
      for (int c0 = (warp >> 2) * 16; c0 < bK; c0 += 32) {
        uint32_t v[16];
        tc::tmem_ld16(lb2 + (uint32_t)c0, v);
        tc::tmem_ld_wait();
        if (j < h) {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (c0 + u < b) out[(int64_t)j * b + c0 + u] = __uint_as_float(v[u]);
        }
      }
      float* o2 = out + (int64_t)h * b + h;
      for (int c0 = (warp >> 2) * 16; c0 < kP; c0 += 32) {
        uint32_t v[16];
        tc::tmem_ld16(lb2 + 256u + (uint32_t)c0, v);
        tc::tmem_ld_wait();
        if (j < h) {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (c0 + u < k) o2[(int64_t)(c0 + u) * h + j] = __uint_as_float(v[u]);
        }
      }
    }
  }
  if (!ok) {
    if (tid == 0) atomicMin(&err[kErrTimeout], 0ull);
    tc::mbar_wait(&mbar, phase, kFWait);   // one more bounded wait for MMAs in flight
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 512);
}

// ---- reduction over tiles + AdamW -----------------------------------------
__global__ void __launch_bounds__(256) enc_adamw_kernel(
    const float* __restrict__ part, int ntiles, int64_t nparam, float* __restrict__ theta,
    float* __restrict__ m, float* __restrict__ v, float* __restrict__ grad_out, int apply,
    float lr, float beta1, float beta2, float eps, float wd, float c1, float c2,
    __nv_bfloat16* __restrict__ w1b, int64_t n_w1, __nv_bfloat16* __restrict__ w2b,
    int64_t off_w2, int64_t n_w2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nparam) return;
  float g = 0.f;
  for (int t = 0; t < ntiles; ++t) g += part[(int64_t)t * nparam + e];
  if (grad_out) grad_out[e] = g;
  if (!apply) return;
  const float mm = beta1 * m[e] + (1.f - beta1) * g;
  const float vv = beta2 * v[e] + (1.f - beta2) * g * g;
  m[e] = mm;
  v[e] = vv;
  const float th = theta[e] - lr * ((mm / c1) / (sqrtf(vv / c2) + eps) + wd * theta[e]);
  theta[e] = th;
  if (e < n_w1) w1b[e] = __float2bfloat16_rn(th);
  else if (e >= off_w2 && e < off_w2 + n_w2) w2b[e - off_w2] = __float2bfloat16_rn(th);
}

__global__ void enc_sum_kernel(const float* __restrict__ part, int n, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                               int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = __float2bfloat16_rn(src[e]);
}

uint64_t sm64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// standard normal from two SplitMix64 outputs (Box-Muller)
double normal_at(uint64_t seed, uint64_t k) {
  const double u1 = ((double)(sm64(seed, 2 * k) >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(sm64(seed, 2 * k + 1) >> 11) * 0x1.0p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct erx_encoder {
  int b = 0, h = 0, k = 0;
  cudaStream_t stream = nullptr;
  bool failed = false;
  int64_t nparam = 0, off_b1 = 0, off_w2 = 0, off_b2 = 0;
  float* theta = nullptr;      // [W1 | b1 | W2 | b2] FP32 master
  float* mom1 = nullptr;
  float* mom2 = nullptr;
  __nv_bfloat16* w1b = nullptr;
  __nv_bfloat16* w2b = nullptr;
  float* shift = nullptr;
  float* scale = nullptr;
  int64_t adam_k = 0;
  // training scratch for lines of up to cap_p pixels
  int cap_p = 0;
  float* codes = nullptr;
  __nv_bfloat16* hbuf = nullptr;
  float* dc = nullptr;
  float* part = nullptr;
  float* loss_part = nullptr;
  float* loss_dev = nullptr;
  float* grad = nullptr;
  // code-space statistics (pipeline buffers, one line)
  double *mu_hat = nullptr, *shiftc = nullptr, *S2f = nullptr, *mu_t = nullptr, *K_t = nullptr,
         *Lf = nullptr, *mu_e = nullptr, *K_e = nullptr;
  float* Lf32 = nullptr;
  unsigned long long* err = nullptr;
  int64_t t_codes = 0;
  std::vector<void*> allocs;
};

namespace {

template <typename T>
erx_status ealloc(erx_encoder* e, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ENOMEM;
  }
  e->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return ERX_OK;
}

erx_status ensure_capacity(erx_encoder* e, int p) {
  if (p <= e->cap_p) return ERX_OK;
  const int ntile = (p + kTile - 1) / kTile;
  erx_status s = ealloc(e, &e->codes, (size_t)p * e->k);
  if (s == ERX_OK) s = ealloc(e, &e->hbuf, (size_t)p * e->h);
  if (s == ERX_OK) s = ealloc(e, &e->dc, (size_t)p * e->k);
  if (s == ERX_OK) s = ealloc(e, &e->part, (size_t)ntile * e->nparam);
  if (s == ERX_OK) s = ealloc(e, &e->loss_part, (size_t)(p + kThreads - 1) / kThreads);
  if (s == ERX_OK) e->cap_p = p;
  return s;
}

erx_status ecuda(erx_encoder* e, cudaError_t c) {
  if (c == cudaSuccess) return ERX_OK;
  cudaGetLastError();
  e->failed = true;
  return ERX_ECUDA;
}

// forward of n pixels on the tensor cores: codes, and relu(W1 xn + b1) in bf16
// into hout when given (training); one persistent CTA per SM
void forward_tc(erx_encoder* e, const float* x, int64_t n, float* codes, __nv_bfloat16* hout,
                cudaStream_t st) {
  const int n_sm = device_shape().n_sm;
  const int64_t tiles = (n + 127) / 128;
  const int grid = (int)std::min<int64_t>(tiles, n_sm);
  enc_fwd_tc_kernel<<<grid, kFT, fwd_tc_smem(e->b, e->h, e->k), st>>>(
      x, n, e->b, e->h, e->k, e->shift, e->scale, e->w1b, e->theta + e->off_b1, e->w2b,
      e->theta + e->off_b2, codes, hout, e->err);
}

// One line: forward, code statistics (update then score), loss, backward and,
// when `apply`, the AdamW step.  grad_out (device, nparam) receives the gradient.
erx_status train_line(erx_encoder* e, const float* line, int p, const double* target,
                      const erx_train_opts* o, int apply, float* grad_out) {
  cudaStream_t st = e->stream;
  erx_status s = ensure_capacity(e, p);
  if (s != ERX_OK) return s;
  forward_tc(e, line, p, e->codes, e->hbuf, st);
  const int k = e->k;
  // code statistics with the FP32 forms' scatter (products in 8-pixel FMA runs
  // added into TwoSum-compensated float pairs, about a float rounding of the
  // exact sums): a line's k x k scatter is one block pair, and in FP64 that one
  // CTA would spend ~1M DFMA on a single SM; the mean, EMA and factor stay FP64
  launch_mean(ERX_F32, e->codes, 0, k, p, k, 1, true, e->mu_hat, e->shiftc, st);
  launch_stats_fp(ERX_F32, false, e->codes, 0, k, p, k, 1, e->shiftc, e->S2f, st);
  launch_ema_scan(false, nullptr, nullptr, e->mu_hat, e->shiftc, e->S2f, 1, k, p, o->momentum,
                  e->t_codes, ERX_UPDATE_THEN_SCORE, e->mu_e, e->K_e, e->mu_t, e->K_t, nullptr,
                  st);
  launch_chol_inv(e->K_t, k, 1, o->ridge, e->Lf, e->Lf32, e->err, e->t_codes, st);
  e->t_codes += 1;
  const int nlb = (p + kThreads - 1) / kThreads;
  enc_loss_kernel<<<nlb, kThreads, 0, st>>>(e->codes, p, k, e->mu_t, e->Lf32, target, e->dc,
                                            e->loss_part);
  enc_sum_kernel<<<1, 32, 0, st>>>(e->loss_part, nlb, e->loss_dev);
  const int ntile = (p + kTile - 1) / kTile;
  enc_bwd_tc_kernel<<<ntile, kThreads, bwd_tc_smem(e->b, e->h, k), st>>>(
      line, p, e->b, e->h, k, e->shift, e->scale, e->w2b, e->hbuf, e->dc, e->part, e->err);
  float c1 = 1.f, c2 = 1.f;
  if (apply) {
    e->adam_k += 1;
    c1 = (float)(1.0 - std::pow((double)o->beta1, (double)e->adam_k));
    c2 = (float)(1.0 - std::pow((double)o->beta2, (double)e->adam_k));
  }
  enc_adamw_kernel<<<(unsigned)((e->nparam + 255) / 256), 256, 0, st>>>(
      e->part, ntile, e->nparam, e->theta, e->mom1, e->mom2, grad_out, apply, o->lr, o->beta1,
      o->beta2, o->eps, o->weight_decay, c1, c2, e->w1b, (int64_t)e->h * e->b, e->w2b, e->off_w2,
      (int64_t)e->k * e->h);
  return ecuda(e, cudaGetLastError());
}

}  // namespace

namespace erx {
int encoder_k(const erx_encoder* e) { return e->k; }
int encoder_bands(const erx_encoder* e) { return e->b; }
void encoder_forward_on(erx_encoder* e, const float* x, int64_t n, float* codes, cudaStream_t st) {
  forward_tc(e, x, n, codes, nullptr, st);
}
}  // namespace erx

namespace {
constexpr char kCkptMagic[8] = {'E', 'R', 'X', 'E', 'N', 'C', '0', '1'};

struct CkptHeader {
  char magic[8];
  int32_t bands, hidden, k, reserved;
  int64_t adam_k, t_codes;
};

// device <-> host copies of the checkpoint's arrays, in file order
struct CkptArrays {
  std::vector<float> shift, scale, theta, m, v;
  std::vector<double> mu, K;
  explicit CkptArrays(const erx_encoder* e)
      : shift(e->b), scale(e->b), theta(e->nparam), m(e->nparam), v(e->nparam), mu(e->k),
        K(packed_size(e->k)) {}
  template <typename F>
  bool each(F&& f) {
    return f(shift.data(), shift.size() * 4) && f(scale.data(), scale.size() * 4) &&
           f(theta.data(), theta.size() * 4) && f(m.data(), m.size() * 4) &&
           f(v.data(), v.size() * 4) && f(mu.data(), mu.size() * 8) && f(K.data(), K.size() * 8);
  }
};
}  // namespace

extern "C" {

void erx_train_opts_default(erx_train_opts* o) {
  if (!o) return;
  o->momentum = 0.1;
  o->ridge = 1e-5;
  o->lr = 1e-3f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->weight_decay = 1e-4f;
}

erx_status erx_encoder_create(int32_t bands, int32_t hidden, int32_t k, uint64_t seed,
                              void* cuda_stream, erx_encoder** out) {
  if (!out) return ERX_EINVAL;
  *out = nullptr;
  if (bands < 1 || hidden < 1 || k < 2) return ERX_EINVAL;
  if (bands > kMaxB || hidden > kMaxH || k > kMaxK) return ERX_EUNSUPPORTED;
  erx_encoder* e = new (std::nothrow) erx_encoder();
  if (!e) return ERX_ENOMEM;
  e->b = bands;
  e->h = hidden;
  e->k = k;
  e->stream = (cudaStream_t)cuda_stream;
  e->off_b1 = (int64_t)hidden * bands;
  e->off_w2 = e->off_b1 + hidden;
  e->off_b2 = e->off_w2 + (int64_t)k * hidden;
  e->nparam = e->off_b2 + k;
  const int64_t P = packed_size(k);
  erx_status s = ERX_OK;
#define EA(p, n) \
  if (s == ERX_OK) s = ealloc(e, &e->p, (size_t)(n))
  EA(theta, e->nparam);
  EA(mom1, e->nparam);
  EA(mom2, e->nparam);
  EA(grad, e->nparam);
  EA(w1b, (int64_t)hidden * bands);
  EA(w2b, (int64_t)k * hidden);
  EA(shift, bands);
  EA(scale, bands);
  EA(loss_dev, 1);
  EA(mu_hat, k);
  EA(shiftc, k);
  EA(S2f, (int64_t)k * k);
  EA(mu_t, k);
  EA(K_t, P);
  EA(Lf, P);
  EA(Lf32, P);
  EA(mu_e, k);
  EA(K_e, P);
  EA(err, kErrSlots);
#undef EA
  if (s == ERX_OK) {
    // the forward keeps both weight matrices and a 128-pixel tile in shared
    // memory, the backward a tile's six operands and dh (plus static shared memory)
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (bwd_tc_smem(bands, hidden, k) + 2048 > (size_t)optin ||
        fwd_tc_smem(bands, hidden, k) + 2048 > (size_t)optin)
      s = ERX_EUNSUPPORTED;
    else if (configure_factor_kernels() != cudaSuccess ||
             cudaFuncSetAttribute(enc_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fwd_tc_smem(bands, hidden, k)) != cudaSuccess ||
             cudaFuncSetAttribute(enc_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bwd_tc_smem(bands, hidden, k)) != cudaSuccess)
      s = ERX_ECUDA;
  }
  if (s == ERX_OK) {
    // He-style initial weights from a counter-based normal draw (SplitMix64 + Box-Muller)
    std::vector<float> th((size_t)e->nparam, 0.f);
    const double s1 = std::sqrt(2.0 / bands), s2 = std::sqrt(1.0 / hidden);
    for (int64_t i = 0; i < e->off_b1; ++i) th[i] = (float)(normal_at(seed, i) * s1);
    for (int64_t i = 0; i < (int64_t)k * hidden; ++i)
      th[e->off_w2 + i] = (float)(normal_at(seed ^ 0x5A5A5A5Aull, i) * s2);
    std::vector<float> ones(bands, 1.f), zeros(bands, 0.f);
    if (cudaMemcpy(e->theta, th.data(), th.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(e->mom1, 0, e->nparam * 4) != cudaSuccess ||
        cudaMemset(e->mom2, 0, e->nparam * 4) != cudaSuccess ||
        cudaMemcpy(e->shift, zeros.data(), bands * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->scale, ones.data(), bands * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(e->err, 0xff, sizeof(unsigned long long) * kErrSlots) != cudaSuccess)
      s = ERX_ECUDA;
    if (s == ERX_OK) {
      to_bf16_kernel<<<(unsigned)((e->off_b1 + 255) / 256), 256>>>(e->theta, e->w1b, e->off_b1);
      to_bf16_kernel<<<(unsigned)(((int64_t)k * hidden + 255) / 256), 256>>>(
          e->theta + e->off_w2, e->w2b, (int64_t)k * hidden);
      if (cudaDeviceSynchronize() != cudaSuccess) s = ERX_ECUDA;
    }
  }
  if (s != ERX_OK) {
    cudaGetLastError();
    for (void* p : e->allocs) cudaFree(p);
    delete e;
    return s;
  }
  *out = e;
  return ERX_OK;
}

erx_status erx_encoder_set_norm(erx_encoder* e, const float* shift, const float* scale) {
  if (!e || !shift || !scale) return ERX_EINVAL;
  if (e->failed) return ERX_ECUDA;
  if (cudaStreamSynchronize(e->stream) != cudaSuccess ||
      cudaMemcpy(e->shift, shift, e->b * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e->scale, scale, e->b * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return ecuda(e, cudaGetLastError());
  return ERX_OK;
}

erx_status erx_encoder_params(erx_encoder* e, float* theta_out, const float* theta_in) {
  if (!e || (!theta_out && !theta_in)) return ERX_EINVAL;
  if (e->failed) return ERX_ECUDA;
  if (cudaStreamSynchronize(e->stream) != cudaSuccess) return ecuda(e, cudaGetLastError());
  if (theta_in) {
    if (cudaMemcpy(e->theta, theta_in, e->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(e->mom1, 0, e->nparam * 4) != cudaSuccess ||
        cudaMemset(e->mom2, 0, e->nparam * 4) != cudaSuccess)
      return ecuda(e, cudaGetLastError());
    e->adam_k = 0;
    to_bf16_kernel<<<(unsigned)((e->off_b1 + 255) / 256), 256, 0, e->stream>>>(e->theta, e->w1b,
                                                                                e->off_b1);
    to_bf16_kernel<<<(unsigned)(((int64_t)e->k * e->h + 255) / 256), 256, 0, e->stream>>>(
        e->theta + e->off_w2, e->w2b, (int64_t)e->k * e->h);
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) return ecuda(e, cudaGetLastError());
  }
  if (theta_out &&
      cudaMemcpy(theta_out, e->theta, e->nparam * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ecuda(e, cudaGetLastError());
  return ERX_OK;
}

int64_t erx_encoder_nparams(const erx_encoder* e) { return e ? e->nparam : -1; }

erx_status erx_encoder_reset_stats(erx_encoder* e) {
  if (!e) return ERX_EINVAL;
  e->t_codes = 0;
  return ERX_OK;
}

erx_status erx_encoder_forward(erx_encoder* e, const float* x_dev, int64_t n_pix,
                               float* codes_dev) {
  if (!e || n_pix < 0 || (n_pix > 0 && (!x_dev || !codes_dev))) return ERX_EINVAL;
  if (e->failed) return ERX_ECUDA;
  if (n_pix == 0) return ERX_OK;
  forward_tc(e, x_dev, n_pix, codes_dev, nullptr, e->stream);
  return ecuda(e, cudaGetLastError());
}

erx_status erx_encoder_train(erx_encoder* e, const float* lines_dev, int64_t n_lines,
                             int32_t width, const double* targets_dev, const erx_train_opts* o,
                             float* loss_host) {
  if (!e || !o || n_lines < 0 || width < 2 || (n_lines > 0 && (!lines_dev || !targets_dev)))
    return ERX_EINVAL;
  if (e->failed) return ERX_ECUDA;
  for (int64_t t = 0; t < n_lines; ++t) {
    erx_status s = train_line(e, lines_dev + t * (int64_t)width * e->b, width,
                              targets_dev + t * (int64_t)width, o, 1, nullptr);
    if (s != ERX_OK) return s;
    if (loss_host) {
      float l = 0.f;
      if (cudaMemcpyAsync(&l, e->loss_dev, 4, cudaMemcpyDeviceToHost, e->stream) != cudaSuccess ||
          cudaStreamSynchronize(e->stream) != cudaSuccess)
        return ecuda(e, cudaGetLastError());
      loss_host[t] = l / (float)width;
    }
  }
  return ERX_OK;
}

erx_status erx_encoder_line_grad(erx_encoder* e, const float* line_dev, int32_t width,
                                 const double* target_dev, const erx_train_opts* o,
                                 float* grad_host, float* loss_host) {
  if (!e || !o || !line_dev || !target_dev || width < 2 || !grad_host) return ERX_EINVAL;
  if (e->failed) return ERX_ECUDA;
  erx_status s = train_line(e, line_dev, width, target_dev, o, 0, e->grad);
  if (s != ERX_OK) return s;
  float l = 0.f;
  if (cudaStreamSynchronize(e->stream) != cudaSuccess ||
      cudaMemcpy(grad_host, e->grad, e->nparam * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&l, e->loss_dev, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ecuda(e, cudaGetLastError());
  if (loss_host) *loss_host = l / (float)width;
  return ERX_OK;
}

erx_status erx_encoder_destroy(erx_encoder* e) {
  if (!e) return ERX_OK;
  cudaStreamSynchronize(e->stream);
  cudaGetLastError();
  for (void* p : e->allocs) cudaFree(p);
  delete e;
  return ERX_OK;
}


erx_status erx_encoder_save(erx_encoder* e, const char* path) {
  if (!e || !path) return ERX_EINVAL;
  if (e->failed) return ERX_ECUDA;
  CkptArrays a(e);
  if (cudaStreamSynchronize(e->stream) != cudaSuccess ||
      cudaMemcpy(a.shift.data(), e->shift, e->b * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(a.scale.data(), e->scale, e->b * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(a.theta.data(), e->theta, e->nparam * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(a.m.data(), e->mom1, e->nparam * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(a.v.data(), e->mom2, e->nparam * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(a.mu.data(), e->mu_e, e->k * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(a.K.data(), e->K_e, a.K.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ecuda(e, cudaGetLastError());
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.bands = e->b;
  hd.hidden = e->h;
  hd.k = e->k;
  hd.adam_k = e->adam_k;
  hd.t_codes = e->t_codes;
  FILE* f = std::fopen(path, "wb");
  if (!f) return ERX_EIO;
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
            a.each([f](const void* p, size_t n) { return std::fwrite(p, 1, n, f) == n; });
  ok = (std::fclose(f) == 0) && ok;
  return ok ? ERX_OK : ERX_EIO;
}

erx_status erx_encoder_load(const char* path, void* cuda_stream, erx_encoder** out) {
  if (!path || !out) return ERX_EINVAL;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return ERX_EIO;
  CkptHeader hd{};
  if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, kCkptMagic, 8) != 0 ||
      hd.bands < 1 || hd.bands > kMaxB || hd.hidden < 1 || hd.hidden > kMaxH || hd.k < 2 ||
      hd.k > kMaxK || hd.adam_k < 0 || hd.t_codes < 0) {
    std::fclose(f);
    return ERX_EIO;
  }
  erx_encoder* e = nullptr;
  erx_status s = erx_encoder_create(hd.bands, hd.hidden, hd.k, 0, cuda_stream, &e);
  if (s != ERX_OK) {
    std::fclose(f);
    return s;
  }
  CkptArrays a(e);
  bool ok = a.each([f](void* p, size_t n) { return std::fread(p, 1, n, f) == n; });
  ok = ok && std::fgetc(f) == EOF;       // nothing after the last array
  std::fclose(f);
  if (!ok) {
    erx_encoder_destroy(e);
    return ERX_EIO;
  }
  if (cudaMemcpy(e->shift, a.shift.data(), e->b * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e->scale, a.scale.data(), e->b * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e->theta, a.theta.data(), e->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e->mom1, a.m.data(), e->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e->mom2, a.v.data(), e->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e->mu_e, a.mu.data(), e->k * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e->K_e, a.K.data(), a.K.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    erx_encoder_destroy(e);
    return ERX_ECUDA;
  }
  e->adam_k = hd.adam_k;
  e->t_codes = hd.t_codes;
  // the bf16 copies the products use, from the loaded FP32 master weights
  to_bf16_kernel<<<(unsigned)((e->off_b1 + 255) / 256), 256, 0, e->stream>>>(e->theta, e->w1b,
                                                                              e->off_b1);
  to_bf16_kernel<<<(unsigned)(((int64_t)e->k * e->h + 255) / 256), 256, 0, e->stream>>>(
      e->theta + e->off_w2, e->w2b, (int64_t)e->k * e->h);
  if (cudaStreamSynchronize(e->stream) != cudaSuccess) {
    cudaGetLastError();
    erx_encoder_destroy(e);
    return ERX_ECUDA;
  }
  *out = e;
  return ERX_OK;
}

int32_t erx_encoder_dims(const erx_encoder* e, int32_t* bands, int32_t* hidden) {
  if (!e) return -1;
  if (bands) *bands = e->b;
  if (hidden) *hidden = e->h;
  return e->k;
}

}  // extern "C"

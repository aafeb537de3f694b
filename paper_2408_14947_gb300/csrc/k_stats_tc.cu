// S2 (Sec. III-C) on the tensor cores: exact integer line sums for u16 samples.
//
// Each sample (< 2^12) is split as x = 64 h + l with h, l < 64, both exact in
// bf16.  Then
//   sum_i x_ia x_ib = 4096 HH_ab + 64 (HL_ab + LH_ab) + LL_ab,
// where HH = H H^T, HL = H L^T, ... are bf16 products accumulated in FP32 in
// tensor memory.  Every partial sum is an integer below 2^24 for lines of up
// to 2048 pixels (products < 2^12, at most 2 * 2048 of them per entry), so
// the FP32 accumulation is exact and the result equals the integer sums of
// the IMAD route bit for bit.  An extra band of ones appended to the operand
// gives sum_i x_ia in the same products (column d).
//
// One persistent CTA per SM walks lines; per line, 64-pixel chunks are
// converted into two bf16 operand tiles (bands x pixels, K-major) in shared
// memory, double-buffered so that the conversion of chunk c+1 overlaps the
// MMAs of chunk c; one thread issues 16 tcgen05.mma (M = 128 bands, N = d+1
// rounded to 16, K = 16 pixels) per chunk into three accumulators
// (HH | HL+LH | LL, 512 TMEM columns) and commits them to the buffer's
// mbarrier.  The drain converts the three FP32 accumulators to int64 sums.
#include <algorithm>

#include <cuda_bf16.h>

#include "erx_internal.cuh"
#include "tc_util.cuh"

namespace erx {
namespace {

constexpr int kThreads = 256;
constexpr int kKC = 64;                              // pixels per chunk
constexpr int kRows = 128;                           // M: bands (+ ones row), padded
constexpr int kTileBytes = kRows * kKC * 2;          // 16 KiB bf16 tile
constexpr uint32_t kLBO = 128;                       // next 8 pixels (K core matrix)
constexpr uint32_t kSBO = (kKC / 8) * 128;           // next 8 bands (M core group)
constexpr uint32_t kWaitLimit = 1u << 26;
constexpr uint32_t kColHH = 0, kColMid = 128, kColLL = 256, kTmemCols = 512;
// more shared memory than two CTAs can hold, so that each SM runs one CTA and
// no CTA waits in tcgen05.alloc for another's 512 TMEM columns
constexpr int kSmemBytes = 118 * 1024;

__device__ __forceinline__ uint32_t tile_off(int m, int g) {
  return (uint32_t)(m >> 3) * kSBO + (uint32_t)g * kLBO + (uint32_t)(m & 7) * 16;
}

// Two integers below 128 in the halves of x -> the bf16 pair of their values,
// exactly: bf16 bits 0x4300 | n encode 128 + n (eight significant bits), and
// one bf16x2 subtraction of 128 leaves n.
__device__ __forceinline__ uint32_t bf16x2_small(uint32_t x) {
  const uint32_t biased = x | 0x43004300u;
  const __nv_bfloat162 r = __hsub2(*reinterpret_cast<const __nv_bfloat162*>(&biased),
                                   __floats2bfloat162_rn(128.0f, 128.0f));
  return *reinterpret_cast<const uint32_t*>(&r);
}

__device__ __forceinline__ uint32_t bf16_pair(uint32_t a, uint32_t b) {
  // small non-negative integers (< 256) are exact in bf16: value v -> bits of float(v) >> 16.
  // float(v) for v < 2^23 without an int-to-float conversion: the float whose
  // mantissa holds v above 2^23, minus 2^23 (exact).
  const uint32_t fa = __float_as_uint(__uint_as_float(0x4B000000u | a) - 8388608.0f) >> 16;
  const uint32_t fb = __float_as_uint(__uint_as_float(0x4B000000u | b) - 8388608.0f) >> 16;
  return fa | (fb << 16);
}

__global__ void __launch_bounds__(kThreads, 1) stats_tc_kernel(
    const uint16_t* __restrict__ X, int64_t line_stride, int W, int d, uint32_t maxv, int T,
    uint64_t* __restrict__ S1, uint64_t* __restrict__ S2, unsigned long long* __restrict__ err,
    int64_t t0) {
  extern __shared__ __align__(1024) unsigned char sm[];   // [2 buffers][H tile | L tile]
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = ((d + 1) + 15) & ~15;                    // N: bands + ones row, mult of 16
  for (int i = tid; i < 4 * kTileBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, kTmemCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t id = tc::idesc(1, kRows, np);
  uint32_t issued[2] = {0u, 0u}, done[2] = {0u, 0u};
  bool timed_out = false;
  const int nchunk = (W + kKC - 1) / kKC;
  const int items = (d + 1) * (kKC / 8);

  for (int t = blockIdx.x; t < T && !timed_out; t += gridDim.x) {
    const uint16_t* x = X + (int64_t)t * line_stride;
    bool bad = false;
    for (int c = 0; c < nchunk; ++c) {
      const int b = c & 1;
      if (issued[b] != done[b]) {
        const bool ok = tc::mbar_wait(&mbar[b], done[b] & 1u, kWaitLimit);
        if (ok) ++done[b];
        if (__syncthreads_or(!ok)) {
          timed_out = true;
          break;
        }
      }
      unsigned char* tH = sm + b * 2 * kTileBytes;
      unsigned char* tL = tH + kTileBytes;
      const int i0 = c * kKC;
      for (int it = tid; it < items; it += kThreads) {
        const int m = it % (d + 1), g = it / (d + 1);
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          uint32_t v[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int i = i0 + g * 8 + q + u;
            uint32_t s = 0u;
            if (i < W) s = (m < d) ? (uint32_t)x[(int64_t)i * d + m] : 1u;
            bad |= (m < d) && (s > maxv);
            v[u] = s;
          }
          hv[q / 2] = bf16_pair(v[0] >> 6, v[1] >> 6);
          lv[q / 2] = bf16_pair(v[0] & 63u, v[1] & 63u);
        }
        const uint32_t off = tile_off(m, g);
        *reinterpret_cast<uint4*>(tH + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(tL + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        const uint32_t aH = tc::smem_u32(tH), aL = tc::smem_u32(tL);
#pragma unroll
        for (int s = 0; s < kKC / 16; ++s) {
          const uint32_t ko = (uint32_t)s * 2u * kLBO;
          const uint64_t dH = tc::desc(aH + ko, kLBO, kSBO);
          const uint64_t dL = tc::desc(aL + ko, kLBO, kSBO);
          const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
          tc::mma_bf16(tmem + kColHH, dH, dH, id, acc);
          tc::mma_bf16(tmem + kColMid, dH, dL, id, acc);
          tc::mma_bf16(tmem + kColMid, dL, dH, id, 1u);
          tc::mma_bf16(tmem + kColLL, dL, dL, id, acc);
        }
        tc::commit(&mbar[b]);
      }
      ++issued[b];
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) atomicMin(&err[kErrRange], (unsigned long long)(t0 + t));
    }
    if (timed_out) break;
    for (int b = 0; b < 2; ++b) {
      if (issued[b] != done[b]) {
        const bool ok = tc::mbar_wait(&mbar[b], done[b] & 1u, kWaitLimit);
        if (ok) ++done[b];
        timed_out |= !ok;
      }
    }
    if (__syncthreads_or(timed_out)) {
      timed_out = true;
      break;
    }
    tc::fence_after_sync();
    // drain: warp w reads TMEM lanes 32 (w % 4) .. +31 (band rows), 16-column chunks
    const int m = 32 * (warp & 3) + lane;
    uint64_t* s2 = S2 + (int64_t)t * d * d;
    for (int c0 = (warp >> 2) * 16; c0 < np; c0 += 32) {
      uint32_t hh[16], md[16], ll[16];
      const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
      tc::tmem_ld16(lane_base + kColHH, hh);
      tc::tmem_ld16(lane_base + kColMid, md);
      tc::tmem_ld16(lane_base + kColLL, ll);
      tc::tmem_ld_wait();
      if (m < d) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c0 + j;
          if (n > m && n != d) continue;        // upper triangle: not needed
          // each accumulator holds an exact integer below 2^24: convert through u32
          const uint64_t v = ((uint64_t)__float2uint_rz(__uint_as_float(hh[j])) << 12) +
                             ((uint64_t)__float2uint_rz(__uint_as_float(md[j])) << 6) +
                             (uint64_t)__float2uint_rz(__uint_as_float(ll[j]));
          if (n < d) {
            if (n <= m) s2[(int64_t)m * d + n] = v;
          } else if (n == d) {
            S1[(int64_t)t * d + m] = v;
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (timed_out && tid == 0) atomicMin(&err[kErrTimeout], (unsigned long long)(t0 + blockIdx.x));
  // outstanding MMAs (only after a timeout) get one more bounded wait before TMEM is released
  for (int b = 0; b < 2; ++b)
    if (issued[b] != done[b]) tc::mbar_wait(&mbar[b], done[b] & 1u, kWaitLimit);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, kTmemCols);
}

// Same sums (the kernel above is the route for unaligned lines), with the
// line's 64-pixel chunks brought into a kRawStages-stage ring in shared memory
// by bulk asynchronous copies (cp.async.bulk, completing on an mbarrier with a
// transaction count) issued kRawStages chunks ahead, so the global-memory
// latency overlaps the conversion and the MMAs.  Needs 16-byte aligned lines
// and p * d * 2 a multiple of 16.
// Roles: warps 0-7 convert the chunks into the bf16 tiles and drain the
// accumulators; warp 8's lane 0 issues each chunk's MMAs and the bulk copies,
// so that the converters go on with the next chunk while the MMAs are issued.
// Each converter's items are the same in every chunk and are worked out once;
// for even d an item is two bands of an 8-pixel group (one 32-bit read per
// pixel, the bf16 values from one bf16x2 subtraction per pair).  Per 16
// pixels two MMAs of N = 256 (A = the H or the L tile, B = the H and L tiles
// together, which lie next to each other) fill four accumulators, HH | HL and
// LH | LL, over the 512 TMEM columns; the drain adds HL + LH as integers.
// split > 1 (a line or a few pushed alone): CTA b takes only the chunks
// b % split, b % split + split, ... of line b / split and adds its sums into
// S1 and S2 (zeroed by the launcher) with 64-bit integer atomics; integer
// sums do not depend on their order, so the result is the same bits.
constexpr int kRawStages = 8;
constexpr int kRawBytes = 16384;                  // >= 64 px * 127 bands * 2 B
// tile buffers (H | L pairs) and raw stages: two and eight (four tile buffers
// with four raw stages measured the same)
constexpr int kTileBufs = 2;
constexpr int kBulkSmem = 2 * kTileBufs * kTileBytes + kRawStages * kRawBytes;

constexpr int kConv = 256;                      // converter threads (warps 0-7)
constexpr int kBulkThreads = kConv + 32;        // + the issuing warp
constexpr int kMaxItems = (kRows * (kKC / 8) + kConv - 1) / kConv;   // items per converter

__global__ void __launch_bounds__(kBulkThreads, 1) stats_tc_bulk_kernel(
    const uint16_t* __restrict__ X, int64_t line_stride, int W, int d, uint32_t maxv, int T,
    uint64_t* __restrict__ S1, uint64_t* __restrict__ S2, unsigned long long* __restrict__ err,
    int64_t t0, int split) {
  extern __shared__ __align__(1024) unsigned char sm[];   // [2][H|L] tiles, then raw ring
  unsigned char* raw = sm + 2 * kTileBufs * kTileBytes;
  __shared__ __align__(8) uint64_t mbar[kTileBufs];
  __shared__ __align__(8) uint64_t rbar[kRawStages];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = ((d + 1) + 15) & ~15;
  for (int i = tid; i < 2 * kTileBufs * kTileBytes / 16; i += kBulkThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  const bool conv = tid < kConv;              // converter; tid == kConv issues
  if (tid == 0) {
    for (int bb = 0; bb < kTileBufs; ++bb) tc::mbar_init(&mbar[bb], 1);
    for (int r = 0; r < kRawStages; ++r) tc::mbar_init(&rbar[r], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, kTmemCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  // one MMA per operand half and 16 pixels: A = H (or L), 128 bands; B = the H
  // and L tiles together (they are adjacent with the same 8-row stride), N =
  // 256, so that columns 0-127 hold H.H^T (or L.H^T) and 128-255 H.L^T (or
  // L.L^T): two MMAs of N = 256 instead of four of N = 112
  const uint32_t id = tc::idesc(1, kRows, 2 * kRows);
  const int nchunk = (W + kKC - 1) / kKC;
  // this CTA's lines and chunks: whole lines blockIdx.x, blockIdx.x + gridDim.x,
  // ... (split 1), or the chunks c0, c0 + split, ... of line blockIdx.x / split
  const int c0 = split > 1 ? (int)blockIdx.x % split : 0, cs = split > 1 ? split : 1;
  const int nch = c0 < nchunk ? (nchunk - c0 + cs - 1) / cs : 0;
  const int nlines = split > 1 ? ((int)blockIdx.x / split < T ? 1 : 0)
                   : (blockIdx.x < T ? (T - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0);
  const int Q = nlines * nch;
  // even d: an item is a pair of bands (2 m2, 2 m2 + 1) over an 8-pixel group,
  // read as one 32-bit word per pixel, and the row of ones is written apart;
  // odd d: an item is one band (the row of ones, m = d, among them)
  const bool pairs = (d & 1) == 0;
  const int dh = d >> 1;
  const int items = pairs ? dh * (kKC / 8) : (d + 1) * (kKC / 8);
  auto line_of = [&](int q) {
    return split > 1 ? (int)blockIdx.x / split : (int)blockIdx.x + (q / nch) * (int)gridDim.x;
  };
  // chunk q of this CTA: the (q % nch)-th of its chunks of line line_of(q)
  auto issue = [&](int q) {
    if (q >= Q) return;
    const int slot = q % kRawStages;
    const int t = line_of(q), ci = c0 + (q % nch) * cs;
    const int npx = min(kKC, W - ci * kKC);
    const uint32_t bytes = (uint32_t)npx * (uint32_t)d * 2u;
    tc::mbar_expect_tx(&rbar[slot], bytes);
    tc::bulk_g2s(raw + slot * kRawBytes, X + (int64_t)t * line_stride + (int64_t)ci * kKC * d,
                 bytes, &rbar[slot]);
  };
  if (tid == kConv)
    for (int q = 0; q < kRawStages; ++q) issue(q);
  // this converter's items: band m, pixel group g
  int im[kMaxItems], ig[kMaxItems], nit = 0;
#pragma unroll
  for (int u = 0; u < kMaxItems; ++u) {
    const int it = tid + u * kConv;
    const int per = pairs ? dh : d + 1;
    im[u] = conv ? it % per : 0;
    ig[u] = conv ? it / per : 0;
    if (conv && it < items) nit = u + 1;
  }
  int issued_raw = min(Q, kRawStages);
  uint32_t issued[kTileBufs] = {}, done[kTileBufs] = {};
  bool timed_out = false, bad = false;
  int q = 0;
  for (; q < Q && !timed_out; ++q) {
    const int t = line_of(q), k = q % nch, ci = c0 + k * cs;
    const int b = q % kTileBufs;
    if (issued[b] != done[b]) {
      const bool ok = tc::mbar_wait(&mbar[b], done[b] & 1u, kWaitLimit);
      if (ok) ++done[b];
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
    }
    {
      const bool ok = tc::mbar_wait(&rbar[q % kRawStages], (uint32_t)(q / kRawStages) & 1u,
                                    kWaitLimit);
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
    }
    const uint16_t* rw = reinterpret_cast<const uint16_t*>(raw + (q % kRawStages) * kRawBytes);
    unsigned char* tH = sm + b * 2 * kTileBytes;
    unsigned char* tL = tH + kTileBytes;
    const int npx = min(kKC, W - ci * kKC);
    if (pairs) {
      const uint32_t* rw32 = reinterpret_cast<const uint32_t*>(rw);
      const uint32_t rmask = ~(maxv | (maxv << 16));
      const bool full = npx == kKC;
#pragma unroll
      for (int u = 0; u < kMaxItems; ++u) {
        if (u >= nit) break;
        const int m2 = im[u], g = ig[u];
        uint32_t w[8], orv = 0u;
#pragma unroll
        for (int k8 = 0; k8 < 8; ++k8) {
          const int px = g * 8 + k8;
          w[k8] = (full || px < npx) ? rw32[px * dh + m2] : 0u;
          orv |= w[k8];
        }
        bad |= (orv & rmask) != 0u;
        uint32_t hA[4], lA[4], hB[4], lB[4];   // bands 2 m2 (A) and 2 m2 + 1 (B)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const uint32_t ta = __byte_perm(w[2 * k2], w[2 * k2 + 1], 0x5410);   // pixels 2k2, 2k2+1
          const uint32_t tb = __byte_perm(w[2 * k2], w[2 * k2 + 1], 0x7632);
          hA[k2] = bf16x2_small((ta >> 6) & 0x003F003Fu);
          lA[k2] = bf16x2_small(ta & 0x003F003Fu);
          hB[k2] = bf16x2_small((tb >> 6) & 0x003F003Fu);
          lB[k2] = bf16x2_small(tb & 0x003F003Fu);
        }
        const uint32_t oA = tile_off(2 * m2, g), oB = tile_off(2 * m2 + 1, g);
        *reinterpret_cast<uint4*>(tH + oA) = make_uint4(hA[0], hA[1], hA[2], hA[3]);
        *reinterpret_cast<uint4*>(tL + oA) = make_uint4(lA[0], lA[1], lA[2], lA[3]);
        *reinterpret_cast<uint4*>(tH + oB) = make_uint4(hB[0], hB[1], hB[2], hB[3]);
        *reinterpret_cast<uint4*>(tL + oB) = make_uint4(lB[0], lB[1], lB[2], lB[3]);
      }
      if (tid < kKC / 8) {   // the row of ones (band d): 1 = 64 * 0 + 1
        const int g = tid;
        uint32_t lv[4];
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const int px = g * 8 + 2 * k2;
          lv[k2] = (px < npx ? 0x3F80u : 0u) | (px + 1 < npx ? 0x3F800000u : 0u);
        }
        const uint32_t off = tile_off(d, g);
        *reinterpret_cast<uint4*>(tH + off) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(tL + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
      }
    } else {
#pragma unroll
    for (int u = 0; u < kMaxItems; ++u) {
      if (u >= nit) break;
      const int m = im[u], g = ig[u];
      uint32_t hv[4], lv[4];
#pragma unroll
      for (int qq = 0; qq < 8; qq += 2) {
        uint32_t v[2];
#pragma unroll
        for (int u2 = 0; u2 < 2; ++u2) {
          const int px = g * 8 + qq + u2;
          uint32_t sv = 0u;
          if (px < npx) sv = (m < d) ? (uint32_t)rw[px * d + m] : 1u;
          bad |= (m < d) && (sv > maxv);
          v[u2] = sv;
        }
        hv[qq / 2] = bf16_pair(v[0] >> 6, v[1] >> 6);
        lv[qq / 2] = bf16_pair(v[0] & 63u, v[1] & 63u);
      }
      const uint32_t off = tile_off(m, g);
      *reinterpret_cast<uint4*>(tH + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
      *reinterpret_cast<uint4*>(tL + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == kConv) {
      const uint32_t aH = tc::smem_u32(tH), aL = tc::smem_u32(tL);
#pragma unroll
      for (int s2 = 0; s2 < kKC / 16; ++s2) {
        const uint32_t ko = (uint32_t)s2 * 2u * kLBO;
        const uint64_t dH = tc::desc(aH + ko, kLBO, kSBO);
        const uint64_t dL = tc::desc(aL + ko, kLBO, kSBO);
        const uint32_t acc = (k > 0 || s2 > 0) ? 1u : 0u;
        tc::mma_bf16(tmem, dH, dH, id, acc);                  // HH | HL
        tc::mma_bf16(tmem + 2 * kRows, dL, dH, id, acc);      // LH | LL
      }
      tc::commit(&mbar[b]);
      issue(q + kRawStages);      // this chunk's raw slot is free: every thread converted it
    }
    issued_raw = min(Q, q + 1 + kRawStages);
    ++issued[b];
    if (k != nch - 1) continue;
    // end of line t: range flag, wait for its MMAs, drain
    if (__syncthreads_or(bad)) {
      if (tid == 0) atomicMin(&err[kErrRange], (unsigned long long)(t0 + t));
    }
    bad = false;
    for (int bb = 0; bb < kTileBufs; ++bb) {
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
    const int m = 32 * (warp & 3) + lane;
    uint64_t* s2p = S2 + (int64_t)t * d * d;
    for (int c0 = (warp >> 2) * 16; conv && c0 < np; c0 += 32) {
      uint32_t hh[16], hl[16], lh[16], ll[16];
      const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
      tc::tmem_ld16(lane_base, hh);
      tc::tmem_ld16(lane_base + kRows, hl);
      tc::tmem_ld16(lane_base + 2 * kRows, lh);
      tc::tmem_ld16(lane_base + 3 * kRows, ll);
      tc::tmem_ld_wait();
      if (m < d) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c0 + j;
          if (n > m && n != d) continue;        // upper triangle: not needed
          // each accumulator holds an exact integer below 2^24: convert through u32
          const uint64_t v = ((uint64_t)__float2uint_rz(__uint_as_float(hh[j])) << 12) +
                             (((uint64_t)__float2uint_rz(__uint_as_float(hl[j])) +
                               (uint64_t)__float2uint_rz(__uint_as_float(lh[j]))) << 6) +
                             (uint64_t)__float2uint_rz(__uint_as_float(ll[j]));
          uint64_t* o = nullptr;
          if (n < d) {
            if (n <= m) o = s2p + (int64_t)m * d + n;
          } else if (n == d) {
            o = S1 + (int64_t)t * d + m;
          }
          if (o) {
            if (split > 1)
              atomicAdd(reinterpret_cast<unsigned long long*>(o), (unsigned long long)v);
            else
              *o = v;
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
      tc::mbar_wait(&rbar[r % kRawStages], (uint32_t)(r / kRawStages) & 1u, kWaitLimit);
    for (int bb = 0; bb < kTileBufs; ++bb)
      if (issued[bb] != done[bb]) tc::mbar_wait(&mbar[bb], done[bb] & 1u, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, kTmemCols);
}

}  // namespace

bool stats_tc_supported(int d, int W, int bits) {
  return d + 1 <= kRows && W <= 2048 && bits <= 12;
}

cudaError_t configure_stats_tc_kernel() {
  cudaError_t e =
      cudaFuncSetAttribute(stats_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stats_tc_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBulkSmem);
  return e;
}

void launch_stats_tc(const uint16_t* x, int64_t line_stride, int W, int d, uint32_t maxv, int T,
                     int n_sm, uint64_t* S1, uint64_t* S2, unsigned long long* err, int64_t t0,
                     cudaStream_t st) {
  const int grid = T < n_sm ? T : n_sm;
  const bool aligned = ((uintptr_t)x % 16 == 0) && ((line_stride * 2) % 16 == 0) &&
                       (((int64_t)W * d * 2) % 16 == 0);
  // fewer lines than half the SMs: split each line's chunks over the idle SMs
  const int nchunk = (W + kKC - 1) / kKC;
  const int split = aligned && 2 * T <= n_sm ? std::min(nchunk, n_sm / T) : 1;
  if (split > 1) {
    cudaMemsetAsync(S2, 0, (size_t)T * d * d * sizeof(uint64_t), st);
    cudaMemsetAsync(S1, 0, (size_t)T * d * sizeof(uint64_t), st);
    stats_tc_bulk_kernel<<<T * split, kBulkThreads, kBulkSmem, st>>>(x, line_stride, W, d, maxv,
                                                                     T, S1, S2, err, t0, split);
  } else if (aligned)
    stats_tc_bulk_kernel<<<grid, kBulkThreads, kBulkSmem, st>>>(x, line_stride, W, d, maxv, T, S1,
                                                                S2, err, t0, 1);
  else
    stats_tc_kernel<<<grid, kThreads, kSmemBytes, st>>>(x, line_stride, W, d, maxv, T, S1, S2,
                                                        err, t0);
}

}  // namespace erx
